// C ABI of libmd: contexts, state I/O, the integrator schedule, observables.
//
// Integrator (Sec. 3, Eq. 4 and its step list, items 1-12): a step is
//   kick(B0) drift(D0) kick(B1) drift(D1) kick(B1) drift(D0) kick(B0)
// with kick p += b dt f(q) and drift q += d dt p.  Each "stage" kernel fuses
// one force evaluation with the kick that uses it and the drift that follows,
// so a step is three stage launches.  The closing kick of a step and the opening
// kick of the next use the same force (item 12), so inside md_step they merge
// into one kick with 2 B0; md_step ends with a kick-only stage that leaves p on
// the step boundary and keeps that force for the next call.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>
#include <unordered_map>

#include "md_internal.cuh"

namespace {

thread_local std::string g_err;
thread_local int g_status = 0;  // status code of this thread's last failure
std::mutex g_alloc_mu;
void *(*g_alloc)(size_t, void *) = nullptr;
void (*g_free)(void *, void *) = nullptr;
void *g_alloc_user = nullptr;

int fail_global(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  g_status = code;
  return code;
}

bool is_finite(double x) { return x == x && x - x == 0.0; }

}  // namespace

int set_err(md_ctx *c, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  g_err = buf;
  g_status = code;
  return code;
}

int cuda_err(md_ctx *c, cudaError_t e, const char *what) {
  return set_err(c, MD_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

// Each block remembers the allocator that made it (host-side registry), so a
// block made before md_set_allocator is released by the allocator that made it.
namespace {
struct AllocRec {
  void (*free_fn)(void *, void *);
  void *user;
};
std::unordered_map<void *, AllocRec> g_blocks;
}  // namespace

void *dev_alloc(size_t bytes) {
  if (bytes == 0) bytes = 16;
  // the hook is called outside the lock (a caller's allocator may itself allocate
  // through this library or take locks of its own); only the registry is guarded
  void *(*alloc)(size_t, void *);
  void (*free_fn)(void *, void *);
  void *user;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    alloc = g_alloc;
    free_fn = g_free;
    user = g_alloc_user;
  }
  void *ptr = nullptr;
  if (alloc) {
    ptr = alloc(bytes, user);
    if (!ptr) return nullptr;
    if ((reinterpret_cast<uintptr_t>(ptr) & 255u) != 0) {  // the kernels' vector loads need 256 B
      free_fn(ptr, user);
      return nullptr;
    }
  } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_blocks[ptr] = AllocRec{alloc ? free_fn : nullptr, alloc ? user : nullptr};
  return ptr;
}

void dev_free(void *p) {
  if (!p) return;
  AllocRec r{nullptr, nullptr};
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    auto it = g_blocks.find(p);
    if (it == g_blocks.end()) return;
    r = it->second;
    g_blocks.erase(it);
  }
  if (r.free_fn) {
    // cudaFree waits for the device; a caching allocator may hand the block out at
    // once, so finish every queued kernel that may still read it first
    cudaDeviceSynchronize();
    r.free_fn(p, r.user);
  } else {
    cudaFree(p);
  }
}

void yoshida_coefficients(double c[4]) {
  const double t = cbrt(2.0);
  const double w1 = 1.0 / (2.0 - t), w0 = -t / (2.0 - t);
  c[0] = 0.5 * w1;         // B0
  c[1] = 0.5 * (w0 + w1);  // B1
  c[2] = w1;               // D0
  c[3] = w0;               // D1
}

md_ctx *create_context(int model, int64_t N, int64_t n_total, int64_t row0, double eps, double dt, uint64_t seed,
                       const char *who) {
  if (model != MD_HMF && model != MD_RING && model != MD_GRAV2D && model != MD_GRAV3D && model != MD_SHEET1D) {
    fail_global(MD_EINVAL, "%s: unknown model %d", who, model);
    return nullptr;
  }
  if (n_total < 1 || n_total > (int64_t)1 << 40) {
    fail_global(MD_EINVAL, "%s: N must be in [1, 2^40], got %lld", who, (long long)n_total);
    return nullptr;
  }
  if (N < 1 || row0 < 0 || row0 + N > n_total) {
    fail_global(MD_EINVAL, "%s: rows [%lld, %lld) outside [0, %lld)", who, (long long)row0, (long long)(row0 + N),
                (long long)n_total);
    return nullptr;
  }
  const bool eps0_ok = model == MD_HMF || model == MD_SHEET1D;  // models with no divergence at eps = 0
  if (!eps_valid(model, eps)) {
    fail_global(MD_EINVAL, "%s: eps must be finite and %s %g, got %g", who, eps0_ok ? "0 or >=" : ">=", kEpsMin,
                eps);
    return nullptr;
  }
  if (!is_finite(dt)) {
    fail_global(MD_EINVAL, "%s: dt must be finite", who);
    return nullptr;
  }
  md_ctx *c = new (std::nothrow) md_ctx();
  if (!c) {
    fail_global(MD_ENOMEM, "md_init: host allocation");
    return nullptr;
  }
  c->model = model;
  c->dim = model == MD_GRAV2D ? 2 : model == MD_GRAV3D ? 3 : 1;
  c->N = N;
  c->n_total = n_total;
  c->row0 = row0;
  c->eps = eps;
  c->dt = dt;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cuda_err(c, e, "md_init: device setup");
    cudaGetLastError();
    md_free(c);
    return nullptr;
  }
  c->own_stream = true;
  const size_t nb = sizeof(double) * (size_t)(c->dim * N);
  c->hmf_grid_max = c->nsm * (2048 / kStreamThreads);
  c->q = (double *)dev_alloc(nb);
  c->p = (double *)dev_alloc(nb);
  c->f = (double *)dev_alloc(nb);
  c->hmf_partials = (double *)dev_alloc(sizeof(double) * 4 * c->hmf_grid_max);
  c->hmf_m = (double *)dev_alloc(sizeof(double) * 16);
  c->hmf_ticket = (unsigned *)dev_alloc(sizeof(unsigned) * 4);
  if (!c->q || !c->p || !c->f || !c->hmf_partials || !c->hmf_m || !c->hmf_ticket) {
    set_err(c, MD_ENOMEM, "md_init: device allocation of %zu bytes failed", 3 * nb);
    md_free(c);
    return nullptr;
  }
  if (cudaMallocHost(&c->host_scalars, 16 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    c->host_scalars = nullptr;
    set_err(c, MD_ENOMEM, "md_init: pinned host scalars");
    md_free(c);
    return nullptr;
  }
  if (cudaMemsetAsync(c->hmf_ticket, 0, sizeof(unsigned) * 4, c->stream) != cudaSuccess) {
    cuda_err(c, cudaGetLastError(), "md_init: memset");
    md_free(c);
    return nullptr;
  }
  if (model == MD_HMF && hmf_sincos_table(c, true) != MD_OK) {
    g_err = c->err;
    md_free(c);
    return nullptr;
  }
  const int kind = model == MD_HMF || model == MD_SHEET1D ? MD_IC_WATERBAG
                   : model == MD_RING                    ? MD_IC_RING
                   : model == MD_GRAV2D                  ? MD_IC_DISK
                                                         : MD_IC_BALL;
  if (ic_draw(c, kind, nullptr, seed) != MD_OK || cudaStreamSynchronize(c->stream) != cudaSuccess) {
    g_err = c->err.empty() ? std::string("md_init: initial state") : c->err;
    md_free(c);
    return nullptr;
  }
  return c;
}

// ------------------------------------------------------------------ ABI ---

extern "C" {

const char *md_last_error(const md_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

int md_last_status(void) { return g_status; }

int md_set_allocator(void *(*alloc)(size_t, void *), void (*free_fn)(void *, void *), void *user) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail_global(MD_EINVAL, "md_set_allocator: give both alloc and free, or neither");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_user = user;
  return MD_OK;
}

void md_free(md_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  dev_free(c->q);
  dev_free(c->p);
  dev_free(c->f);
  dev_free(c->hmf_partials);
  dev_free(c->hmf_m);
  dev_free(c->hmf_ticket);
  dev_free(c->hmf_cs);
  dev_free(c->mirror[0]);
  dev_free(c->mirror[1]);
  dev_free(c->sk_slots);
  dev_free(c->sk_tickets);
  dev_free(c->sym_rowfull);
  dev_free(c->sym_colslot);
  dev_free(c->sym_chunks);
  destroy_step_graphs(c);
  dev_free(c->red);
  dev_free(c->gw);
  dev_free(c->shard_sums);
  if (c->shard_event) cudaEventDestroy(c->shard_event);
  if (c->host_scalars) cudaFreeHost(c->host_scalars);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

md_ctx *md_init(int model, int64_t N, double eps, double dt, uint64_t seed) {
  return create_context(model, N, N, 0, eps, dt, seed, "md_init");
}

#define CHECK_CTX(c)                                              \
  do {                                                            \
    if (!(c)) return fail_global(MD_EINVAL, "NULL context");      \
  } while (0)
// calls that need the whole system's state, not one row shard's
#define CHECK_WHOLE(c, what)                                                                          \
  do {                                                                                                \
    if ((c)->shard)                                                                                   \
      return set_err((c), MD_ESTATE, "%s: not defined on a row shard (use the md_shard_* calls)", what); \
  } while (0)

int md_set_precision(md_ctx *c, int prec) {
  CHECK_CTX(c);
  if (prec != MD_FP64 && prec != MD_MIXED) return set_err(c, MD_EINVAL, "unknown precision %d", prec);
  c->prec = prec;
  return MD_OK;
}

int md_set_stream(md_ctx *c, void *stream) {
  CHECK_CTX(c);
  MD_CUDA(c, cudaStreamSynchronize(c->stream));
  if (c->own_stream) cudaStreamDestroy(c->stream);
  c->stream = (cudaStream_t)stream;
  c->own_stream = false;
  return MD_OK;
}

int md_set_dt(md_ctx *c, double dt) {
  CHECK_CTX(c);
  if (!is_finite(dt)) return set_err(c, MD_EINVAL, "dt must be finite");
  c->dt = dt;
  return MD_OK;
}

int md_set_tuning(md_ctx *c, const char *key, int64_t value) {
  CHECK_CTX(c);
  if (!key) return set_err(c, MD_EINVAL, "NULL key");
  std::string k(key);
  if (k == "r_mixed" && (value == 4 || value == 8)) c->pt.r_mixed = (int)value;
  else if (k == "r_fp64" && (value == 2 || value == 4)) c->pt.r_fp64 = (int)value;
  else if (k == "pair_ctas_per_sm" && value >= 0 && value <= 32) c->pt.ctas_per_sm = (int)value;
  else if (k == "pair_vcta" && value >= 0 && value <= 32) c->pt.vcta = (int)value;
  else if (k == "hmf_ctas_per_sm" && value >= 0 && value <= 32) c->ht.ctas_per_sm = (int)value;
  else if (k == "ring_tc" && value >= 0 && value <= 2) c->pt.ring_tc = (int)value;
  else if (k == "symmetric" && (value == 0 || value == 1)) c->pt.symmetric = (int)value;
  else if (k == "step_graphs" && (value == 0 || value == 1)) c->use_graphs = value != 0;
  else return set_err(c, MD_EINVAL, "unknown tuning key or value: %s=%lld", key, (long long)value);
  return MD_OK;
}

int md_set_ic(md_ctx *c, int kind, const double *params, uint64_t seed) {
  CHECK_CTX(c);
  return ic_draw(c, kind, params, seed);
}

static int invalidate(md_ctx *c) {
  c->fsal_valid = false;
  c->hmf_m_valid = false;
  c->mirror_valid = false;
  c->shard_primed = false;
  return MD_OK;
}

int md_set_state(md_ctx *c, const double *q, const double *p) {
  CHECK_CTX(c);
  if (!q || !p) return set_err(c, MD_EINVAL, "md_set_state: NULL array");
  const size_t nb = sizeof(double) * (size_t)(c->dim * c->N);
  MD_CUDA(c, cudaMemcpyAsync(c->q, q, nb, cudaMemcpyHostToDevice, c->stream));
  MD_CUDA(c, cudaMemcpyAsync(c->p, p, nb, cudaMemcpyHostToDevice, c->stream));
  MD_CUDA(c, cudaStreamSynchronize(c->stream));
  return invalidate(c);
}

int md_get_state(md_ctx *c, double *q, double *p) {
  CHECK_CTX(c);
  const size_t nb = sizeof(double) * (size_t)(c->dim * c->N);
  if (q) MD_CUDA(c, cudaMemcpyAsync(q, c->q, nb, cudaMemcpyDeviceToHost, c->stream));
  if (p) MD_CUDA(c, cudaMemcpyAsync(p, c->p, nb, cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(c, cudaStreamSynchronize(c->stream));
  return MD_OK;
}

int md_set_state_device(md_ctx *c, const double *q, const double *p) {
  CHECK_CTX(c);
  if (!q || !p) return set_err(c, MD_EINVAL, "md_set_state_device: NULL array");
  const size_t nb = sizeof(double) * (size_t)(c->dim * c->N);
  MD_CUDA(c, cudaMemcpyAsync(c->q, q, nb, cudaMemcpyDeviceToDevice, c->stream));
  MD_CUDA(c, cudaMemcpyAsync(c->p, p, nb, cudaMemcpyDeviceToDevice, c->stream));
  return invalidate(c);
}

int md_get_state_device(md_ctx *c, double *q, double *p) {
  CHECK_CTX(c);
  const size_t nb = sizeof(double) * (size_t)(c->dim * c->N);
  if (q) MD_CUDA(c, cudaMemcpyAsync(q, c->q, nb, cudaMemcpyDeviceToDevice, c->stream));
  if (p) MD_CUDA(c, cudaMemcpyAsync(p, c->p, nb, cudaMemcpyDeviceToDevice, c->stream));
  return MD_OK;
}

int md_step(md_ctx *c, int64_t nsteps) {
  CHECK_CTX(c);
  CHECK_WHOLE(c, "md_step");
  if (nsteps < 0) return set_err(c, MD_EINVAL, "md_step: nsteps < 0");
  return integrate(c, nsteps);
}

}  // extern "C"

namespace {

constexpr int kStepGraphSteps = 8;  // even: every stage flips the ping-pong parity, 3 per step

// One step after the first: (2 B0, D0) (B1, D1) (B1, D0), kick-drift stages.
int middle_step(md_ctx *c, const double *k, double h) {
  int rc;
  if (c->model == MD_HMF) {
    if ((rc = hmf_stage(c, STAGE_KICK_DRIFT, 2.0 * k[0] * h, k[2] * h, nullptr))) return rc;
    if ((rc = hmf_stage(c, STAGE_KICK_DRIFT, k[1] * h, k[3] * h, nullptr))) return rc;
    return hmf_stage(c, STAGE_KICK_DRIFT, k[1] * h, k[2] * h, nullptr);
  }
  if ((rc = pair_stage(c, STAGE_KICK_DRIFT, 2.0 * k[0] * h, k[2] * h, nullptr))) return rc;
  if ((rc = pair_stage(c, STAGE_KICK_DRIFT, k[1] * h, k[3] * h, nullptr))) return rc;
  return pair_stage(c, STAGE_KICK_DRIFT, k[1] * h, k[2] * h, nullptr);
}

StepGraphKey step_key_of(const md_ctx *c, double h) {
  StepGraphKey key;
  memset((void *)&key, 0, sizeof key);  // padding bytes too: keys are compared with memcmp
  key.model = c->model;
  key.prec = c->prec;
  key.N = c->N;
  key.h = h;
  key.eps = c->eps;
  key.stream = (void *)c->stream;
  key.pt = c->pt;
  key.ht = c->ht;
  key.mirror_fmt = c->mirror_fmt;
  const void *b[14] = {c->q,           c->p,          c->mirror[0],    c->mirror[1], c->sk_slots,
                       c->sk_tickets,  c->sym_rowfull, c->sym_colslot, c->sym_chunks, c->hmf_partials,
                       c->hmf_m,       c->hmf_ticket, c->f,            c->hmf_cs};
  memcpy(key.bufs, b, sizeof b);
  return key;
}

int parity_of(const md_ctx *c) { return c->model == MD_HMF ? c->hmf_cur : c->mirror_cur; }

// Graphs are captured only on a stream of our own choosing that is not already
// being captured: the legacy and per-thread default streams cannot be captured,
// and inside a caller's capture the stages are simply recorded into it.
bool graphs_usable(md_ctx *c) {
  if (!c->use_graphs || c->stream == nullptr || c->stream == cudaStreamLegacy || c->stream == cudaStreamPerThread)
    return false;
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(c->stream, &st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return st == cudaStreamCaptureStatusNone;
}

// kStepGraphSteps middle steps from the graph of the current parity, captured on
// first use and again whenever anything the launches depend on has changed.
// Every kernel it holds has already run once in this call (the first step), so
// capture loads no module and allocates nothing.
int replay_steps(md_ctx *c, const double *k, double h) {
  const int par = parity_of(c);
  const StepGraphKey key = step_key_of(c, h);
  if (c->step_graph[par] && memcmp(&key, &c->step_key[par], sizeof key) != 0) {
    cudaGraphExecDestroy(c->step_graph[par]);
    c->step_graph[par] = nullptr;
  }
  if (!c->step_graph[par]) {
    MD_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
    const int64_t l0 = c->launches;
    int rc = MD_OK;
    for (int g = 0; g < kStepGraphSteps && rc == MD_OK; g++) rc = middle_step(c, k, h);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    c->step_graph_launches[par] = c->launches - l0;
    c->launches = l0;
    if (rc != MD_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      c->mirror_valid = c->hmf_m_valid = false;  // host-side parity no longer matches the device
      return rc != MD_OK ? rc : cuda_err(c, e, "md_step: graph capture");
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->step_graph[par], graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      c->step_graph[par] = nullptr;
      return cuda_err(c, ei, "md_step: graph instantiate");
    }
    c->step_key[par] = key;
  }
  MD_CUDA(c, cudaGraphLaunch(c->step_graph[par], c->stream));
  c->launches += c->step_graph_launches[par];
  return MD_OK;
}

}  // namespace

void destroy_step_graphs(md_ctx *c) {
  for (int k = 0; k < 2; k++)
    if (c->step_graph[k]) {
      cudaGraphExecDestroy(c->step_graph[k]);
      c->step_graph[k] = nullptr;
    }
}

// md_step's body: step 1 (whose first kick is B0, or comes from the cached
// force), steps 2..n with the merged 2 B0 kicks (blocks of kStepGraphSteps from
// CUDA graphs), and the closing B0 kick whose force is kept (first-same-as-last).
int integrate(md_ctx *c, int64_t nsteps) {
  if (nsteps == 0) return MD_OK;
  double k[4];
  yoshida_coefficients(k);
  const double h = c->dt, B0 = k[0], B1 = k[1], D0 = k[2], D1 = k[3];
  int rc;
  if (c->model == MD_HMF) {
    if ((rc = hmf_stage(c, STAGE_KICK_DRIFT, B0 * h, D0 * h, nullptr))) return rc;
    if ((rc = hmf_stage(c, STAGE_KICK_DRIFT, B1 * h, D1 * h, nullptr))) return rc;
    if ((rc = hmf_stage(c, STAGE_KICK_DRIFT, B1 * h, D0 * h, nullptr))) return rc;
  } else {
    const bool cached = c->fsal_valid && c->fsal_prec == c->prec && c->mirror_valid && c->mirror_prec == c->prec;
    c->fsal_valid = false;
    rc = cached ? kick_drift_cached(c, B0 * h, D0 * h) : pair_stage(c, STAGE_KICK_DRIFT, B0 * h, D0 * h, nullptr);
    if (rc) return rc;
    if ((rc = pair_stage(c, STAGE_KICK_DRIFT, B1 * h, D1 * h, nullptr))) return rc;
    if ((rc = pair_stage(c, STAGE_KICK_DRIFT, B1 * h, D0 * h, nullptr))) return rc;
  }
  int64_t rest = nsteps - 1;
  if (rest >= kStepGraphSteps && graphs_usable(c))
    for (; rest >= kStepGraphSteps; rest -= kStepGraphSteps)
      if ((rc = replay_steps(c, k, h))) return rc;
  for (; rest > 0; rest--)
    if ((rc = middle_step(c, k, h))) return rc;
  if (c->model == MD_HMF) return hmf_stage(c, STAGE_KICK_ONLY, B0 * h, 0.0, nullptr);
  if ((rc = pair_stage(c, STAGE_KICK_ONLY, B0 * h, 0.0, c->f))) return rc;
  c->fsal_valid = true;
  c->fsal_prec = c->prec;
  return MD_OK;
}

extern "C" {

void md_yoshida(double *c4) {
  if (c4) yoshida_coefficients(c4);
}

int md_stage(md_ctx *c, double b, double d) {
  CHECK_CTX(c);
  CHECK_WHOLE(c, "md_stage");
  if (!is_finite(b) || !is_finite(d)) return set_err(c, MD_EINVAL, "md_stage: non-finite coefficient");
  const double h = c->dt;
  if (c->model == MD_HMF)
    return d == 0.0 ? hmf_stage(c, STAGE_KICK_ONLY, b * h, 0.0, nullptr)
                    : hmf_stage(c, STAGE_KICK_DRIFT, b * h, d * h, nullptr);
  if (d == 0.0) {
    int rc = pair_stage(c, STAGE_KICK_ONLY, b * h, 0.0, c->f);
    if (rc) return rc;
    c->fsal_valid = true;
    c->fsal_prec = c->prec;
    return MD_OK;
  }
  c->fsal_valid = false;
  return pair_stage(c, STAGE_KICK_DRIFT, b * h, d * h, nullptr);
}

int md_force_device(md_ctx *c, double *f) {
  CHECK_CTX(c);
  CHECK_WHOLE(c, "md_force");
  if (!f) return set_err(c, MD_EINVAL, "md_force_device: NULL output");
  if (c->model == MD_HMF) return hmf_stage(c, STAGE_FORCE_ONLY, 0.0, 0.0, f);
  return pair_stage(c, STAGE_FORCE_ONLY, 0.0, 0.0, f);
}

int md_force(md_ctx *c, double *f) {
  CHECK_CTX(c);
  CHECK_WHOLE(c, "md_force");
  if (!f) return set_err(c, MD_EINVAL, "md_force: NULL output");
  int rc = md_force_device(c, c->f);
  if (rc) return rc;
  if (c->model != MD_HMF) {
    c->fsal_valid = true;
    c->fsal_prec = c->prec;
  }
  const size_t nb = sizeof(double) * (size_t)(c->dim * c->N);
  MD_CUDA(c, cudaMemcpyAsync(f, c->f, nb, cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(c, cudaStreamSynchronize(c->stream));
  return MD_OK;
}

int md_energy(md_ctx *c, double *K, double *V) {
  CHECK_CTX(c);
  CHECK_WHOLE(c, "md_energy");
  int rc;
  double *d = c->hmf_m + 8;  // device scalars [8..11]
  if ((rc = kinetic_fp64(c, d))) return rc;
  if (c->model == MD_HMF) {
    if ((rc = hmf_sums_fp64(c, d + 2))) return rc;
  } else {
    if ((rc = pair_potential_fp64(c, d + 1))) return rc;
  }
  MD_CUDA(c, cudaMemcpyAsync(c->host_scalars, d, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(c, cudaStreamSynchronize(c->stream));
  const double n = (double)c->N;
  const double kin = c->host_scalars[0];
  double pot;
  if (c->model == MD_HMF) {
    const double mx = c->host_scalars[2] / n, my = c->host_scalars[3] / n;
    pot = 0.5 * n * (1.0 - mx * mx - my * my);  // Eq. 5
  } else if (c->model == MD_RING) {
    pot = -c->host_scalars[1] / (2.0 * n);  // Eq. 1 with 1 - cos + eps = 2 (sin^2(d/2) + eps/2)
  } else if (c->model == MD_GRAV3D) {
    pot = -c->host_scalars[1] / n;  // softened 3D gravitational potential
  } else if (c->model == MD_SHEET1D) {
    pot = c->host_scalars[1] / n;  // 1D sheets: (1/N) sum_{i<j} |x_i - x_j| (softened for eps > 0)
  } else {
    pot = c->host_scalars[1] / n;  // Eq. 3
  }
  if (K) *K = kin;
  if (V) *V = pot;
  if (!is_finite(kin) || !is_finite(pot)) return set_err(c, MD_ENONFINITE, "md_energy: non-finite energy (K=%g, V=%g)", kin, pot);
  return MD_OK;
}

int md_magnetization(md_ctx *c, double *mx, double *my) {
  CHECK_CTX(c);
  CHECK_WHOLE(c, "md_magnetization");
  if (c->model != MD_HMF && c->model != MD_RING)
    return set_err(c, MD_EINVAL, "md_magnetization: defined for the HMF and Ring models only");
  double *d = c->hmf_m + 12;
  int rc = hmf_sums_fp64(c, d);
  if (rc) return rc;
  MD_CUDA(c, cudaMemcpyAsync(c->host_scalars + 4, d, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(c, cudaStreamSynchronize(c->stream));
  const double n = (double)c->N;
  if (mx) *mx = c->host_scalars[4] / n;
  if (my) *my = c->host_scalars[5] / n;
  if (!is_finite(c->host_scalars[4]) || !is_finite(c->host_scalars[5]))
    return set_err(c, MD_ENONFINITE, "md_magnetization: non-finite");
  return MD_OK;
}

int md_synchronize(md_ctx *c) {
  CHECK_CTX(c);
  MD_CUDA(c, cudaStreamSynchronize(c->stream));
  return MD_OK;
}

int64_t md_launch_count(const md_ctx *c) { return c ? c->launches : 0; }

}  // extern "C"
