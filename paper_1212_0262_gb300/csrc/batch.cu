// Batched ensembles of independent Ring / 2D systems of uneven N.
//
// Each integrator stage of every system in the ensemble is one persistent
// launch.  The grid is split into a Ring part and a 2D part (the two models
// have different pair arithmetic); within a part, the (system, i-tile, j-tile)
// units of all its systems form one linear range that is split stream-K style
// across the part's CTAs, so every CTA does the same number of pair
// interactions whatever the spread of N (work per system grows as N^2).  Rows
// (i-tiles) covered by several CTAs are finished by the last contributor, as
// in the single-system kernel.  The Ring/2D split, the register blocking R and
// the CTAs per SM are chosen by md_batch_autotune, which times candidate
// configurations on force-only launches (state untouched).  md_batch_step
// replays a CUDA graph holding a block of steps.
#include <vector>

#include "pairs_impl.cuh"

namespace {

constexpr int kGraphSteps = 10;  // even: three mirror flips per step keep the parity

struct SysDesc {
  double *q, *p, *f;
  const unsigned char *mir[2];
  int64_t N, n_it, n_jt;
  int64_t ubeg;  // first unit of the system in its part
  int64_t rbeg;  // first row (i-tile) of the system in its part
  double epsd, dt;
};

struct PartArgs {
  const SysDesc *sys;
  int nsys;
  int64_t U;
  int P;
  int cur;
  double b, d;
  double *slots;
  unsigned *tickets;
};

// index of the system whose unit range holds u (binary search on ubeg)
__device__ __forceinline__ int sys_of_unit(const PartArgs &A, int64_t u) {
  int lo = 0, hi = A.nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (A.sys[mid].ubeg <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int64_t row_of_unit(const PartArgs &A, int64_t u) {
  const SysDesc &S = A.sys[sys_of_unit(A, u)];
  return S.rbeg + (u - S.ubeg) / S.n_jt;
}

__device__ __forceinline__ PairArgs view(const PartArgs &A, const SysDesc &S) {
  PairArgs v{};
  v.mirror_in = S.mir[A.cur];
  v.mirror_out = (void *)S.mir[1 - A.cur];
  v.q = S.q;
  v.p = S.p;
  v.fout = S.f;
  v.N = S.N;
  v.epsd = S.epsd;
  v.kick = A.b * S.dt;
  v.drift = A.d * S.dt;
  return v;
}

// Not inlined: the Ring and 2D parts then get separate register allocations.
template <class Pol, int MODEL, bool MIXED, int MODE>
__device__ __noinline__ void batch_part(const PartArgs &A, int64_t cta) {
  constexpr int R = Pol::R, TJ = Pol::TJ, NACC = Pol::NACC;
  constexpr int TILE_BYTES = TJ * Pol::JB;
  constexpr int CHUNKS = TILE_BYTES / 16;
  constexpr int64_t TI = (int64_t)NT * R;
  __shared__ __align__(16) unsigned char sbuf[2][TILE_BYTES];
  __shared__ bool s_last;

  const int64_t u0 = unit_begin(A.U, A.P, cta), u1 = unit_begin(A.U, A.P, cta + 1);
  if (u0 >= u1) return;
  const int64_t first_row = row_of_unit(A, u0);
  int s = sys_of_unit(A, u0);
  int64_t it = (u0 - A.sys[s].ubeg) / A.sys[s].n_jt, jt = (u0 - A.sys[s].ubeg) % A.sys[s].n_jt;
  bool row_from_start = (jt == 0);

  auto prefetch = [&](int buf, int sp, int64_t jtp) {
    const unsigned char *src = A.sys[sp].mir[A.cur] + jtp * (int64_t)TILE_BYTES;
    for (int ch = threadIdx.x; ch < CHUNKS; ch += NT) cp_async16(&sbuf[buf][ch * 16], src + ch * 16);
    cp_async_commit();
  };

  typename Pol::State st;
  PairArgs v = view(A, A.sys[s]);
  int64_t i0 = it * TI;  // tile base; each thread's rows come from Pol::row_of
  Pol::load(st, v.mirror_in, i0);
  prefetch(0, s, jt);

  for (int64_t u = u0; u < u1; u++) {
    const int buf = (int)((u - u0) & 1);
    if (u + 1 < u1) {
      int sn = s;
      int64_t jn = jt + 1;
      if (jn == A.sys[s].n_jt) {
        jn = 0;
        if (it + 1 == A.sys[s].n_it) sn = s + 1;
      }
      prefetch(buf ^ 1, sn, jn);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int64_t j0 = jt * TJ;
    const bool diag = Pol::MASK && (j0 < it * TI + TI) && (it * TI < j0 + TJ);
    if (diag)
      Pol::template tile<true>(st, sbuf[buf], v, i0, j0);
    else
      Pol::template tile<false>(st, sbuf[buf], v, i0, j0);
    __syncthreads();
    jt++;
    const bool row_end = (jt == A.sys[s].n_jt);
    if (row_end || u + 1 == u1) {
      const int64_t row = A.sys[s].rbeg + it;
      if (row_end && row_from_start) {
#pragma unroll
        for (int r = 0; r < Pol::NR; r++) {
          double ex[NACC];
          Pol::total(st, r, ex);
          const int lr = Pol::row_of(r);  // row offset in the tile, -1: another lane's
          if (lr >= 0) finish<Pol, MODEL, MIXED, MODE>(v, i0 + lr, ex);
        }
      } else {
        const int slot = (row == first_row) ? 0 : 1;
        double *sp = A.slots + ((cta * 2 + slot) * NACC) * TI;
#pragma unroll
        for (int r = 0; r < Pol::NR; r++) {
          double ex[NACC];
          Pol::total(st, r, ex);
          const int lr = Pol::row_of(r);  // row offset in the tile, -1: another lane's
          if (lr >= 0)
#pragma unroll
            for (int d = 0; d < NACC; d++) sp[d * TI + lr] = ex[d];
        }
        __threadfence();
        __syncthreads();
        const int64_t ub = A.sys[s].ubeg + it * A.sys[s].n_jt;
        const int64_t cf = cta_of_unit(A.U, A.P, ub);
        const int64_t cl = cta_of_unit(A.U, A.P, ub + A.sys[s].n_jt - 1);
        if (threadIdx.x == 0) {
          unsigned cnt = atomicAdd(&A.tickets[row], 1u) + 1u;
          s_last = (cnt == (unsigned)(cl - cf + 1));
        }
        __syncthreads();
        if (s_last) {
          __threadfence();
          double tot[Pol::NR][NACC];
#pragma unroll
          for (int r = 0; r < Pol::NR; r++)
#pragma unroll
            for (int d = 0; d < NACC; d++) tot[r][d] = 0.0;
          for (int64_t c2 = cf; c2 <= cl; c2++) {
            const int sl = (row == row_of_unit(A, unit_begin(A.U, A.P, c2))) ? 0 : 1;
            const double *src = A.slots + ((c2 * 2 + sl) * NACC) * TI;
#pragma unroll
            for (int r = 0; r < Pol::NR; r++) {
              const int lr = Pol::row_of(r);  // row offset in the tile, -1: another lane's
              if (lr >= 0)
#pragma unroll
                for (int d = 0; d < NACC; d++) tot[r][d] += __ldcg(src + d * TI + lr);
            }
          }
#pragma unroll
          for (int r = 0; r < Pol::NR; r++) {
            const int lr = Pol::row_of(r);  // row offset in the tile, -1: another lane's
            if (lr >= 0) finish<Pol, MODEL, MIXED, MODE>(v, i0 + lr, tot[r]);
          }
          if (threadIdx.x == 0) A.tickets[row] = 0u;
        }
      }
      if (row_end && u + 1 < u1) {
        it++;
        jt = 0;
        row_from_start = true;
        if (it == A.sys[s].n_it) {
          s++;
          it = 0;
          v = view(A, A.sys[s]);
        }
        i0 = it * TI;
        Pol::load(st, v.mirror_in, i0);
      }
    }
  }
}

template <class PolR, class PolG, bool MIXED, int MODE>
__global__ void __launch_bounds__(NT) batch_kernel(PartArgs ring, PartArgs grav) {
  if ((int)blockIdx.x < ring.P)
    batch_part<PolR, MD_RING, MIXED, MODE>(ring, blockIdx.x);
  else
    batch_part<PolG, MD_GRAV2D, MIXED, MODE>(grav, (int64_t)blockIdx.x - ring.P);
}

struct Config {
  int r = 8;            // i-particles per thread (mixed: 4 or 8; FP64: 2)
  double split = 0.5;   // fraction of CTAs given to the Ring part
  int ctas_per_sm = 0;  // 0: occupancy limit
};

}  // namespace

struct md_batch {
  std::vector<md_ctx *> ctx;
  std::vector<int> model;
  int nsys = 0, prec = MD_MIXED, nsm = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int cur = 0;
  bool mirrors_valid = false;
  Config cfg;
  SysDesc *d_sys = nullptr;  // Ring descriptors, then 2D descriptors
  size_t d_sys_count = 0;
  double *slots = nullptr;
  size_t slots_bytes = 0;
  unsigned *tickets = nullptr;
  size_t tickets_count = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_key[2] = {-1, -1};
  // unit / row layout uploaded for tile shape (layout_ti, layout_tj)
  int64_t layout_ti = -1, layout_tj = -1;
  int64_t Ur = 0, Ug = 0, rows_r = 0, rows_g = 0;
  int nr = 0;
  std::vector<std::pair<const void *, int>> occ_cache;  // occupancy per kernel, queried outside captures
  int64_t launches = 0;
  std::string err;
};

namespace {

int berr(md_batch *b, int code, const char *fmt, const char *what) {
  char buf[512];
  snprintf(buf, sizeof buf, fmt, what);
  b->err = buf;
  set_err(nullptr, code, "%s", buf);
  return code;
}

#define B_CUDA(b, call)                                                             \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return berr((b), MD_ECUDA, #call ": %s", cudaGetErrorString(e_)); \
  } while (0)

void drop_graphs(md_batch *b) {
  for (int k = 0; k < 2; k++) {
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    b->graph[k] = nullptr;
    b->graph_key[k] = -1;
  }
}

// Descriptors and the unit / row layout of both parts for tile sizes (TI, TJ).
int build_layout(md_batch *b, int64_t TI, int64_t TJ, std::vector<SysDesc> &hs, int64_t &Ur, int64_t &Ug,
                 int64_t &rows_r, int64_t &rows_g, int &nr) {
  hs.clear();
  Ur = Ug = rows_r = rows_g = 0;
  nr = 0;
  for (int pass = 0; pass < 2; pass++) {
    const int want = pass == 0 ? MD_RING : MD_GRAV2D;
    for (int s = 0; s < b->nsys; s++) {
      if (b->model[s] != want) continue;
      md_ctx *c = b->ctx[s];
      SysDesc d;
      d.q = c->q;
      d.p = c->p;
      d.f = c->f;
      d.mir[0] = (const unsigned char *)c->mirror[0];
      d.mir[1] = (const unsigned char *)c->mirror[1];
      d.N = c->N;
      d.n_it = (c->N + TI - 1) / TI;
      d.n_jt = (c->N + TJ - 1) / TJ;
      d.epsd = want == MD_RING ? 0.5 * c->eps : c->eps;
      d.dt = c->dt;
      int64_t &U = pass == 0 ? Ur : Ug;
      int64_t &rows = pass == 0 ? rows_r : rows_g;
      d.ubeg = U;
      d.rbeg = rows;
      U += d.n_it * d.n_jt;
      rows += d.n_it;
      hs.push_back(d);
      if (pass == 0) nr++;
    }
  }
  return MD_OK;
}

template <class PolR, class PolG, bool MIXED, int MODE>
int launch_batch(md_batch *b, double bc, double dc) {
  constexpr int64_t TI = (int64_t)NT * PolR::R, TJ = PolR::TJ;
  static_assert(PolR::R == PolG::R && PolR::TJ == PolG::TJ, "parts share the tile shape");
  if (b->layout_ti != TI || b->layout_tj != TJ) {
    // (re)build and upload the layout; never inside a stream capture, because the
    // first step of md_batch_step and every autotune trial run uncaptured first
    std::vector<SysDesc> hs;
    build_layout(b, TI, TJ, hs, b->Ur, b->Ug, b->rows_r, b->rows_g, b->nr);
    if (hs.size() > b->d_sys_count) {
      dev_free(b->d_sys);
      b->d_sys = (SysDesc *)dev_alloc(hs.size() * sizeof(SysDesc));
      if (!b->d_sys) return berr(b, MD_ENOMEM, "%s", "batch descriptors");
      b->d_sys_count = hs.size();
    }
    B_CUDA(b, cudaStreamSynchronize(b->stream));  // no launch may still read the old layout
    B_CUDA(b, cudaMemcpy(b->d_sys, hs.data(), hs.size() * sizeof(SysDesc), cudaMemcpyHostToDevice));
    b->layout_ti = TI;
    b->layout_tj = TJ;
  }
  const int64_t Ur = b->Ur, Ug = b->Ug, rows_r = b->rows_r, rows_g = b->rows_g;
  const int nr = b->nr;
  auto kern = batch_kernel<PolR, PolG, MIXED, MODE>;
  int occ = 0;
  for (const auto &kv : b->occ_cache)
    if (kv.first == (const void *)kern) occ = kv.second;
  if (occ == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, 0);
    if (occ < 1) occ = 1;
    b->occ_cache.push_back({(const void *)kern, occ});
  }
  if (b->cfg.ctas_per_sm > 0 && b->cfg.ctas_per_sm < occ) occ = b->cfg.ctas_per_sm;
  const int64_t P = (int64_t)b->nsm * occ;
  int64_t Pr = 0, Pg = 0;
  if (Ur > 0 && Ug > 0) {
    Pr = (int64_t)(b->cfg.split * (double)P + 0.5);
    if (Pr < 1) Pr = 1;
    if (Pr > P - 1) Pr = P - 1;
    Pg = P - Pr;
  } else if (Ur > 0) {
    Pr = P;
  } else {
    Pg = P;
  }
  if (Pr > Ur) Pr = Ur;
  if (Pg > Ug) Pg = Ug;
  // device buffers: slots of both parts, tickets of both parts
  const size_t slot_r = (size_t)Pr * 2 * PolR::NACC * TI, slot_g = (size_t)Pg * 2 * PolG::NACC * TI;
  const size_t need = (slot_r + slot_g) * sizeof(double);
  if (need > b->slots_bytes) {
    dev_free(b->slots);
    b->slots = (double *)dev_alloc(need);
    if (!b->slots) return berr(b, MD_ENOMEM, "%s", "batch slots");
    b->slots_bytes = need;
  }
  const size_t nt = (size_t)(rows_r + rows_g);
  if (nt > b->tickets_count) {
    dev_free(b->tickets);
    b->tickets = (unsigned *)dev_alloc(nt * sizeof(unsigned));
    if (!b->tickets) return berr(b, MD_ENOMEM, "%s", "batch tickets");
    b->tickets_count = nt;
    B_CUDA(b, cudaMemsetAsync(b->tickets, 0, nt * sizeof(unsigned), b->stream));
  }
  PartArgs ar{}, ag{};
  ar.sys = b->d_sys;
  ar.nsys = nr;
  ar.U = Ur;
  ar.P = (int)Pr;
  ag.sys = b->d_sys + nr;
  ag.nsys = b->nsys - nr;
  ag.U = Ug;
  ag.P = (int)Pg;
  ar.cur = ag.cur = b->cur;
  ar.b = ag.b = bc;
  ar.d = ag.d = dc;
  ar.slots = b->slots;
  ag.slots = b->slots + slot_r;
  ar.tickets = b->tickets;
  ag.tickets = b->tickets + rows_r;
  kern<<<(int)(Pr + Pg), NT, 0, b->stream>>>(ar, ag);
  b->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return berr(b, MD_ECUDA, "batch launch: %s", cudaGetErrorString(e));
  if (MODE == STAGE_KICK_DRIFT) b->cur = 1 - b->cur;
  return MD_OK;
}

template <bool MIXED, int MODE>
int dispatch(md_batch *b, double bc, double dc) {
  if constexpr (MIXED) {
    if (b->cfg.r == 4)
      return launch_batch<RingMixed<4, 256, MODE>, GravMixed<4, 256, MODE>, true, MODE>(b, bc, dc);
    return launch_batch<RingMixed<8, 256, MODE>, GravMixed<8, 256, MODE>, true, MODE>(b, bc, dc);
  } else {
    return launch_batch<RingF64<2, 128, MODE>, GravF64<2, 128, MODE>, false, MODE>(b, bc, dc);
  }
}

int stage(md_batch *b, int mode, double bc, double dc) {
  const bool mixed = b->prec == MD_MIXED;
  switch (mode) {
  case STAGE_KICK_DRIFT: return mixed ? dispatch<true, STAGE_KICK_DRIFT>(b, bc, dc) : dispatch<false, STAGE_KICK_DRIFT>(b, bc, dc);
  case STAGE_KICK_ONLY: return mixed ? dispatch<true, STAGE_KICK_ONLY>(b, bc, dc) : dispatch<false, STAGE_KICK_ONLY>(b, bc, dc);
  default: return mixed ? dispatch<true, STAGE_FORCE_ONLY>(b, bc, dc) : dispatch<false, STAGE_FORCE_ONLY>(b, bc, dc);
  }
}

int refresh_mirrors(md_batch *b) {
  if (b->mirrors_valid) return MD_OK;
  for (md_ctx *c : b->ctx) {
    c->prec = b->prec;
    c->pt.ring_tc = 0;  // the batched kernel reads the interleaved records
    c->mirror_cur = b->cur;
    int rc = mirror_refresh(c);
    if (rc) return berr(b, rc, "%s", c->err.c_str());
  }
  b->mirrors_valid = true;
  return MD_OK;
}

}  // namespace

extern "C" {

md_batch *md_batch_init(int nsys, const int *model, const int64_t *N, const double *eps, const double *dt,
                        const uint64_t *seed) {
  if (nsys < 1 || !model || !N || !eps || !dt || !seed) {
    set_err(nullptr, MD_EINVAL, "md_batch_init: need nsys >= 1 and non-NULL arrays");
    return nullptr;
  }
  for (int s = 0; s < nsys; s++)
    if (model[s] != MD_RING && model[s] != MD_GRAV2D) {
      set_err(nullptr, MD_EINVAL, "md_batch_init: system %d: only MD_RING and MD_GRAV2D systems batch", s);
      return nullptr;
    }
  md_batch *b = new (std::nothrow) md_batch();
  if (!b) {
    set_err(nullptr, MD_ENOMEM, "md_batch_init: host allocation");
    return nullptr;
  }
  b->nsys = nsys;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_err(nullptr, MD_ECUDA, "md_batch_init: device setup: %s", cudaGetErrorString(cudaGetLastError()));
    delete b;
    return nullptr;
  }
  b->own_stream = true;
  double work_r = 0.0, work_g = 0.0;
  for (int s = 0; s < nsys; s++) {
    md_ctx *c = md_init(model[s], N[s], eps[s], dt[s], seed[s]);
    if (!c) {
      std::string m = md_last_error(nullptr);
      md_batch_free(b);
      set_err(nullptr, MD_EINVAL, "md_batch_init: system %d: %s", s, m.c_str());
      return nullptr;
    }
    if (md_set_stream(c, b->stream) != MD_OK) {
      md_free(c);
      md_batch_free(b);
      set_err(nullptr, MD_ECUDA, "md_batch_init: stream");
      return nullptr;
    }
    c->prec = MD_MIXED;
    b->ctx.push_back(c);
    b->model.push_back(model[s]);
    (model[s] == MD_RING ? work_r : work_g) += (double)N[s] * (double)N[s];
  }
  // first split: pair counts weighted by the measured single-system costs per pair
  // (Ring / 2D about 1.07 on GB300); md_batch_autotune refines it
  const double wr = 1.07 * work_r, wg = work_g;
  b->cfg.split = (wr + wg) > 0.0 ? wr / (wr + wg) : 0.5;
  return b;
}

void md_batch_free(md_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  for (md_ctx *c : b->ctx) {
    c->stream = nullptr;
    c->own_stream = false;
    md_free(c);
  }
  dev_free(b->d_sys);
  dev_free(b->slots);
  dev_free(b->tickets);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char *md_batch_last_error(const md_batch *b) { return b ? b->err.c_str() : md_last_error(nullptr); }

int64_t md_batch_launch_count(const md_batch *b) {
  if (!b) return 0;
  int64_t n = b->launches;
  for (const md_ctx *c : b->ctx) n += c->launches;
  return n;
}

int md_batch_set_precision(md_batch *b, int prec) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  if (prec != MD_FP64 && prec != MD_MIXED) return berr(b, MD_EINVAL, "%s", "unknown precision");
  if (prec != b->prec) {
    b->prec = prec;
    b->mirrors_valid = false;
    drop_graphs(b);
  }
  return MD_OK;
}

int md_batch_set_stream(md_batch *b, void *stream) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  if (b->own_stream) cudaStreamDestroy(b->stream);
  b->stream = (cudaStream_t)stream;
  b->own_stream = false;
  for (md_ctx *c : b->ctx) c->stream = b->stream;
  drop_graphs(b);
  return MD_OK;
}

int md_batch_set_tuning(md_batch *b, int r, double split, int ctas_per_sm) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  if ((r != 4 && r != 8) || !(split > 0.0 && split < 1.0) || ctas_per_sm < 0 || ctas_per_sm > 16)
    return berr(b, MD_EINVAL, "%s", "md_batch_set_tuning: need r in {4, 8}, 0 < split < 1, 0 <= ctas_per_sm <= 16");
  b->cfg.r = r;
  b->cfg.split = split;
  b->cfg.ctas_per_sm = ctas_per_sm;
  drop_graphs(b);
  return MD_OK;
}

int md_batch_autotune(md_batch *b, double *best_ms) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  int rc = refresh_mirrors(b);
  if (rc) return rc;
  const Config base = b->cfg;
  std::vector<Config> cand;
  const int rs[2] = {8, 4};
  const double fs[5] = {0.90, 0.95, 1.0, 1.05, 1.10};
  const int cps[2] = {0, 3};
  for (int r : rs)
    for (double f : fs)
      for (int cp : cps) {
        Config c = base;
        c.r = b->prec == MD_MIXED ? r : base.r;
        c.split = base.split * f > 0.98 ? 0.98 : base.split * f;
        c.ctas_per_sm = cp;
        cand.push_back(c);
      }
  cudaEvent_t e0, e1;
  B_CUDA(b, cudaEventCreate(&e0));
  B_CUDA(b, cudaEventCreate(&e1));
  float best = 1e30f;
  Config pick = base;
  for (const Config &c : cand) {
    b->cfg = c;
    if ((rc = stage(b, STAGE_FORCE_ONLY, 0.0, 0.0))) break;  // warm-up (allocations)
    B_CUDA(b, cudaEventRecord(e0, b->stream));
    if ((rc = stage(b, STAGE_FORCE_ONLY, 0.0, 0.0))) break;
    B_CUDA(b, cudaEventRecord(e1, b->stream));
    B_CUDA(b, cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->cfg = pick;
  drop_graphs(b);
  if (best_ms) *best_ms = best;
  return rc;
}

int md_batch_step(md_batch *b, int64_t nsteps) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  if (nsteps < 0) return berr(b, MD_EINVAL, "%s", "md_batch_step: nsteps < 0");
  if (nsteps == 0) return MD_OK;
  int rc = refresh_mirrors(b);
  if (rc) return rc;
  double k[4];
  yoshida_coefficients(k);
  const double B0 = k[0], B1 = k[1], D0 = k[2], D1 = k[3];
  // first step (uncaptured: it also makes every buffer the graph will use)
  if ((rc = stage(b, STAGE_KICK_DRIFT, B0, D0)) || (rc = stage(b, STAGE_KICK_DRIFT, B1, D1)) ||
      (rc = stage(b, STAGE_KICK_DRIFT, B1, D0)))
    return rc;
  int64_t left = nsteps - 1;
  while (left >= kGraphSteps) {
    const int key = b->cur;
    if (b->graph_key[key] != key || !b->graph[key]) {
      cudaGraph_t g;
      B_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      for (int s = 0; s < kGraphSteps && !rc; s++) {
        if (!rc) rc = stage(b, STAGE_KICK_DRIFT, 2.0 * B0, D0);
        if (!rc) rc = stage(b, STAGE_KICK_DRIFT, B1, D1);
        if (!rc) rc = stage(b, STAGE_KICK_DRIFT, B1, D0);
      }
      cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
      if (rc) return rc;
      if (ee != cudaSuccess) return berr(b, MD_ECUDA, "graph capture: %s", cudaGetErrorString(ee));
      b->launches -= 3 * kGraphSteps;  // captured, not launched
      B_CUDA(b, cudaGraphInstantiate(&b->graph[key], g, 0));
      cudaGraphDestroy(g);
      b->graph_key[key] = key;
    }
    B_CUDA(b, cudaGraphLaunch(b->graph[key], b->stream));
    b->launches += 3 * kGraphSteps;
    left -= kGraphSteps;
  }
  for (; left > 0; left--) {
    if ((rc = stage(b, STAGE_KICK_DRIFT, 2.0 * B0, D0)) || (rc = stage(b, STAGE_KICK_DRIFT, B1, D1)) ||
        (rc = stage(b, STAGE_KICK_DRIFT, B1, D0)))
      return rc;
  }
  rc = stage(b, STAGE_KICK_ONLY, B0, 0.0);
  for (md_ctx *c : b->ctx) {
    c->mirror_cur = b->cur;
    c->fsal_valid = false;
  }
  return rc;
}

int md_batch_energy(md_batch *b, double *K, double *V) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  for (int s = 0; s < b->nsys; s++) {
    double k = 0.0, v = 0.0;
    int rc = md_energy(b->ctx[s], &k, &v);
    if (rc) return berr(b, rc, "%s", b->ctx[s]->err.c_str());
    if (K) K[s] = k;
    if (V) V[s] = v;
  }
  return MD_OK;
}

int md_batch_get_state(md_batch *b, int s, double *q, double *p) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  if (s < 0 || s >= b->nsys) return berr(b, MD_EINVAL, "%s", "system index out of range");
  int rc = md_get_state(b->ctx[s], q, p);
  return rc ? berr(b, rc, "%s", b->ctx[s]->err.c_str()) : MD_OK;
}

int md_batch_set_state(md_batch *b, int s, const double *q, const double *p) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  if (s < 0 || s >= b->nsys) return berr(b, MD_EINVAL, "%s", "system index out of range");
  int rc = md_set_state(b->ctx[s], q, p);
  b->mirrors_valid = false;
  return rc ? berr(b, rc, "%s", b->ctx[s]->err.c_str()) : MD_OK;
}

}  // extern "C"
