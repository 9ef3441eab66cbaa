// Row shards: one system of N particles advanced by several ranks, each owning a
// contiguous range of rows (particles), as in the paper's two-GPU schemes:
//
//  HMF (Sec. 3.1, last paragraph): each rank evaluates the mean-field stage on its
//    own particles and the partial magnetizations (sum cos, sum sin) of all ranks
//    are added before the next stage.
//  Ring / 2D (Sec. 3.2, Fig. 2 and its two-GPU stage list): each rank evaluates the
//    forces on its own rows against all N positions; after each drift the updated
//    positions of every rank are copied to all the others before the next force
//    evaluation.
//
// Generalised to P ranks, the exchange after every stage is one buffer per rank
// (HMF: the P partial sums; Ring / 2D: the whole position mirror) in which every
// rank writes its own segment, and the segments of the others are copied in.  The
// copy itself is the transport's: md_shard_exchange does it for ranks held by one
// process (cudaMemcpyAsync between their buffers, ordered by events), and a
// multi-process transport moves the same byte ranges (md_shard_buffer).
#include <vector>

#include "md_internal.cuh"

namespace {

int64_t row_align(int model) { return model == MD_HMF ? 1 : kShardRowAlign; }

// Row boundary of rank r: N r / P rounded down to the model's row alignment.
int64_t boundary(int model, int64_t N, int r, int nranks) {
  if (r >= nranks) return N;
  const int64_t A = row_align(model);
  return (N * (int64_t)r / nranks) / A * A;
}

int check_split(int model, int64_t N, int nranks, const char *who) {
  if (model != MD_HMF && model != MD_RING && model != MD_GRAV2D)
    return set_err(nullptr, MD_EINVAL, "%s: row shards are built for the HMF, Ring and 2D models", who);
  if (nranks < 1 || nranks > kMaxShards)
    return set_err(nullptr, MD_EINVAL, "%s: nranks must be in [1, %d], got %d", who, kMaxShards, nranks);
  if (N < 1 || N > (int64_t)1 << 40) return set_err(nullptr, MD_EINVAL, "%s: N must be in [1, 2^40]", who);
  for (int r = 0; r < nranks; r++)
    if (boundary(model, N, r + 1, nranks) <= boundary(model, N, r, nranks))
      return set_err(nullptr, MD_EINVAL,
                     "%s: rank %d gets no rows (N = %lld over %d ranks in blocks of %lld rows)", who, r,
                     (long long)N, nranks, (long long)row_align(model));
  return MD_OK;
}

int check_shard(md_ctx *c, const char *who) {
  if (!c) return set_err(nullptr, MD_EINVAL, "%s: NULL context", who);
  if (!c->shard) return set_err(c, MD_ESTATE, "%s: not a row shard (make it with md_shard_init)", who);
  return MD_OK;
}

int check_primed(md_ctx *c, const char *who) {
  int rc = check_shard(c, who);
  if (rc) return rc;
  if (!c->shard_primed || c->shard_prec != c->prec)
    return set_err(c, MD_ESTATE, "%s: call md_shard_begin first (after md_shard_init, a state or precision change)",
                   who);
  return MD_OK;
}

// Runs `fn` with the context's device current, restoring the caller's device.
template <class F>
int on_device(md_ctx *c, F fn) {
  int prev = 0;
  MD_CUDA(c, cudaGetDevice(&prev));
  if (prev != c->device) MD_CUDA(c, cudaSetDevice(c->device));
  int rc = fn();
  if (prev != c->device) cudaSetDevice(prev);
  return rc;
}

int segment(md_ctx *c, void **buf, size_t *off, size_t *bytes) {
  if (c->model == MD_HMF) {
    *buf = c->shard_sums + 2 * c->shard_nranks * c->shard_cur;
    *off = 2 * sizeof(double) * (size_t)c->shard_rank;
    *bytes = 2 * sizeof(double);
    return MD_OK;
  }
  return pair_shard_segment(c, buf, off, bytes);
}

int check_group(md_ctx *const *ctx, int nranks, const char *who, bool need_primed) {
  if (!ctx || nranks < 1 || nranks > kMaxShards)
    return set_err(nullptr, MD_EINVAL, "%s: need an array of 1 to %d shard contexts", who, kMaxShards);
  for (int r = 0; r < nranks; r++) {
    md_ctx *c = ctx[r];
    int rc = need_primed ? check_primed(c, who) : check_shard(c, who);
    if (rc) return rc;
    if (c->shard_rank != r || c->shard_nranks != nranks || c->model != ctx[0]->model ||
        c->n_total != ctx[0]->n_total || c->prec != ctx[0]->prec)
      return set_err(c, MD_EINVAL,
                     "%s: entry %d must be rank %d of the same %d-rank system, model and precision (it is rank %d of %d)",
                     who, r, r, nranks, c->shard_rank, c->shard_nranks);
    if (need_primed && ((c->model == MD_HMF && c->shard_cur != ctx[0]->shard_cur) ||
                        (c->model != MD_HMF && c->mirror_cur != ctx[0]->mirror_cur)))
      return set_err(c, MD_ESTATE, "%s: the ranks have run different numbers of stages", who);
  }
  return MD_OK;
}

int begin(md_ctx *c) {
  return on_device(c, [&] {
    int rc = c->model == MD_HMF ? hmf_shard_prime(c) : pair_shard_prime(c);
    if (rc) return rc;
    c->shard_primed = true;
    c->shard_prec = c->prec;
    c->fsal_valid = false;
    return MD_OK;
  });
}

int stage(md_ctx *c, double b, double d) {
  return on_device(c, [&] {
    const double h = c->dt;
    return c->model == MD_HMF ? hmf_shard_stage(c, STAGE_KICK_DRIFT, b * h, d * h, nullptr)
                              : pair_shard_stage(c, STAGE_KICK_DRIFT, b * h, d * h, nullptr);
  });
}

int exchange(md_ctx *const *ctx, int nranks) {
  // every rank's last stage (or md_shard_begin) is complete before anyone copies from it
  for (int r = 0; r < nranks; r++) {
    md_ctx *c = ctx[r];
    int rc = on_device(c, [&] {
      MD_CUDA(c, cudaEventRecord(c->shard_event, c->stream));
      return MD_OK;
    });
    if (rc) return rc;
  }
  for (int r = 0; r < nranks; r++) {
    md_ctx *c = ctx[r];
    void *dst = nullptr;
    size_t off = 0, bytes = 0;
    int rc = segment(c, &dst, &off, &bytes);
    if (rc) return rc;
    rc = on_device(c, [&] {
      for (int s = 0; s < nranks; s++) {
        if (s == r) continue;
        md_ctx *o = ctx[s];
        void *src = nullptr;
        size_t so = 0, sb = 0;
        int rc2 = segment(o, &src, &so, &sb);
        if (rc2) return rc2;
        MD_CUDA(c, cudaStreamWaitEvent(c->stream, o->shard_event, 0));
        MD_CUDA(c, cudaMemcpyAsync((char *)dst + so, (const char *)src + so, sb, cudaMemcpyDefault, c->stream));
      }
      return MD_OK;
    });
    if (rc) return rc;
  }
  return MD_OK;
}

}  // namespace

extern "C" {

int md_shard_range(int model, int64_t N, int rank, int nranks, int64_t *lo, int64_t *hi) {
  int rc = check_split(model, N, nranks, "md_shard_range");
  if (rc) return rc;
  if (rank < 0 || rank >= nranks || !lo || !hi)
    return set_err(nullptr, MD_EINVAL, "md_shard_range: need 0 <= rank < nranks and non-NULL outputs");
  *lo = boundary(model, N, rank, nranks);
  *hi = boundary(model, N, rank + 1, nranks);
  return MD_OK;
}

md_ctx *md_shard_init(int model, int64_t N, double eps, double dt, uint64_t seed, int rank, int nranks) {
  if (check_split(model, N, nranks, "md_shard_init")) return nullptr;
  if (rank < 0 || rank >= nranks) {
    set_err(nullptr, MD_EINVAL, "md_shard_init: rank %d outside [0, %d)", rank, nranks);
    return nullptr;
  }
  const int64_t lo = boundary(model, N, rank, nranks), hi = boundary(model, N, rank + 1, nranks);
  md_ctx *c = create_context(model, hi - lo, N, lo, eps, dt, seed, "md_shard_init");
  if (!c) return nullptr;
  c->shard = true;
  c->shard_rank = rank;
  c->shard_nranks = nranks;
  if (cudaEventCreateWithFlags(&c->shard_event, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    c->shard_event = nullptr;
    set_err(nullptr, MD_ECUDA, "md_shard_init: event");
    md_free(c);
    return nullptr;
  }
  return c;
}

int md_shard_begin(md_ctx *c) {
  int rc = check_shard(c, "md_shard_begin");
  return rc ? rc : begin(c);
}

int md_shard_stage(md_ctx *c, double b, double d) {
  int rc = check_primed(c, "md_shard_stage");
  if (rc) return rc;
  if (!(b - b == 0.0) || !(d - d == 0.0)) return set_err(c, MD_EINVAL, "md_shard_stage: non-finite coefficient");
  return stage(c, b, d);
}

int md_shard_buffer(md_ctx *c, void **buf, size_t *seg_offset, size_t *seg_bytes) {
  int rc = check_primed(c, "md_shard_buffer");
  if (rc) return rc;
  if (!buf || !seg_offset || !seg_bytes) return set_err(c, MD_EINVAL, "md_shard_buffer: NULL output");
  return segment(c, buf, seg_offset, seg_bytes);
}

int md_shard_exchange(md_ctx *const *ctx, int nranks) {
  int rc = check_group(ctx, nranks, "md_shard_exchange", true);
  return rc ? rc : exchange(ctx, nranks);
}

int md_shard_step(md_ctx *const *ctx, int nranks, int64_t nsteps) {
  int rc = check_group(ctx, nranks, "md_shard_step", false);
  if (rc) return rc;
  if (nsteps < 0) return set_err(ctx[0], MD_EINVAL, "md_shard_step: nsteps < 0");
  if (nsteps == 0) return MD_OK;
  bool primed = true;
  for (int r = 0; r < nranks; r++) primed = primed && ctx[r]->shard_primed && ctx[r]->shard_prec == ctx[r]->prec;
  if (!primed) {
    for (int r = 0; r < nranks; r++)
      if ((rc = begin(ctx[r]))) return rc;
    if ((rc = exchange(ctx, nranks))) return rc;
  }
  if ((rc = check_group(ctx, nranks, "md_shard_step", true))) return rc;
  double k[4];
  yoshida_coefficients(k);
  const double B0 = k[0], B1 = k[1], D0 = k[2], D1 = k[3];
  // Sec. 3 step list with Eq. 4's constants; the closing kick of a step and the
  // opening kick of the next merge (2 B0), and the last step ends with a B0 kick
  std::vector<std::pair<double, double>> st;
  for (int64_t s = 0; s < nsteps; s++) {
    st.push_back({s == 0 ? B0 : 2.0 * B0, D0});
    st.push_back({B1, D1});
    st.push_back({B1, D0});
  }
  st.push_back({B0, 0.0});
  for (const auto &bd : st) {
    for (int r = 0; r < nranks; r++)
      if ((rc = stage(ctx[r], bd.first, bd.second))) return rc;
    if ((rc = exchange(ctx, nranks))) return rc;
  }
  return MD_OK;
}

int md_shard_force(md_ctx *c, double *f) {
  int rc = check_primed(c, "md_shard_force");
  if (rc) return rc;
  if (!f) return set_err(c, MD_EINVAL, "md_shard_force: NULL output");
  return on_device(c, [&] {
    int rc2 = c->model == MD_HMF ? hmf_shard_stage(c, STAGE_FORCE_ONLY, 0.0, 0.0, c->f)
                                 : pair_shard_stage(c, STAGE_FORCE_ONLY, 0.0, 0.0, c->f);
    if (rc2) return rc2;
    MD_CUDA(c, cudaMemcpyAsync(f, c->f, sizeof(double) * (size_t)(c->dim * c->N), cudaMemcpyDeviceToHost, c->stream));
    MD_CUDA(c, cudaStreamSynchronize(c->stream));
    return MD_OK;
  });
}

}  // extern "C"
