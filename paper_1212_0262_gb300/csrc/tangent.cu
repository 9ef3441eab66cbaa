// md_tangent_step: the state and a tangent vector advanced together by the
// linearisation of md_step's map (forward-mode derivative), the building block
// of largest-Lyapunov-exponent estimates.  Each stage is one fused kernel: the
// force and J(q) dq from a single pair pass (pair models) or from four mean-field
// sums (HMF), then the kick and drift of both.
#include "md_internal.cuh"

namespace {

// Workspace: the tangent (dq, dp) as 2 dim N doubles, then 16 scalars (HMF sums
// ping-pong in [0, 8), the squared norm's half at [8], the log accumulator at [9]).
int tangent_workspace(md_ctx *c, const char *who) {
  const int64_t n = (int64_t)c->dim * c->N;
  const size_t need = sizeof(double) * (size_t)(2 * n + 16);
  if (need > c->gw_bytes) {
    dev_free(c->gw);
    c->gw = (double *)dev_alloc(need);
    if (!c->gw) {
      c->gw_bytes = 0;
      return set_err(c, MD_ENOMEM, "%s: workspace", who);
    }
    c->gw_bytes = need;
  }
  return MD_OK;
}

int tangent_checks(md_ctx *c, const char *who) {
  if (!c) return set_err(nullptr, MD_EINVAL, "%s: NULL context", who);
  if (c->shard) return set_err(c, MD_ESTATE, "%s: not defined on a row shard (use the md_shard_* calls)", who);
  if (c->model == MD_SHEET1D && !(c->eps > 0.0))
    return set_err(c, MD_EINVAL, "%s: the eps = 0 sheet force is piecewise constant; derivatives need eps > 0", who);
  return MD_OK;
}

// nsteps steps of the state with the tangent (tq, tp) in the workspace, queued on
// the stream (the stage list of md_step).
int tangent_run(md_ctx *c, int64_t nsteps) {
  const int64_t n = (int64_t)c->dim * c->N;
  double *tq = c->gw, *tp = c->gw + n, *sums = c->gw + 2 * n;
  double k[4];
  yoshida_coefficients(k);
  const double h = c->dt, B0 = k[0], B1 = k[1], D0 = k[2], D1 = k[3];
  int cur = 0, rc;
  auto stage = [&](double b, double d) -> int {
    if (c->model == MD_HMF) {
      int r = hmf_tangent_stage(c, b * h, d * h, tq, tp, sums + 4 * cur, sums + 4 * (1 - cur));
      if (d != 0.0) cur = 1 - cur;
      return r;
    }
    return pair_tangent_stage(c, b * h, d * h, tq, tp);
  };
  rc = c->model == MD_HMF ? hmf_adjoint_prime(c, tq, sums) : adjoint_mirror_refresh(c, tq);
  if (rc) return rc;
  for (int64_t s = 0; s < nsteps && !rc; s++) {
    if (!rc) rc = stage(s == 0 ? B0 : 2.0 * B0, D0);
    if (!rc) rc = stage(B1, D1);
    if (!rc) rc = stage(B1, D0);
  }
  if (!rc) rc = stage(B0, 0.0);
  // the state advanced; the force cache and the mirrors no longer describe it
  c->fsal_valid = false;
  c->hmf_m_valid = false;
  c->mirror_valid = false;
  return rc;
}

// x[0..m) scaled by 1 / |x|, |x| = sqrt(2 half_sq); if count, log |x| added to *log_acc.
__global__ void renorm_kernel(double *__restrict__ x, int64_t m, const double *half_sq, double *log_acc, int count) {
  const double nrm = sqrt(2.0 * *half_sq);
  const double inv = 1.0 / nrm;
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += G) x[i] *= inv;
  if (count && blockIdx.x == 0 && threadIdx.x == 0) *log_acc += log(nrm);
}

// Normalise the tangent in the workspace to unit length (FP64 norm of (dq, dp)).
int renorm(md_ctx *c, bool count) {
  const int64_t n = (int64_t)c->dim * c->N;
  double *scal = c->gw + 2 * n + 8;
  int rc = half_sumsq_fp64(c, c->gw, 2 * n, scal);
  if (rc) return rc;
  int64_t blocks = (2 * n + 255) / 256;
  if (blocks > (int64_t)c->nsm * 8) blocks = (int64_t)c->nsm * 8;
  renorm_kernel<<<(int)blocks, 256, 0, c->stream>>>(c->gw, 2 * n, scal, scal + 1, count ? 1 : 0);
  MD_LAUNCHED(c);
  return MD_OK;
}

}  // namespace

extern "C" int md_tangent_step(md_ctx *c, int64_t nsteps, double *dq, double *dp) {
  int rc = tangent_checks(c, "md_tangent_step");
  if (rc) return rc;
  if (nsteps < 0 || !dq || !dp) return set_err(c, MD_EINVAL, "md_tangent_step: need nsteps >= 0 and arrays");
  if (nsteps == 0) return MD_OK;
  if ((rc = tangent_workspace(c, "md_tangent_step"))) return rc;
  const int64_t n = (int64_t)c->dim * c->N;
  const size_t nb = sizeof(double) * (size_t)n;
  MD_CUDA(c, cudaMemcpyAsync(c->gw, dq, nb, cudaMemcpyHostToDevice, c->stream));
  MD_CUDA(c, cudaMemcpyAsync(c->gw + n, dp, nb, cudaMemcpyHostToDevice, c->stream));
  if ((rc = tangent_run(c, nsteps))) return rc;
  MD_CUDA(c, cudaMemcpyAsync(dq, c->gw, nb, cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(c, cudaMemcpyAsync(dp, c->gw + n, nb, cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(c, cudaStreamSynchronize(c->stream));
  return MD_OK;
}

extern "C" int md_lyapunov(md_ctx *c, int64_t nsteps, int64_t renorm_every, double *dq, double *dp,
                           double *sum_log) {
  int rc = tangent_checks(c, "md_lyapunov");
  if (rc) return rc;
  if (nsteps < 1 || renorm_every < 1 || !dq || !dp || !sum_log)
    return set_err(c, MD_EINVAL, "md_lyapunov: need nsteps >= 1, renorm_every >= 1 and non-NULL arrays");
  if ((rc = tangent_workspace(c, "md_lyapunov"))) return rc;
  const int64_t n = (int64_t)c->dim * c->N;
  const size_t nb = sizeof(double) * (size_t)n;
  MD_CUDA(c, cudaMemcpyAsync(c->gw, dq, nb, cudaMemcpyHostToDevice, c->stream));
  MD_CUDA(c, cudaMemcpyAsync(c->gw + n, dp, nb, cudaMemcpyHostToDevice, c->stream));
  MD_CUDA(c, cudaMemsetAsync(c->gw + 2 * n + 9, 0, sizeof(double), c->stream));
  if ((rc = renorm(c, false))) return rc;  // unit initial tangent, not counted
  for (int64_t done = 0; done < nsteps;) {
    const int64_t k = renorm_every < nsteps - done ? renorm_every : nsteps - done;
    if ((rc = tangent_run(c, k)) || (rc = renorm(c, true))) return rc;
    done += k;
  }
  MD_CUDA(c, cudaMemcpyAsync(dq, c->gw, nb, cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(c, cudaMemcpyAsync(dp, c->gw + n, nb, cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(c, cudaMemcpyAsync(c->host_scalars + 8, c->gw + 2 * n + 9, sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
  MD_CUDA(c, cudaStreamSynchronize(c->stream));
  *sum_log = c->host_scalars[8];
  if (!(*sum_log - *sum_log == 0.0)) return set_err(c, MD_ENONFINITE, "md_lyapunov: non-finite tangent norm");
  return MD_OK;
}
