// md_tangent_step: the state and a tangent vector advanced together by the
// linearisation of md_step's map (forward-mode derivative), the building block
// of largest-Lyapunov-exponent estimates.  Each stage is one fused kernel: the
// force and J(q) dq from a single pair pass (pair models) or from four mean-field
// sums (HMF), then the kick and drift of both.
#include "md_internal.cuh"

extern "C" int md_tangent_step(md_ctx *c, int64_t nsteps, double *dq, double *dp) {
  if (!c) return set_err(nullptr, MD_EINVAL, "md_tangent_step: NULL context");
  if (c->model == MD_SHEET1D && !(c->eps > 0.0))
    return set_err(c, MD_EINVAL, "md_tangent_step: the eps = 0 sheet force is piecewise constant; derivatives need eps > 0");
  if (nsteps < 0 || !dq || !dp) return set_err(c, MD_EINVAL, "md_tangent_step: need nsteps >= 0 and arrays");
  if (nsteps == 0) return MD_OK;
  const int64_t n = (int64_t)c->dim * c->N;
  const size_t nb = sizeof(double) * (size_t)n;
  const size_t need = 2 * nb + 16 * sizeof(double);
  if (need > c->gw_bytes) {
    dev_free(c->gw);
    c->gw = (double *)dev_alloc(need);
    if (!c->gw) {
      c->gw_bytes = 0;
      return set_err(c, MD_ENOMEM, "md_tangent_step: workspace");
    }
    c->gw_bytes = need;
  }
  double *tq = c->gw, *tp = c->gw + n, *sums = c->gw + 2 * n;
  MD_CUDA(c, cudaMemcpyAsync(tq, dq, nb, cudaMemcpyHostToDevice, c->stream));
  MD_CUDA(c, cudaMemcpyAsync(tp, dp, nb, cudaMemcpyHostToDevice, c->stream));
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
  if (rc) return rc;
  MD_CUDA(c, cudaMemcpyAsync(dq, tq, nb, cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(c, cudaMemcpyAsync(dp, tp, nb, cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(c, cudaStreamSynchronize(c->stream));
  // the state advanced; the force cache and the mirrors no longer describe it
  c->fsal_valid = false;
  c->hmf_m_valid = false;
  c->mirror_valid = false;
  return MD_OK;
}
