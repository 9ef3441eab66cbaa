// md_grad: discrete adjoint of md_step (gradient of a final-time observable with
// respect to the initial state and eps).
//
// md_step's map is a sequence of kicks p' = p + b dt f(q) and drifts
// q' = q + d dt p (Sec. 3 step list, Eq. 4 splitting; consecutive B0 kicks at the
// same position merged).  Its transpose, applied map by map from the last to the
// first, is
//   kick:  lambda_q += b dt J(q) lambda_p,   dO/deps += b dt <lambda_p, df/deps(q)>
//   drift: lambda_p += d dt lambda_q
// with J = df/dq (symmetric).  The positions q of the kicks are rebuilt by running
// the step backwards (undo the kick with the force at the same q, then undo the
// drift), which the symmetric, time-reversible splitting (Sec. 3, after Eq. 4)
// makes exact up to rounding; every `checkpoint_every` steps the state is reset
// to an FP64 copy stored by the forward pass, which bounds the accumulated
// rounding drift.  Each reverse stage is one fused kernel: force, J lambda_p and
// df/deps from a single pair pass (pair models) or from four mean-field sums (HMF).
#include "md_internal.cuh"

extern "C" int md_grad(md_ctx *c, int observable, int64_t nsteps, int checkpoint_every, double *grad_q,
                       double *grad_p, double *grad_eps, double *value) {
  if (!c) return set_err(nullptr, MD_EINVAL, "md_grad: NULL context");
  if (c->shard) return set_err(c, MD_ESTATE, "md_grad: not defined on a row shard (use the md_shard_* calls)");
  if (observable != MD_OBS_KINETIC && observable != MD_OBS_MAGNETIZATION)
    return set_err(c, MD_EINVAL, "md_grad: unknown observable %d", observable);
  if (c->model == MD_SHEET1D && !(c->eps > 0.0))
    return set_err(c, MD_EINVAL, "md_grad: the eps = 0 sheet force is piecewise constant; derivatives need eps > 0");
  if (observable == MD_OBS_MAGNETIZATION && c->model != MD_HMF && c->model != MD_RING)
    return set_err(c, MD_EINVAL, "md_grad: the magnetization is defined for HMF and Ring only");
  if (nsteps < 0 || checkpoint_every < 1) return set_err(c, MD_EINVAL, "md_grad: need nsteps >= 0, checkpoint_every >= 1");
  if (!grad_q || !grad_p) return set_err(c, MD_EINVAL, "md_grad: NULL gradient output");

  const int64_t n = (int64_t)c->dim * c->N, N = c->N;
  const size_t nb = sizeof(double) * (size_t)n;
  const int64_t K = checkpoint_every;
  const int64_t nseg = (nsteps + K - 1) / K;
  const int64_t nck = nseg + 1;
  const size_t need = sizeof(double) * ((size_t)nck * 2 * n + 2 * n + N + 16);
  if (need > c->gw_bytes) {
    dev_free(c->gw);
    c->gw = (double *)dev_alloc(need);
    if (!c->gw) {
      c->gw_bytes = 0;
      return set_err(c, MD_ENOMEM, "md_grad: workspace of %zu bytes", need);
    }
    c->gw_bytes = need;
  }
  double *ck = c->gw;
  double *lq = ck + nck * 2 * n, *lp = lq + n, *epsacc = lp + n;
  double *sums = epsacc + N;  // two slots of four sums
  double *scal = sums + 8;    // [0] observable value, [1] d O / d eps, [2..3] magnetization sums
  auto save = [&](int64_t m) -> int {
    MD_CUDA(c, cudaMemcpyAsync(ck + m * 2 * n, c->q, nb, cudaMemcpyDeviceToDevice, c->stream));
    MD_CUDA(c, cudaMemcpyAsync(ck + m * 2 * n + n, c->p, nb, cudaMemcpyDeviceToDevice, c->stream));
    return MD_OK;
  };
  auto restore = [&](int64_t m) -> int {
    MD_CUDA(c, cudaMemcpyAsync(c->q, ck + m * 2 * n, nb, cudaMemcpyDeviceToDevice, c->stream));
    MD_CUDA(c, cudaMemcpyAsync(c->p, ck + m * 2 * n + n, nb, cudaMemcpyDeviceToDevice, c->stream));
    return MD_OK;
  };
  int rc;

  // ---- forward, with checkpoints at steps 0, K, 2K, ..., nsteps
  if ((rc = save(0))) return rc;
  for (int64_t m = 0; m < nseg; m++) {
    const int64_t steps = (nsteps - m * K) < K ? (nsteps - m * K) : K;
    if ((rc = integrate(c, steps))) return rc;
    if ((rc = save(m + 1))) return rc;
  }

  // ---- observable and terminal adjoint
  double cx = 0.0, cy = 0.0;
  if (observable == MD_OBS_KINETIC) {
    if ((rc = kinetic_fp64(c, scal))) return rc;
    MD_CUDA(c, cudaMemcpyAsync(lp, c->p, nb, cudaMemcpyDeviceToDevice, c->stream));
    MD_CUDA(c, cudaMemsetAsync(lq, 0, nb, c->stream));
  } else {
    if ((rc = hmf_sums_fp64(c, scal + 2))) return rc;
    MD_CUDA(c, cudaMemcpyAsync(c->host_scalars, scal + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MD_CUDA(c, cudaStreamSynchronize(c->stream));
    const double mx = c->host_scalars[0] / (double)N, my = c->host_scalars[1] / (double)N;
    const double m = sqrt(mx * mx + my * my);
    if (!(m > 0.0)) return set_err(c, MD_ENONFINITE, "md_grad: |M| = 0 has no gradient");
    cx = my / ((double)N * m);
    cy = mx / ((double)N * m);
    c->host_scalars[8] = m;
    if ((rc = hmf_magnetization_terminal(c, cx, cy, lq))) return rc;
    MD_CUDA(c, cudaMemsetAsync(lp, 0, nb, c->stream));
  }
  MD_CUDA(c, cudaMemsetAsync(epsacc, 0, sizeof(double) * (size_t)N, c->stream));

  // ---- reverse sweep
  double k4[4];
  yoshida_coefficients(k4);
  const double h = c->dt, B0 = k4[0], B1 = k4[1], D0 = k4[2], D1 = k4[3];
  int cur = 0;
  auto prime = [&]() -> int {
    if (c->model == MD_HMF) return hmf_adjoint_prime(c, lp, sums + 4 * cur);
    return adjoint_mirror_refresh(c, lp);
  };
  auto rstage = [&](double badj, double bundo, double d) -> int {
    if (c->model == MD_HMF) {
      int r = hmf_adjoint_stage(c, badj * h, bundo * h, d * h, lq, lp, sums + 4 * cur, sums + 4 * (1 - cur));
      if (d != 0.0) cur = 1 - cur;
      return r;
    }
    return pair_adjoint_stage(c, badj * h, bundo * h, d * h, lq, lp, epsacc);
  };
  if (nsteps > 0) {
    if ((rc = restore(nseg))) return rc;
    if ((rc = prime())) return rc;
    bool just_reset = true;  // the stored p sits between the two B0 kicks at that position
    for (int64_t t = nsteps - 1; t >= 0; t--) {
      const double badj = (t == nsteps - 1) ? B0 : 2.0 * B0;
      const double bundo = just_reset ? B0 : 2.0 * B0;
      if ((rc = rstage(badj, bundo, D0))) return rc;
      if ((rc = rstage(B1, B1, D1))) return rc;
      if ((rc = rstage(B1, B1, D0))) return rc;
      just_reset = false;
      if (t % K == 0) {
        if ((rc = restore(t / K))) return rc;
        if ((rc = prime())) return rc;
        just_reset = true;
      }
    }
    if ((rc = rstage(B0, B0, 0.0))) return rc;  // opening kick of the first step, at q(0)
  }

  // ---- outputs
  if ((rc = sum_fp64(c, epsacc, N, scal + 1))) return rc;
  MD_CUDA(c, cudaMemcpyAsync(grad_q, lq, nb, cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(c, cudaMemcpyAsync(grad_p, lp, nb, cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(c, cudaMemcpyAsync(c->host_scalars + 4, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  // the context's state is unchanged: back to the starting point
  if ((rc = restore(0))) return rc;
  MD_CUDA(c, cudaStreamSynchronize(c->stream));
  c->fsal_valid = false;
  c->hmf_m_valid = false;
  c->mirror_valid = false;
  if (value) *value = observable == MD_OBS_KINETIC ? c->host_scalars[4] : c->host_scalars[8];
  if (grad_eps) *grad_eps = c->model == MD_HMF ? 0.0 : c->host_scalars[5];
  return MD_OK;
}

extern "C" int md_set_eps(md_ctx *c, double eps) {
  if (!c) return set_err(nullptr, MD_EINVAL, "md_set_eps: NULL context");
  const bool eps0_ok = c->model == MD_HMF || c->model == MD_SHEET1D;
  if (!eps_valid(c->model, eps))
    return set_err(c, MD_EINVAL, "md_set_eps: eps must be finite and %s %g", eps0_ok ? "0 or >=" : ">=", kEpsMin);
  c->eps = eps;
  c->fsal_valid = false;    // the cached force depends on eps
  c->mirror_valid = false;  // and the sheet model's padding records do
  return MD_OK;
}
