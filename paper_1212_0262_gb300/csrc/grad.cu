// Discrete adjoint of md_step (gradient of a final-time observable).
#include "md_internal.cuh"

extern "C" int md_grad(md_ctx *c, int observable, int64_t nsteps, int checkpoint_every, double *grad_q,
                       double *grad_p, double *grad_eps, double *value) {
  (void)observable; (void)nsteps; (void)checkpoint_every; (void)grad_q; (void)grad_p; (void)grad_eps; (void)value;
  if (!c) return MD_EINVAL;
  return set_err(c, MD_ESTATE, "md_grad: not available in this build");
}
