// FP64 observables: kinetic energy and the pair potentials of Eqs. 1 and 3 (and
// of the 3D self-gravitating model).
//
// All sums are deterministic: per-thread sums, a fixed shuffle/block tree, one
// partial per CTA (or per tile pair), and a final pass that adds the partials in
// index order (the last CTA to finish does it; no waiting).
#include "md_internal.cuh"

namespace {

constexpr int NT = 256;
constexpr int PT = 256;  // potential tile (particles per side)

__device__ __forceinline__ void finish_sum(double v, double *partials, double *out, unsigned *ticket) {
  __shared__ double2 red[NT / 32];
  __shared__ bool last;
  double2 b = block_sum2<NT>(v, 0.0, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = b.x;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int j = threadIdx.x; j < (int)gridDim.x; j += NT) s += __ldcg(partials + j);
  __syncthreads();
  double2 t = block_sum2<NT>(s, 0.0, red);
  if (threadIdx.x == 0) {
    *out = t.x;
    *ticket = 0u;
  }
}

// SQUARE: sum of x^2 / 2, else plain sum.
template <bool SQUARE>
__global__ void __launch_bounds__(NT) sum_kernel(const double *__restrict__ x, int64_t n, double *partials,
                                                 double *out, unsigned *ticket) {
  double s = 0.0;
  const int64_t G = (int64_t)gridDim.x * NT;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += G) {
    double v = x[i];
    s += SQUARE ? v * v : v;
  }
  if (SQUARE) s *= 0.5;
  finish_sum(s, partials, out, ticket);
}

// (sin, cos) of half the range-reduced angle, for the Ring potential.
__global__ void half_angle_kernel(const double *__restrict__ q, int64_t N, double2 *__restrict__ ag) {
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += G) {
    double a, g;
    sincos(0.5 * reduce_2pi(q[i]), &a, &g);
    ag[i] = make_double2(a, g);
  }
}

// m * s as a mantissa in [1, 2) and a power of two added to e: a positive normal m
// times a positive normal s keeps an exact binary exponent, and rescaling by a
// power of two is exact.  Integer-pipe work only, beside the FP64 multiply.
// A product that is not a normal double (a NaN or infinite factor, an overflow, or
// a subnormal or zero factor) has the exponent field 0x7ff or 0; `odd` records it
// so that the row falls back to the plain sum of logarithms.
__device__ __forceinline__ double mul_renorm(double m, double s, int &e, unsigned &odd) {
  const double r = m * s;
  const int hi = __double2hiint(r);
  const int ex = (hi >> 20) & 0x7ff;
  e += ex - 1023;
  odd |= (unsigned)(ex - 1) >= 0x7feu;
  return __hiloint2double((hi & 0x800fffff) | 0x3ff00000, __double2loint(r));
}

// One tile pair (ti <= tj) of the i<j potential sum.
//  Ring: -(1/(2N)) sum d^(-1/2), d = sin^2((ti-tj)/2) + eps/2  (Eq. 1, with
//        1 - cos d + eps = 2 d)
//  2D:   (1/N) sum log(|r_ij|^2 + eps)                        (Eq. 3)
// The 2D sum of logarithms of one thread's row of the tile is the logarithm of the
// product of its s = |r|^2 + eps values: the product is kept as m 2^e (m in [1, 2),
// renormalised after every factor, so it can neither overflow nor underflow while
// every s is a normal double), and log m + e ln 2 replaces up to 256 logarithms.
// A row with a factor that is not a normal double (a non-finite position, or
// coincident particles with a subnormal eps) sums its logarithms one by one, so a
// NaN or infinite position gives a NaN or infinite V.
// Relative rounding of m: at most one unit roundoff per factor, i.e. about
// 2.8e-14 absolute in the row's sum of 256 logarithms, the size of the rounding of
// the sum of the logarithms themselves.
// The prefactor is applied on the host.
template <int MODEL>
__global__ void __launch_bounds__(NT) potential_tiles_kernel(const double *__restrict__ q,
                                                              const double2 *__restrict__ ag, int64_t N,
                                                              int ntiles, double epsd, double *unit_sums) {
  const int ti = blockIdx.x, tj = blockIdx.y;
  if (tj < ti) return;
  __shared__ double2 sj[PT];
  const int64_t j0 = (int64_t)tj * PT;
  for (int t = threadIdx.x; t < PT; t += NT) {
    int64_t j = j0 + t;
    if (j < N) sj[t] = MODEL == MD_RING ? ag[j] : make_double2(q[j], q[N + j]);
  }
  __syncthreads();
  const int64_t i = (int64_t)ti * PT + threadIdx.x;
  double s = 0.0;
  if (i < N) {
    const double2 me = MODEL == MD_RING ? ag[i] : make_double2(q[i], q[N + i]);
    int kbeg = 0;
    if (ti == tj) kbeg = threadIdx.x + 1;  // j > i inside the diagonal tile
    int kend = (int)((N - j0) < PT ? (N - j0) : PT);
    if constexpr (MODEL == MD_RING) {
      for (int k = kbeg; k < kend; k++) {
        const double2 o = sj[k];
        double sh = fma(me.x, o.y, -(me.y * o.x));
        s += rsqrt_nr(fma(sh, sh, epsd));
      }
    } else {
      double m = 1.0;
      int e = 0;
      unsigned odd = 0u;
      for (int k = kbeg; k < kend; k++) {
        const double2 o = sj[k];
        const double dx = me.x - o.x, dy = me.y - o.y;
        m = mul_renorm(m, fma(dx, dx, fma(dy, dy, epsd)), e, odd);
      }
      s = log(m) + (double)e * 0.69314718055994530942;
      if (odd) {  // a factor outside the normal range: NaN, inf or a tiny s stay exact per pair
        s = 0.0;
        for (int k = kbeg; k < kend; k++) {
          const double2 o = sj[k];
          const double dx = me.x - o.x, dy = me.y - o.y;
          s += log(fma(dx, dx, fma(dy, dy, epsd)));
        }
      }
    }
  }
  __shared__ double2 red[NT / 32];
  double2 b = block_sum2<NT>(s, 0.0, red);
  if (threadIdx.x == 0) unit_sums[(int64_t)ti * ntiles + tj] = b.x;
}

// 3D: one tile pair (ti <= tj) of sum_{i<j} (|r_ij|^2 + eps)^(-1/2); the prefactor
// -1/N is applied at the end.
__global__ void __launch_bounds__(NT) potential3d_tiles_kernel(const double *__restrict__ q, int64_t N, int ntiles,
                                                                double eps, double *unit_sums) {
  const int ti = blockIdx.x, tj = blockIdx.y;
  if (tj < ti) return;
  __shared__ double sx[PT], sy[PT], sz[PT];
  const int64_t j0 = (int64_t)tj * PT;
  for (int t = threadIdx.x; t < PT; t += NT) {
    const int64_t j = j0 + t;
    if (j < N) {
      sx[t] = q[j];
      sy[t] = q[N + j];
      sz[t] = q[2 * N + j];
    }
  }
  __syncthreads();
  const int64_t i = (int64_t)ti * PT + threadIdx.x;
  double s = 0.0;
  if (i < N) {
    const double x = q[i], y = q[N + i], z = q[2 * N + i];
    const int kbeg = ti == tj ? threadIdx.x + 1 : 0;  // j > i inside the diagonal tile
    const int kend = (int)((N - j0) < PT ? (N - j0) : PT);
    for (int k = kbeg; k < kend; k++) {
      const double dx = x - sx[k], dy = y - sy[k], dz = z - sz[k];
      s += rsqrt_nr(fma(dx, dx, fma(dy, dy, fma(dz, dz, eps))));
    }
  }
  __shared__ double2 red[NT / 32];
  double2 b = block_sum2<NT>(s, 0.0, red);
  if (threadIdx.x == 0) unit_sums[(int64_t)ti * ntiles + tj] = b.x;
}

// 1D sheets: one tile pair (ti <= tj) of sum_{i<j} |x_i - x_j| (eps = 0) or
// sqrt((x_i - x_j)^2 + eps); the prefactor 1/N is applied at the end.  The two
// forms are separate instantiations: with the choice inside the loop the compiler
// predicates the square root into every iteration of the eps = 0 sum.
template <bool SOFT>
__global__ void __launch_bounds__(NT) potential_sheet_tiles_kernel(const double *__restrict__ q, int64_t N,
                                                                    int ntiles, double eps, double *unit_sums) {
  const int ti = blockIdx.x, tj = blockIdx.y;
  if (tj < ti) return;
  __shared__ double sx[PT];
  const int64_t j0 = (int64_t)tj * PT;
  for (int t = threadIdx.x; t < PT; t += NT) {
    const int64_t j = j0 + t;
    if (j < N) sx[t] = q[j];
  }
  __syncthreads();
  const int64_t i = (int64_t)ti * PT + threadIdx.x;
  double s = 0.0;
  if (i < N) {
    const double x = q[i];
    const int kbeg = ti == tj ? threadIdx.x + 1 : 0;  // j > i inside the diagonal tile
    const int kend = (int)((N - j0) < PT ? (N - j0) : PT);
    for (int k = kbeg; k < kend; k++) {
      const double d = x - sx[k];
      if constexpr (SOFT)
        s += sqrt(fma(d, d, eps));
      else
        s += fabs(d);
    }
  }
  __shared__ double2 red[NT / 32];
  double2 b = block_sum2<NT>(s, 0.0, red);
  if (threadIdx.x == 0) unit_sums[(int64_t)ti * ntiles + tj] = b.x;
}

int grid_sum(md_ctx *c, int64_t n) {
  int64_t g = (n + NT - 1) / NT;
  int64_t cap = (int64_t)c->nsm * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

namespace {

// V of Eqs. 1 / 3 / 5 from the device sums, written to a device scalar.
__global__ void potential_finalize_kernel(int model, int64_t N, const double *sums, double *V) {
  const double n = (double)N;
  if (model == MD_HMF) {
    const double mx = sums[0] / n, my = sums[1] / n;
    *V = 0.5 * n * (1.0 - mx * mx - my * my);
  } else if (model == MD_RING) {
    *V = -sums[0] / (2.0 * n);
  } else if (model == MD_GRAV3D) {
    *V = -sums[0] / n;
  } else if (model == MD_SHEET1D) {
    *V = sums[0] / n;
  } else {
    *V = sums[0] / n;
  }
}

}  // namespace

// Potential energy into device *V with all scratch supplied by the caller:
// unit_sums (>= ceil(N/256)^2 doubles, zeroed by the caller), ag (>= N double2,
// 16-byte aligned; Ring only), partials (>= grid_cap doubles), sums (>= 2
// doubles), ticket (zeroed).  Same kernels and summation order as md_energy.
int potential_with_scratch(cudaStream_t st, int nsm, int grid_cap, int model, int64_t N, double eps,
                           const double *q, double *unit_sums, double2 *ag, double *partials, double *sums,
                           unsigned *ticket, double *V) {
  if (model == MD_HMF) {
    hmf_sums_raw(st, nsm, grid_cap, q, N, partials, sums, ticket);
  } else {
    const int ntiles = (int)((N + PT - 1) / PT);
    if (model == MD_RING) {
      int64_t b = (N + 255) / 256;
      if (b > (int64_t)nsm * 16) b = (int64_t)nsm * 16;
      half_angle_kernel<<<(int)b, 256, 0, st>>>(q, N, ag);
      potential_tiles_kernel<MD_RING><<<dim3(ntiles, ntiles), NT, 0, st>>>(q, ag, N, ntiles, 0.5 * eps, unit_sums);
    } else if (model == MD_GRAV3D) {
      potential3d_tiles_kernel<<<dim3(ntiles, ntiles), NT, 0, st>>>(q, N, ntiles, eps, unit_sums);
    } else if (model == MD_SHEET1D) {
      if (eps > 0.0)
        potential_sheet_tiles_kernel<true><<<dim3(ntiles, ntiles), NT, 0, st>>>(q, N, ntiles, eps, unit_sums);
      else
        potential_sheet_tiles_kernel<false><<<dim3(ntiles, ntiles), NT, 0, st>>>(q, N, ntiles, eps, unit_sums);
    } else {
      potential_tiles_kernel<MD_GRAV2D><<<dim3(ntiles, ntiles), NT, 0, st>>>(q, nullptr, N, ntiles, eps, unit_sums);
    }
    const int64_t units = (int64_t)ntiles * ntiles;
    int64_t g = (units + NT - 1) / NT;
    if (g > (int64_t)nsm * 8) g = (int64_t)nsm * 8;
    if (g > grid_cap) g = grid_cap;
    sum_kernel<false><<<(int)g, NT, 0, st>>>(unit_sums, units, partials, sums, ticket);
  }
  potential_finalize_kernel<<<1, 1, 0, st>>>(model, N, sums, V);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MD_OK : MD_ECUDA;
}

int reduce_scratch(md_ctx *c, size_t bytes) {
  if (bytes <= c->red_bytes) return MD_OK;
  dev_free(c->red);
  c->red = (double *)dev_alloc(bytes);
  if (!c->red) {
    c->red_bytes = 0;
    return set_err(c, MD_ENOMEM, "reduction scratch: %zu bytes", bytes);
  }
  c->red_bytes = bytes;
  return MD_OK;
}

// Kinetic energy (1/2) sum p^2 into device *d_out.  The CTA partials use the
// HMF partial buffer and ticket (sized for the largest streaming grid).
int kinetic_fp64(md_ctx *c, double *d_out) {
  const int64_t n = (int64_t)c->dim * c->N;
  int g = grid_sum(c, n);
  if (g > c->hmf_grid_max) g = c->hmf_grid_max;
  sum_kernel<true><<<g, NT, 0, c->stream>>>(c->p, n, c->hmf_partials, d_out, c->hmf_ticket);
  MD_LAUNCHED(c);
  return MD_OK;
}

// Deterministic FP64 (1/2) sum of x[i]^2 over x[0..n) into device *d_out.
int half_sumsq_fp64(md_ctx *c, const double *x, int64_t n, double *d_out) {
  int g = grid_sum(c, n);
  if (g > c->hmf_grid_max) g = c->hmf_grid_max;
  sum_kernel<true><<<g, NT, 0, c->stream>>>(x, n, c->hmf_partials, d_out, c->hmf_ticket);
  MD_LAUNCHED(c);
  return MD_OK;
}

// Deterministic FP64 sum of x[0..n) into device *d_out.
int sum_fp64(md_ctx *c, const double *x, int64_t n, double *d_out) {
  int g = grid_sum(c, n);
  if (g > c->hmf_grid_max) g = c->hmf_grid_max;
  sum_kernel<false><<<g, NT, 0, c->stream>>>(x, n, c->hmf_partials, d_out, c->hmf_ticket);
  MD_LAUNCHED(c);
  return MD_OK;
}

// Pair-sum part of the potential of Eq. 1 (Ring), Eq. 3 (2D) or of the 3D model,
// prefactor applied by the caller, into device *d_out.  Uses ctx->red as scratch.
int pair_potential_fp64(md_ctx *c, double *d_out) {
  const int64_t N = c->N;
  const int ntiles = (int)((N + PT - 1) / PT);
  if (ntiles > 65535) return set_err(c, MD_EINVAL, "potential: N too large for the tile grid");
  size_t units = (size_t)ntiles * ntiles;
  const size_t units_al = (units + 1) & ~(size_t)1;  // keeps the double2 array 16-byte aligned
  size_t need = units_al * sizeof(double) + (c->model == MD_RING ? (size_t)N * sizeof(double2) : 0) + 64;
  int rc = reduce_scratch(c, need);
  if (rc) return rc;
  double *unit_sums = c->red;
  double2 *ag = (double2 *)(c->red + units_al);
  MD_CUDA(c, cudaMemsetAsync(unit_sums, 0, units * sizeof(double), c->stream));
  if (c->model == MD_RING) {
    int64_t b = (N + 255) / 256;
    if (b > (int64_t)c->nsm * 16) b = (int64_t)c->nsm * 16;
    half_angle_kernel<<<(int)b, 256, 0, c->stream>>>(c->q, N, ag);
    MD_LAUNCHED(c);
    potential_tiles_kernel<MD_RING><<<dim3(ntiles, ntiles), NT, 0, c->stream>>>(c->q, ag, N, ntiles, 0.5 * c->eps,
                                                                                unit_sums);
  } else if (c->model == MD_GRAV3D) {
    potential3d_tiles_kernel<<<dim3(ntiles, ntiles), NT, 0, c->stream>>>(c->q, N, ntiles, c->eps, unit_sums);
  } else if (c->model == MD_SHEET1D) {
    if (c->eps > 0.0)
      potential_sheet_tiles_kernel<true><<<dim3(ntiles, ntiles), NT, 0, c->stream>>>(c->q, N, ntiles, c->eps, unit_sums);
    else
      potential_sheet_tiles_kernel<false><<<dim3(ntiles, ntiles), NT, 0, c->stream>>>(c->q, N, ntiles, c->eps, unit_sums);
  } else {
    potential_tiles_kernel<MD_GRAV2D><<<dim3(ntiles, ntiles), NT, 0, c->stream>>>(c->q, nullptr, N, ntiles, c->eps,
                                                                                  unit_sums);
  }
  MD_LAUNCHED(c);
  int g = grid_sum(c, (int64_t)units);
  if (g > c->hmf_grid_max) g = c->hmf_grid_max;
  sum_kernel<false><<<g, NT, 0, c->stream>>>(unit_sums, (int64_t)units, c->hmf_partials, d_out, c->hmf_ticket);
  MD_LAUNCHED(c);
  return MD_OK;
}
