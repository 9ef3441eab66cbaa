// Seeded initial states drawn on the device.
//
// Generator: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used counter-based:
// draw k of a seed is mix(seed + (k + 1) * 0x9E3779B97F4A7C15), the k-th output
// of the sequential generator started at state `seed`.  Uniform: (x >> 11) 2^-53.
// Gaussian: Box-Muller (1958) from two consecutive uniforms,
// sqrt(-2 log(1 - u1)) cos(2 pi u2).  Draw order: positions first, then momenta.
// Affine maps are (hi - lo) * u + lo with two separate roundings (no FMA), so
// the uniform-based arrays are bit-identical to any other implementation of the
// same recipe.
#include "md_internal.cuh"

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double u01(uint64_t seed, uint64_t k) {
  return (double)(splitmix64(seed, k) >> 11) * 0x1.0p-53;
}

__device__ __forceinline__ double affine(double u, double width, double lo) {
  return __dadd_rn(__dmul_rn(width, u), lo);
}

__device__ __forceinline__ double gauss(uint64_t seed, uint64_t k) {
  const double two_pi = 2.0 * M_PI;
  double u1 = u01(seed, k), u2 = u01(seed, k + 1);
  double m = __dmul_rn(-2.0, log(__dsub_rn(1.0, u1)));
  return __dmul_rn(sqrt(m), cos(__dmul_rn(two_pi, u2)));
}

struct IcArgs {
  double *q, *p;
  int64_t N;         // rows held (leading dimension of q and p)
  int64_t Ng, row0;  // the whole system's size and the global index of row 0 (counters)
  int kind;
  uint64_t seed;
  double a0, a1, a2, a3;  // recipe parameters (widths and offsets precomputed on the host)
};

__global__ void ic_kernel(IcArgs a) {
  const double two_pi = 2.0 * M_PI;
  const int64_t N = a.N;
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += G) {
    const uint64_t ui = (uint64_t)(a.row0 + i), un = (uint64_t)a.Ng;
    switch (a.kind) {
    case MD_IC_WATERBAG:  // a0 = th width, a1 = th_lo, a2 = p width, a3 = p_lo
      a.q[i] = affine(u01(a.seed, ui), a.a0, a.a1);
      a.p[i] = affine(u01(a.seed, un + ui), a.a2, a.a3);
      break;
    case MD_IC_RING:  // a0 = 2 pi, a1 = -pi, a2 = sigma
      a.q[i] = affine(u01(a.seed, ui), a.a0, a.a1);
      a.p[i] = __dmul_rn(a.a2, gauss(a.seed, un + 2 * ui));
      break;
    case MD_IC_UNIFORM_REST:
      a.q[i] = affine(u01(a.seed, ui), a.a0, a.a1);
      a.p[i] = 0.0;
      break;
    case MD_IC_DISK:     // a2 = sigma
    case MD_IC_ANNULUS: {  // a0 = r2^2 - r1^2, a1 = r1^2
      double u = u01(a.seed, 2 * ui), v = u01(a.seed, 2 * ui + 1);
      double r = a.kind == MD_IC_DISK ? sqrt(u) : sqrt(__dadd_rn(__dmul_rn(a.a0, u), a.a1));
      double phi = __dmul_rn(two_pi, v);
      a.q[i] = __dmul_rn(r, cos(phi));
      a.q[N + i] = __dmul_rn(r, sin(phi));
      if (a.kind == MD_IC_DISK) {
        a.p[i] = __dmul_rn(a.a2, gauss(a.seed, 2 * un + 2 * ui));
        a.p[N + i] = __dmul_rn(a.a2, gauss(a.seed, 2 * un + 2 * (un + ui)));
      } else {
        a.p[i] = a.p[N + i] = 0.0;
      }
      break;
    }
    case MD_IC_BALL: {  // a2 = sigma; counters 3i .. 3i+2, then Gaussian momenta
      double u = u01(a.seed, 3 * ui), v = u01(a.seed, 3 * ui + 1), w = u01(a.seed, 3 * ui + 2);
      double r = cbrt(u);
      double ct = __dsub_rn(1.0, __dmul_rn(2.0, v));
      double st = sqrt(fmax(0.0, __dsub_rn(1.0, __dmul_rn(ct, ct))));
      double phi = __dmul_rn(two_pi, w);
      double rs = __dmul_rn(r, st);
      a.q[i] = __dmul_rn(rs, cos(phi));
      a.q[N + i] = __dmul_rn(rs, sin(phi));
      a.q[2 * N + i] = __dmul_rn(r, ct);
      for (int d = 0; d < 3; d++) a.p[d * N + i] = __dmul_rn(a.a2, gauss(a.seed, 3 * un + 2 * (d * un + ui)));
      break;
    }
    }
  }
}

}  // namespace

int ic_draw(md_ctx *c, int kind, const double *params, uint64_t seed) {
  IcArgs a;
  a.q = c->q;
  a.p = c->p;
  a.N = c->N;
  a.Ng = c->n_total;
  a.row0 = c->row0;
  a.kind = kind;
  a.seed = seed;
  a.a0 = a.a1 = a.a2 = a.a3 = 0.0;
  const bool angle = c->model == MD_HMF || c->model == MD_RING;
  switch (kind) {
  case MD_IC_WATERBAG:
    if (!angle && c->model != MD_SHEET1D) return set_err(c, MD_EINVAL, "water-bag needs an angle or sheet model");
    {
      // defaults: HMF theta~U[-1,1), p~U[-1.2,1.2); sheets x~U[-1,1), p~U[-0.5,0.5)
      const double pd = c->model == MD_SHEET1D ? 0.5 : 1.2;
      double tl = params ? params[0] : -1.0, th = params ? params[1] : 1.0;
      double pl = params ? params[2] : -pd, ph = params ? params[3] : pd;
      if (!(th > tl) || !(ph >= pl)) return set_err(c, MD_EINVAL, "water-bag: empty interval");
      a.a0 = th - tl;
      a.a1 = tl;
      a.a2 = ph - pl;
      a.a3 = pl;
    }
    break;
  case MD_IC_RING:
    if (!angle) return set_err(c, MD_EINVAL, "ring initial state needs an angle model");
    a.a0 = M_PI - (-M_PI);
    a.a1 = -M_PI;
    a.a2 = params ? params[0] : 0.5;
    if (!(a.a2 >= 0.0)) return set_err(c, MD_EINVAL, "sigma must be >= 0");
    break;
  case MD_IC_UNIFORM_REST:
    if (!angle) return set_err(c, MD_EINVAL, "uniform-at-rest needs an angle model");
    a.a0 = M_PI - (-M_PI);
    a.a1 = -M_PI;
    break;
  case MD_IC_DISK:
    if (c->model != MD_GRAV2D) return set_err(c, MD_EINVAL, "disk needs the 2D model");
    a.a2 = params ? params[0] : 0.3;
    if (!(a.a2 >= 0.0)) return set_err(c, MD_EINVAL, "sigma must be >= 0");
    break;
  case MD_IC_ANNULUS: {
    if (c->model != MD_GRAV2D) return set_err(c, MD_EINVAL, "annulus needs the 2D model");
    double r1 = params ? params[0] : 1.0, r2 = params ? params[1] : 1.5;
    if (!(r1 >= 0.0) || !(r2 > r1)) return set_err(c, MD_EINVAL, "annulus: need 0 <= r1 < r2");
    a.a0 = r2 * r2 - r1 * r1;
    a.a1 = r1 * r1;
    break;
  }
  case MD_IC_BALL:
    if (c->model != MD_GRAV3D) return set_err(c, MD_EINVAL, "ball needs the 3D model");
    a.a2 = params ? params[0] : 0.3;
    if (!(a.a2 >= 0.0)) return set_err(c, MD_EINVAL, "sigma must be >= 0");
    break;
  default:
    return set_err(c, MD_EINVAL, "unknown initial-state kind %d", kind);
  }
  int64_t blocks = (c->N + 255) / 256;
  if (blocks > (int64_t)c->nsm * 16) blocks = (int64_t)c->nsm * 16;
  ic_kernel<<<(int)blocks, 256, 0, c->stream>>>(a);
  MD_LAUNCHED(c);
  c->fsal_valid = false;
  c->hmf_m_valid = false;
  c->mirror_valid = false;
  c->shard_primed = false;
  return MD_OK;
}
