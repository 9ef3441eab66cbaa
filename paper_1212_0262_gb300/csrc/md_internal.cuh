// Internal declarations shared by the libmd translation units.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>

#include "md.h"

// ------------------------------------------------------------------ tuning --

// Threads per CTA of the streaming (HMF, elementwise) kernels.
constexpr int kStreamThreads = 256;
// Threads per CTA of the all-pairs kernels.
constexpr int kPairThreads = 128;

struct PairTuning {
  int r_mixed = 8;    // i-particles per thread, FP32 pair path
  int r_fp64 = 2;     // i-particles per thread, FP64 pair path
  int tj = 256;       // j-tile (particles staged in shared memory per unit)
  int ring_tc = 1;    // Ring FP32: sin(d) and sin(d/2) from tensor-core MMAs (split TF32); 1: 4, 2: 2 m-blocks per warp
  int symmetric = 1;  // forward stages: each unordered pair once (Newton's third law)
  int ctas_per_sm = 0;  // 0: occupancy-derived
  int vcta = 0;         // stream-K ranges per resident CTA (0: the kernel's default)
};

struct HmfTuning {
  int ctas_per_sm = 0;  // 0: occupancy-derived
};

// ----------------------------------------------------------------- context --

// Everything the launches of a captured block of md_step's steps depend on,
// besides the ping-pong parity (one graph per parity).  Compared bytewise.
struct StepGraphKey {
  int model, prec;
  int64_t N;
  double h, eps;
  void *stream;
  PairTuning pt;
  HmfTuning ht;
  int mirror_fmt;
  const void *bufs[14];
};

struct md_ctx {
  int model = 0, dim = 1, prec = MD_FP64;
  int64_t N = 0;
  double eps = 0.0, dt = 0.0;
  int device = 0, nsm = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;

  double *q = nullptr, *p = nullptr;  // dim*N each (FP64 state)
  double *f = nullptr;                // dim*N: first-same-as-last force cache / scratch force
  bool fsal_valid = false;            // f holds the force at the current q
  int fsal_prec = -1;

  // HMF: per-CTA partial sums, magnetization double buffer, finish ticket
  double *hmf_partials = nullptr;  // 2 * hmf_grid_max
  double *hmf_m = nullptr;         // [2][2]: (sum cos, sum sin) of the current / next angles
  unsigned *hmf_ticket = nullptr;
  int hmf_grid_max = 0;
  int hmf_cur = 0;
  int hmf_rev = 0;                    // sweep direction of the next stage (alternates)
  bool hmf_m_valid = false;           // FP64: the (cos, sin) buffer is valid with the sums
  double *hmf_cs = nullptr;           // FP64 path: (cos, sin) of the current angles, N double2
  size_t hmf_cs_bytes = 0;
  int hmf_m_prec = -1;

  // Ring / 2D: position mirrors (ping-pong), stream-K partial slots and tickets
  void *mirror[2] = {nullptr, nullptr};
  size_t mirror_bytes = 0;
  int mirror_cur = 0;
  bool mirror_valid = false;
  int mirror_prec = -1;
  int mirror_fmt = -1;  // record format of the valid mirror (0 interleaved, 1 Ring / 2 2D tensor-core fragments)
  double *sk_slots = nullptr;
  size_t sk_slots_bytes = 0;
  unsigned *sk_tickets = nullptr;
  size_t sk_tickets_count = 0;
  double *sym_rowfull = nullptr;  // Newton's-third-law variant: row partials of whole rows
  size_t sym_rowfull_bytes = 0;
  void *sym_colslot = nullptr;    // and column partials per unit (FP32 or FP64)
  size_t sym_colslot_bytes = 0;
  double *sym_chunks = nullptr;   // and chunk sums of the column partials
  size_t sym_chunk_bytes = 0;

  // reductions (energies)
  double *red = nullptr;
  size_t red_bytes = 0;
  // md_grad workspace: checkpoints, lambda_q, lambda_p, eps terms, sums
  double *gw = nullptr;
  size_t gw_bytes = 0;
  double *host_scalars = nullptr;  // pinned, 16 doubles

  PairTuning pt;
  HmfTuning ht;
  int64_t launches = 0;
  std::string err;

  // md_step: steps 2.. replayed from CUDA graphs of kStepGraphSteps steps, one per parity
  cudaGraphExec_t step_graph[2] = {nullptr, nullptr};
  StepGraphKey step_key[2];
  int64_t step_graph_launches[2] = {0, 0};
  bool use_graphs = true;

  // Row shard (md_shard_*): the state holds rows [row0, row0 + N) of a system of
  // n_total particles split among shard_nranks ranks (n_total == N, row0 == 0 for a
  // whole system).  Ring / 2D keep the whole position mirror (n_total records); HMF
  // keeps every rank's (sum cos, sum sin) in shard_sums[2][nranks][2] (ping-pong).
  bool shard = false;
  int shard_rank = 0, shard_nranks = 1;
  int64_t n_total = 0, row0 = 0;
  double *shard_sums = nullptr;
  int shard_cur = 0;
  bool shard_primed = false;       // this rank's segment of the exchange buffer is written
  int shard_prec = -1;             // precision the shard was primed in
  cudaEvent_t shard_event = nullptr;
};

constexpr int kMaxShards = 64;
// Ring / 2D row shards start on multiples of this many rows (whole mirror record
// groups and whole i-tiles of every pair kernel).
constexpr int64_t kShardRowAlign = 1024;

// ------------------------------------------------------------ host helpers --

// Smallest positive softening accepted.  Every softened square distance
// |r|^2 + eps (and the Ring's 1 - cos d + eps) is then at least this, a normal
// number in FP32, the precision in which the FP32 pair kernels divide and the FP64
// ones take the seeds of their reciprocals and reciprocal square roots.
constexpr double kEpsMin = 1e-30;

// eps is finite, >= 0, and either 0 (HMF, and the sheets' unsoftened force only)
// or >= kEpsMin.
inline bool eps_valid(int model, double eps) {
  if (!(eps == eps) || eps - eps != 0.0 || eps < 0.0) return false;
  if (eps == 0.0) return model == MD_HMF || model == MD_SHEET1D;
  return eps >= kEpsMin;
}

int set_err(md_ctx *c, int code, const char *fmt, ...);
int cuda_err(md_ctx *c, cudaError_t e, const char *what);
void *dev_alloc(size_t bytes);
void dev_free(void *p);
#define MD_CUDA(ctx, call)                                        \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return cuda_err((ctx), e_, #call);     \
  } while (0)
#define MD_LAUNCHED(ctx)                                                      \
  do {                                                                        \
    (ctx)->launches++;                                                        \
    cudaError_t e_ = cudaGetLastError();                                      \
    if (e_ != cudaSuccess) return cuda_err((ctx), e_, "kernel launch");       \
  } while (0)

void destroy_step_graphs(md_ctx *c);

// Yoshida coefficients of Eq. 4 (B0, B1, D0, D1), from the triple-jump closed form.
void yoshida_coefficients(double c[4]);

// ---------------------------------------------------------- kernel drivers --

// Stage modes of the fused force kernels.
enum StageMode {
  STAGE_KICK_DRIFT = 0,  // f(q); p += kick f; q += drift p; refresh mirror / reduction
  STAGE_KICK_ONLY = 1,   // f(q); p += kick f; store f in ctx->f (first-same-as-last cache)
  STAGE_FORCE_ONLY = 2,  // f(q) into an output array
  STAGE_ADJOINT = 3,     // reverse stage of md_grad (kick adjoint and undo, drift adjoint and undo)
  STAGE_TANGENT = 4,     // forward stage of the tangent dynamics (state and tangent vector together)
};

// pairs.cu / hmf.cu: one forward stage of the tangent (linearised) dynamics,
//   p += kick f(q);  dp += kick J(q) dq;  then, if drift != 0: q += drift p;  dq += drift dp.
// The pair version reads adjoint-format records holding (q, dq).
int pair_tangent_stage(md_ctx *c, double kick, double drift, double *dq, double *dp);
int hmf_tangent_stage(md_ctx *c, double kick, double drift, double *dq, double *dp, const double *s_in,
                      double *s_out);

// api.cu: nsteps integrator steps of Sec. 3 on the context's state (md_step's body).
int integrate(md_ctx *c, int64_t nsteps);

// pairs.cu: adjoint records (position and lambda_p) and one reverse stage:
//   lambda_q += b_adj J(q) lambda_p; epsacc += b_adj <lambda_p, df/deps>;
//   p -= b_undo f(q); then, if drift != 0: lambda_p += drift lambda_q; q -= drift p.
int adjoint_mirror_refresh(md_ctx *c, const double *lp);
int pair_adjoint_stage(md_ctx *c, double b_adj, double b_undo, double drift, double *lq, double *lp,
                       double *epsacc);

// hmf.cu: the same reverse stage in mean-field form; sums = (sum cos, sum sin,
// sum cos lambda_p, sum sin lambda_p) of the current state.
int hmf_adjoint_prime(md_ctx *c, const double *lp, double *sums);
int hmf_adjoint_stage(md_ctx *c, double b_adj, double b_undo, double drift, double *lq, double *lp,
                      const double *s_in, double *s_out);
int hmf_magnetization_terminal(md_ctx *c, double cx, double cy, double *lq);

// hmf.cu
int hmf_prime(md_ctx *c);                                         // sums of the current angles
int hmf_sincos_table(md_ctx *c, bool probe);  // the FP64 stages' sine/cosine table on the context's device
int hmf_stage(md_ctx *c, int mode, double kick, double drift, double *fout);
int hmf_sums_fp64(md_ctx *c, double *d_out2);                     // FP64 (sum cos, sum sin) into device out
int hmf_sums_fp64_of(md_ctx *c, const double *q, double *d_out2);

// pairs.cu
int mirror_refresh(md_ctx *c);                                    // mirror[mirror_cur] from q
int pair_stage(md_ctx *c, int mode, double kick, double drift, double *fout);
int kick_drift_cached(md_ctx *c, double kick, double drift);      // first stage from the cached force
int ensure_pair_buffers(md_ctx *c, int TI, int P, int nacc);       // stream-K slots and tickets

// sym.cu (Newton's-third-law variant of the FP32 forward stages)
bool sym_applies(const md_ctx *c);
int sym_pair_stage(md_ctx *c, int mode, double kick, double drift, double *fout);

// pairs.cu / hmf.cu: row shards (md_shard_*).  *_shard_prime writes this rank's segment of
// the exchange buffer from its state; *_shard_stage runs one fused stage over the shard's
// rows (STAGE_KICK_DRIFT, drift 0 allowed, or STAGE_FORCE_ONLY into fout); *_shard_segment
// gives the exchange buffer and this rank's byte range in it.
int pair_shard_prime(md_ctx *c);
int pair_shard_stage(md_ctx *c, int mode, double kick, double drift, double *fout);
int pair_shard_segment(md_ctx *c, void **buf, size_t *off, size_t *bytes);
int hmf_shard_prime(md_ctx *c);
int hmf_shard_stage(md_ctx *c, int mode, double kick, double drift, double *fout);

// api.cu: a context for rows [row0, row0 + n_local) of a system of n_total particles
// (the whole system when n_local == n_total), state drawn with the global counters.
md_ctx *create_context(int model, int64_t n_local, int64_t n_total, int64_t row0, double eps, double dt,
                       uint64_t seed, const char *who);

// energy.cu
int kinetic_fp64(md_ctx *c, double *d_out);                       // (1/2) sum p^2 into device out
int pair_potential_fp64(md_ctx *c, double *d_out);                // i<j sum of Eq. 1 / Eq. 3
int reduce_scratch(md_ctx *c, size_t bytes);
int sum_fp64(md_ctx *c, const double *x, int64_t n, double *d_out);  // deterministic sum into device out
int half_sumsq_fp64(md_ctx *c, const double *x, int64_t n, double *d_out);  // (1/2) sum x^2 into device out

// ic.cu
int ic_draw(md_ctx *c, int kind, const double *params, uint64_t seed);

// Raw-scratch launchers (no context, no allocation).
void hmf_sums_raw(cudaStream_t st, int nsm, int grid_cap, const double *q, int64_t N, double *partials,
                  double *out2, unsigned *ticket);
int potential_with_scratch(cudaStream_t st, int nsm, int grid_cap, int model, int64_t N, double eps,
                           const double *q, double *unit_sums, double2 *ag, double *partials, double *sums,
                           unsigned *ticket, double *V);

// -------------------------------------------------------- device helpers ----
#ifdef __CUDACC__

__device__ __forceinline__ float mufu_rsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float mufu_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Seeds for the FP64 reciprocal (square) roots below.  A positive double becomes a
// float by moving bits (mantissa truncated; beyond the float range +inf, below the
// normal range 0), and a non-negative float a double the same way, so neither
// conversion runs on the FP64 pipe, which bounds the FP64 pair kernels.
__device__ __forceinline__ float seed_d2f(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned f = ((hi - 0x38000000u) << 3) | (lo >> 29);
  return __uint_as_float(hi >= 0x47F00000u ? 0x7f800000u : hi < 0x38100000u ? 0u : f);
}
__device__ __forceinline__ double seed_f2d(float f) {
  const unsigned u = __float_as_uint(f);
  if (u == 0u) return 0.0;
  if (u >= 0x7f800000u) return __longlong_as_double(0x7ff0000000000000LL);
  return __hiloint2double((int)((u >> 3) + 0x38000000u), (int)(u << 29));
}

// 1/sqrt(d) in FP64 for d in the normal float range: FP32 hardware seed y (relative
// error below 2^-22), then one third-order Householder step for y^-2 = d:
// e = 1 - d y^2, y <- y (1 + e/2 + 3 e^2/8) (the series of (1 - e)^(-1/2) to e^2),
// which leaves a truncation error of (5/16) e^3 < 2^-63.
__device__ __forceinline__ double rsqrt_nr(double d) {
  const double y = seed_f2d(mufu_rsqrt(seed_d2f(d)));
  const double e = fma(-(d * y), y, 1.0);
  return fma(y * e, fma(0.375, e, 0.5), y);
}

// 1/s in FP64 for s in the normal float range: FP32 hardware seed y, then one
// third-order step e = 1 - s y, y <- y (1 + e + e^2) (truncation error e^3 < 2^-66).
__device__ __forceinline__ double rcp_nr(double s) {
  const double y = seed_f2d(mufu_rcp(seed_d2f(s)));
  const double e = fma(-s, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// sin and cos of a float of modest size (|x| < 2^20), for arguments that were
// already range-reduced in FP64.  x = k pi/2 + y with k the nearest integer
// (found with the 1.5*2^23 rounding constant, which also leaves k mod 4 in the
// low mantissa bits) and pi/2 split into two floats (each FMA keeps k*C exact
// before its single rounding); then the Taylor series of sin and cos on
// |y| <= pi/4, whose truncation errors there are 1.8e-9 and 1.2e-10.
__device__ __forceinline__ void sincos_small(float x, float *s, float *c) {
  const float t = fmaf(x, 0.636619772f, 12582912.0f);
  const int q = __float_as_int(t) & 3;
  const float k = t - 12582912.0f;
  float y = fmaf(-k, 1.5707963705062866f, x);
  y = fmaf(-k, -4.371138828673793e-08f, y);
  const float z = y * y;
  float ps = fmaf(z, 1.0f / 362880.0f, -1.0f / 5040.0f);
  ps = fmaf(z, ps, 1.0f / 120.0f);
  ps = fmaf(z, ps, -1.0f / 6.0f);
  const float sy = fmaf(y * z, ps, y);
  float pc = fmaf(z, -1.0f / 3628800.0f, 1.0f / 40320.0f);
  pc = fmaf(z, pc, -1.0f / 720.0f);
  pc = fmaf(z, pc, 1.0f / 24.0f);
  pc = fmaf(z, pc, -0.5f);
  const float cy = fmaf(z, pc, 1.0f);
  const float a = (q & 1) ? cy : sy;
  const float b = (q & 1) ? sy : cy;
  *s = (q & 2) ? -a : a;
  *c = ((q + 1) & 2) ? -b : b;
}

// Exact float -> double by moving bits (no FP64 instruction): exponent rebias
// 127 -> 1023 and mantissa shift 23 -> 52.  Zero and subnormal floats give a
// signed zero; infinities and NaN are not handled (they never reach it).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7fffffffu;
  unsigned hi = (u & 0x80000000u) | ((a >> 3) + 0x38000000u);
  unsigned lo = a << 29;
  if (a < 0x00800000u) {
    hi = u & 0x80000000u;
    lo = 0u;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// double -> float by truncating the mantissa (moving bits, no FP64 instruction),
// for |d| below 2^128; magnitudes below the float normal range give zero.
__device__ __forceinline__ float d2f_trunc_bits(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned a = hi & 0x7fffffffu;
  unsigned fb = ((a - 0x38000000u) << 3) | (lo >> 29);
  if (a < 0x38100000u) fb = 0u;
  return __uint_as_float((hi & 0x80000000u) | fb);
}

// theta - 2 pi k (k the nearest integer to theta / 2 pi) as a float, for
// |theta| < 2^20, using no FP64 instruction.  theta = th_hi + th_lo exactly up
// to its last 6 bits: th_hi is theta truncated to a float and th_lo the next 23
// mantissa bits (an integer made exact by the 2^23 magic constant, scaled by a
// power of two built from theta's exponent).  Then one Cody-Waite step with
// 2 pi split into two floats.  Absolute error a few 1e-7.
__device__ __forceinline__ float reduce_2pi_f(double th) {
  const unsigned hi = (unsigned)__double2hiint(th), lo = (unsigned)__double2loint(th);
  const unsigned sign = hi & 0x80000000u, a = hi & 0x7fffffffu, E = a >> 20;
  float th_hi = __uint_as_float(sign | (((a - 0x38000000u) << 3) | (lo >> 29)));
  const unsigned m23 = (lo & 0x1fffffffu) >> 6;  // weight of bit 0: 2^(E - 1069)
  float th_lo = (__uint_as_float(0x4b000000u | m23) - 8388608.0f) * __uint_as_float((E - 942u) << 23);
  th_lo = __uint_as_float(__float_as_uint(th_lo) | sign);
  if (E < 943u) th_lo = 0.0f;
  if (E < 897u) th_hi = 0.0f;
  const float t = fmaf(th_hi, 0.15915493667125702f, 12582912.0f);
  const float k = t - 12582912.0f;
  float r = fmaf(-k, 6.2831854820251465f, th_hi);
  r = fmaf(-k, -1.7484555314695172e-07f, r);
  return r + th_lo;
}

// theta - 2 pi k with k = rint(theta / 2 pi), in FP64 (two-constant Cody-Waite).
__device__ __forceinline__ double reduce_2pi(double th) {
  const double inv2pi = 0.15915494309189535;
  const double hi = 6.283185307179586;       // 2 pi rounded to double
  const double lo = 2.4492935982947064e-16;  // 2 pi - hi
  double k = rint(th * inv2pi);
  double r = fma(-k, hi, th);
  return fma(-k, lo, r);
}

// Deterministic block sum of two doubles (fixed shuffle tree, then warps in order).
template <int NT>
__device__ __forceinline__ double2 block_sum2(double a, double b, double2 *smem) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) smem[w] = make_double2(a, b);
  __syncthreads();
  double2 r = make_double2(0.0, 0.0);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NT / 32; i++) {
      r.x += smem[i].x;
      r.y += smem[i].y;
    }
  }
  return r;  // valid in thread 0
}

#endif  // __CUDACC__
