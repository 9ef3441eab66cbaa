// Shared pieces of the all-pairs kernels (single systems in pairs.cu, batched
// ensembles in batch.cu): launch arguments, mirror records, per-model pair
// policies (tile bodies) and epilogues.  See pairs.cu for the method.
#pragma once
#include <algorithm>
#include <type_traits>

#include "md_internal.cuh"

namespace {

constexpr int NT = kPairThreads;
constexpr int kPadMultiple = 1024;  // mirror padding: multiple of every TI and TJ

// bytes per particle of a mirror record
template <int MODEL, bool MIXED, bool ADJ>
struct RecordBytes {
  static constexpr int value = MODEL == MD_RING      ? (MIXED ? (ADJ ? 24 : 16) : (ADJ ? 48 : 32))
                               : MODEL == MD_GRAV3D  ? (MIXED ? (ADJ ? 24 : 16) : (ADJ ? 64 : 32))
                               : MODEL == MD_SHEET1D ? (MIXED ? (ADJ ? 8 : 4) : (ADJ ? 16 : 8))
                                                     : (MIXED ? (ADJ ? 16 : 8) : (ADJ ? 32 : 16));
};

// spatial components of a model's positions
template <int MODEL>
constexpr int dim_of() {
  return MODEL == MD_GRAV2D ? 2 : MODEL == MD_GRAV3D ? 3 : 1;
}

// 3D records: FP32, per particle pair (2k, 2k+1) the floats (-x, -x', -y, -y'),
// (-z, -z', 0, 0); FP64, per particle (x, y, z, 0).  Padding: far enough that
// |r|^2 overflows (FP32: 3e19 per component; FP64: 1e150, whose FP32 seed of the
// reciprocal square root is 0 and stays 0), so its terms are exactly zero.
template <bool MIXED>
__device__ __forceinline__ void write_record3(void *mirror, int64_t i, double x, double y, double z) {
  if constexpr (MIXED) {
    float *m = (float *)mirror + (i >> 1) * 8 + (i & 1);
    m[0] = -(float)x;
    m[2] = -(float)y;
    m[4] = -(float)z;
    m[6] = 0.f;
  } else {
    double *m = (double *)mirror + i * 4;
    m[0] = x;
    m[1] = y;
    m[2] = z;
    m[3] = 0.0;
  }
}
// 1D-sheet records: FP32, per particle pair (2k, 2k+1) the floats (-x, -x').
// FP64 sheet records hold an order-preserving integer key of x: the bits for x >= 0,
// the bits with the magnitude flipped for x < 0, so signed comparison of keys orders
// as the doubles do (-0 is stored as +0: equal values, equal keys).  The sign of
// x_i - x_j at eps = 0 is then two integer comparisons on the ALU pipe, exactly the
// FP64 decision; at eps > 0 the kernel turns the key back into x.
__device__ __forceinline__ long long sheet_key(double x) {
  const long long b = __double_as_longlong(x + 0.0);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double sheet_unkey(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

template <bool MIXED>
__device__ __forceinline__ void write_record1(void *mirror, int64_t i, double x) {
  if constexpr (MIXED)
    ((float *)mirror)[i] = -(float)x;
  else
    ((long long *)mirror)[i] = sheet_key(x);
}
// Padding: at eps > 0 far away (FP32: x^2 overflows, so the term is d * rsqrt(inf) = 0;
// FP64: rsqrt_nr saturates to 0 beyond the float range); at eps = 0 FP32 NaN (both
// comparisons false) and FP64 the smallest key, which adds exactly +1 to every real
// row (removed in the epilogue: n_jt TJ - N padding records per row).
template <bool MIXED>
__device__ __forceinline__ void write_pad1(void *mirror, int64_t i, double eps) {
  if constexpr (MIXED)
    ((float *)mirror)[i] = eps > 0.0 ? -3.0e19f : __int_as_float(0x7fc00000);
  else
    ((long long *)mirror)[i] = eps > 0.0 ? sheet_key(1.0e150) : (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ double sheet_pad(double eps, bool mixed) {
  return eps > 0.0 ? (mixed ? 3.0e19 : 1.0e150) : __longlong_as_double(0x7FF8000000000000LL);
}

// Adjoint records (positions and lambda_p): 3D FP32 per particle pair the floats
// (-x, -x', -y, -y'), (-z, -z', -vx, -vx'), (-vy, -vy', -vz, -vz'); FP64 per particle
// (x, y, z, vx, vy, vz, 0, 0).  Sheets FP32 per pair (-x, -x', -v, -v'); FP64 (x, v).
template <bool MIXED>
__device__ __forceinline__ void write_record3_adj(void *mirror, int64_t i, const double *x, const double *v) {
  if constexpr (MIXED) {
    float *m = (float *)mirror + (i >> 1) * 12 + (i & 1);
    m[0] = -(float)x[0];
    m[2] = -(float)x[1];
    m[4] = -(float)x[2];
    m[6] = -(float)v[0];
    m[8] = -(float)v[1];
    m[10] = -(float)v[2];
  } else {
    double *m = (double *)mirror + i * 8;
    for (int d = 0; d < 3; d++) {
      m[d] = x[d];
      m[3 + d] = v[d];
    }
    m[6] = m[7] = 0.0;
  }
}
template <bool MIXED>
__device__ __forceinline__ void write_record1_adj(void *mirror, int64_t i, double x, double v) {
  if constexpr (MIXED) {
    float *m = (float *)mirror + (i >> 1) * 4 + (i & 1);
    m[0] = -(float)x;
    m[2] = -(float)v;
  } else {
    double *m = (double *)mirror + i * 2;
    m[0] = x;
    m[1] = v;
  }
}

template <bool MIXED>
__device__ __forceinline__ void write_pad3(void *mirror, int64_t i) {
  if constexpr (MIXED)
    write_record3<true>(mirror, i, 3.0e19, 3.0e19, 3.0e19);
  else
    write_record3<false>(mirror, i, 1.0e150, 1.0e150, 1.0e150);
}

// CTAs per SM that the one-sided stream-K kernel's register budget is set for: a
// policy's STREAMK_MINB when it declares one, else its MINB (the budget of its symmetric
// form), else 1 (the compiler's choice).  Budgeted, the one-sided FP32 kernels run 3-5%
// faster than at the 180-240 registers the compiler picks on its own.
template <class P, class = void>
struct StreamkMinBlocksFwd {
  static constexpr int value = 1;
};
template <class P>
struct StreamkMinBlocksFwd<P, std::void_t<decltype(P::MINB)>> {
  static constexpr int value = P::MINB;
};
template <class P, class = void>
struct StreamkMinBlocks {
  static constexpr int value = StreamkMinBlocksFwd<P>::value;
};
template <class P>
struct StreamkMinBlocks<P, std::void_t<decltype(P::STREAMK_MINB)>> {
  static constexpr int value = P::STREAMK_MINB;
};

struct PairArgs {
  const void *mirror_in;
  void *mirror_out;
  double *q, *p;
  int64_t N;
  int64_t n_it, n_jt, U;
  int P;
  double epsd;    // Ring: eps/2; 2D: eps
  double kick, drift;
  double *slots;  // [P][2][NACC][TI] FP64 partial sums
  unsigned *tickets;
  double *fout;   // STAGE_KICK_ONLY / STAGE_FORCE_ONLY force output (dim*N)
  // adjoint stages
  double *lq, *lp;   // lambda_q, lambda_p (dim*N)
  double *epsacc;    // per-particle accumulated d O / d eps terms (N)
  double undo;       // kick coefficient (times dt) removed from p
  // row shard (md_shard_*): the i-tiles cover global rows [row0, row0 + nrow) and the
  // state arrays q, p, fout hold those rows only (leading dimension nrow); the
  // mirror and N stay global
  int64_t row0, nrow;
  // dynamic stream-K: [0] next virtual CTA to take, [1] CTAs done (both 0 between launches)
  unsigned *sched;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

__host__ __device__ __forceinline__ int64_t unit_begin(int64_t U, int P, int64_t c) { return (U * c) / P; }
// CTA whose range holds unit u: max c with U c / P <= u.
__device__ __forceinline__ int64_t cta_of_unit(int64_t U, int P, int64_t u) { return ((u + 1) * P - 1) / U; }

// Dynamic stream-K.  The U units are split into P static ranges ("virtual CTAs",
// several per CTA), which the CTAs of the launch take in increasing order from
// sched[0]: the CTAs that share an SM progress unevenly under its warp schedulers,
// and with one static range per CTA the SM's last CTA ran alone, at a fraction of
// the SM's throughput, at the end of every launch.  The ranges keep every partial
// row and ticket of the static scheme; only their order of execution changes.
__device__ __forceinline__ int64_t take_vcta(unsigned *sched, unsigned &s_slot) {
  if (threadIdx.x == 0) s_slot = atomicAdd(sched, 1u);
  __syncthreads();
  const unsigned v = s_slot;
  __syncthreads();
  return (int64_t)v;
}
// After the CTA's last take: the last CTA of the launch to get here sets both
// counters back to 0 (every other CTA has taken its last virtual CTA before it
// counted itself done).
__device__ __forceinline__ void vcta_done(unsigned *sched) {
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(sched + 1, 1u) == gridDim.x - 1) {
      atomicExch(sched, 0u);
      atomicExch(sched + 1, 0u);
    }
  }
}

// The two dynamic stream-K counters of a context: after the stream-K tickets (see
// ensure_pair_buffers).
inline unsigned *pair_sched(md_ctx *c) { return c->sk_tickets + c->sk_tickets_count - 2; }

// Virtual CTAs of a dynamic stream-K launch of G CTAs over U units: k per CTA (the
// pair_vcta tuning, else the kernel's default), at least 16 units each.
inline int64_t vcta_count(int64_t G, int64_t U, int k) {
  int64_t P = G * k;
  if (P > U / 16) P = U / 16;
  if (P < G) P = G;
  if (P > U) P = U;
  return P < 1 ? 1 : P;
}

// Triangular unit table of the Newton's-third-law form: row I (i-tile of m
// j-tiles) holds the j-tiles J = m I .. n_jt - 1.
__host__ __device__ __forceinline__ int64_t sym_rowstart(int64_t I, int64_t n_jt, int m) {
  return I * n_jt - (int64_t)m * I * (I - 1) / 2;
}

// Policies with a Newton's-third-law diagonal tile (tile_diag: the above-diagonal
// pairs of an i-tile with its own particles evaluated once, with column sums).  Their
// diagonal units write column partials too, and the finish phase of tile T adds the
// column partials of the rows I <= T (else I < T).
template <class P, class = void>
struct HasDiagSym : std::false_type {};
template <class P>
struct HasDiagSym<P, std::void_t<decltype(&P::tile_diag)>> : std::true_type {};

// The row holding unit u: the largest I < n_it with rowstart(I) <= u.
__device__ int64_t sym_row_of_unit(int64_t u, int64_t n_it, int64_t n_jt, int m) {
  int64_t lo = 0, hi = n_it - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (sym_rowstart(mid, n_jt, m) <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// Compensated FP32 running sum (Knuth's TwoSum: hi + lo carries the exact sum of
// the added floats up to the rounding of lo).  Used for the per-particle sums of
// the FP32 pair kernels across j-tiles, so the FP64 pipe stays out of the main
// loop; the total is read out once, as the double hi + lo.
struct CompSum {
  float hi, lo;
};
__device__ __forceinline__ void csum_add(CompSum &c, float x) {
  const float s = c.hi + x;
  const float bp = s - c.hi;
  c.lo += (c.hi - (s - bp)) + (x - bp);
  c.hi = s;
}
__device__ __forceinline__ void csum_add2(CompSum &c, float2 x) {
  csum_add(c, x.x);
  csum_add(c, x.y);
}
__device__ __forceinline__ double csum_total(const CompSum &c) { return (double)c.hi + (double)c.lo; }

// Reduce-scatter of V values per lane over the lanes spanned by the xor masks
// MASK0, MASK0/2, ..., MASK0*2/V: each round halves the values a lane keeps
// (lanes with the mask bit set keep the upper half) and adds the partner's copy
// of them.  Returns the sum over those lanes of value number
// sum_r (bit MASK_r of the lane ? V/2^(r+1) : 0).
template <int V, int MASK0, class T>
__device__ __forceinline__ T butterfly_sum(T (&v)[V], int lane) {
#pragma unroll
  for (int h = V / 2, mask = MASK0; h >= 1; h /= 2, mask /= 2) {
    const bool up = (lane & mask) != 0;
#pragma unroll
    for (int i = 0; i < h; i++) {
      const T send = up ? v[i] : v[i + h];
      const T keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
    }
  }
  return v[0];
}

// ============================================================ records ======

// Mirror record of particle i at FP64 position(s) (x, y) and, for adjoint
// records, lambda_p (vx, vy).  FP32 records interleave particles 2k and 2k+1
// so that one 128-bit load gives a packed operand for two j's.
template <int MODEL, bool MIXED, bool ADJ>
__device__ __forceinline__ void write_record(void *mirror, int64_t i, double x, double y, double vx, double vy) {
  if constexpr (MODEL == MD_RING) {
    const double r = reduce_2pi(x);
    if constexpr (MIXED) {
      float s, c, a, g;
      sincos_small((float)r, &s, &c);
      sincos_small(0.5f * (float)r, &a, &g);
      float *m = (float *)mirror + (i >> 1) * (ADJ ? 12 : 8) + (i & 1);
      m[0] = -s;
      m[2] = c;
      m[4] = -a;
      m[6] = g;
      if (ADJ) {
        m[8] = -(float)vx;
        m[10] = 0.f;
      }
    } else {
      double s, c, a, g;
      sincos(x, &s, &c);
      sincos(0.5 * r, &a, &g);
      double *m = (double *)mirror + i * (ADJ ? 6 : 4);
      m[0] = s;
      m[1] = c;
      m[2] = a;
      m[3] = g;
      if (ADJ) {
        m[4] = vx;
        m[5] = 0.0;
      }
    }
  } else {
    if constexpr (MIXED) {
      float *m = (float *)mirror + (i >> 1) * (ADJ ? 8 : 4) + (i & 1);
      m[0] = -(float)x;
      m[2] = -(float)y;
      if (ADJ) {
        m[4] = -(float)vx;
        m[6] = -(float)vy;
      }
    } else {
      double *m = (double *)mirror + i * (ADJ ? 4 : 2);
      m[0] = x;
      m[1] = y;
      if (ADJ) {
        m[2] = vx;
        m[3] = vy;
      }
    }
  }
}

// Padding record: contributes exactly zero to every sum.  Ring: all-zero
// (sin d = 0 with a positive denominator).  2D: so far away that |r|^2 overflows
// to +inf in FP32, whose reciprocal is 0 (FP64: 1e150, whose FP32 Newton seed
// is +inf -> 0, and the Newton steps keep 0).
template <int MODEL, bool MIXED, bool ADJ>
__device__ __forceinline__ void write_pad(void *mirror, int64_t i) {
  if constexpr (MODEL == MD_RING) {
    if constexpr (MIXED) {
      float *m = (float *)mirror + (i >> 1) * (ADJ ? 12 : 8) + (i & 1);
      m[0] = m[2] = m[4] = m[6] = 0.f;
      if (ADJ) m[8] = m[10] = 0.f;
    } else {
      double *m = (double *)mirror + i * (ADJ ? 6 : 4);
      for (int k = 0; k < (ADJ ? 6 : 4); k++) m[k] = 0.0;
    }
  } else {
    if constexpr (MIXED) {
      float *m = (float *)mirror + (i >> 1) * (ADJ ? 8 : 4) + (i & 1);
      m[0] = m[2] = -3.0e19f;
      if (ADJ) m[4] = m[6] = 0.f;
    } else {
      double *m = (double *)mirror + i * (ADJ ? 4 : 2);
      m[0] = m[1] = 1.0e150;
      if (ADJ) m[2] = m[3] = 0.0;
    }
  }
}

// ============================================================ policies =====
//
// A policy gives the skeleton: R, TJ, the record size JB, the number NACC of
// FP64 per-particle sums, whether the diagonal must be masked, the i-side state,
// its loader, the tile body and the epilogue.

// ---------------------------------------------------------- forward Ring FP32
template <int R_, int TJ_, int MODE>
struct RingMixed {
  static constexpr int R = R_, TJ = TJ_, NACC = 1, JB = RecordBytes<MD_RING, true, false>::value;
  static constexpr bool MASK = true;
  static constexpr int NR = R;  // rows finished per thread
  static constexpr int FMT = 0;  // mirror record format
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    float2 s[R], c[R], a[R], g[R], acc[R];
    CompSum cs[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = csum_total(st.cs[r][d]);
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int64_t i = i0 + row_of(r);
      const float *m = (const float *)mirror + (i >> 1) * 8 + (i & 1);
      st.s[r] = f2(-m[0]);
      st.c[r] = f2(m[2]);
      st.a[r] = f2(-m[4]);
      st.g[r] = f2(m[6]);
      st.acc[r] = f2(0.f);
      st.cs[r][0] = CompSum{0.f, 0.f};
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t i0, int64_t j0) {
    const float4 *sm = (const float4 *)smb;
    const float2 he = f2((float)a.epsd);
#pragma unroll 4
    for (int k = 0; k < TJ / 2; k++) {
      const float4 A = sm[2 * k], B = sm[2 * k + 1];
      const float2 nsj = make_float2(A.x, A.y), cj = make_float2(A.z, A.w);
      const float2 naj = make_float2(B.x, B.y), gj = make_float2(B.z, B.w);
#pragma unroll
      for (int r = 0; r < R; r++) {
        float2 S = __ffma2_rn(st.s[r], cj, __fmul2_rn(st.c[r], nsj));   // sin(theta_i - theta_j)
        float2 sh = __ffma2_rn(st.a[r], gj, __fmul2_rn(st.g[r], naj));  // sin((theta_i - theta_j)/2)
        float2 d = __ffma2_rn(sh, sh, he);                               // (1 - cos + eps)/2
        float2 y = make_float2(mufu_rsqrt(d.x), mufu_rsqrt(d.y));
        float2 y2 = __fmul2_rn(y, y);
        float2 qq = __fmul2_rn(S, y);
        if (DIAG) {
          const int64_t i = i0 + row_of(r), j = j0 + 2 * k;
          if (i == j) qq.x = 0.f;
          if (i == j + 1) qq.y = 0.f;
        }
        st.acc[r] = __ffma2_rn(qq, y2, st.acc[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      csum_add2(st.cs[r][0], st.acc[r]);
      st.acc[r] = f2(0.f);
    }
  }
};

// ------------------------------------------------------------ forward 2D FP32
template <int R_, int TJ_, int MODE, int MINB_ = 4>
struct GravMixed {
  static constexpr int THREADS = NT, MINB = MINB_;  // CTA size and CTAs per SM of the register budget
  using ColT = float;                           // column partials of the symmetric form
  static constexpr int R = R_, TJ = TJ_, NACC = 2, JB = RecordBytes<MD_GRAV2D, true, false>::value;
  static constexpr bool MASK = false;
  static constexpr int NR = R;  // rows finished per thread
  static constexpr int FMT = 0;  // mirror record format
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    float2 x[R], y[R], fx[R], fy[R];
    CompSum cs[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = csum_total(st.cs[r][d]);
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int64_t i = i0 + row_of(r);
      const float *m = (const float *)mirror + (i >> 1) * 4 + (i & 1);
      st.x[r] = f2(-m[0]);
      st.y[r] = f2(-m[2]);
      st.fx[r] = st.fy[r] = f2(0.f);
      for (int d = 0; d < NACC; d++) st.cs[r][d] = CompSum{0.f, 0.f};
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t, int64_t) {
    const float4 *sm = (const float4 *)smb;
    const float2 e2 = f2((float)a.epsd);
    auto body = [&](int k) {
      const float4 X = sm[k];
      const float2 nx = make_float2(X.x, X.y), ny = make_float2(X.z, X.w);
#pragma unroll
      for (int r = 0; r < R; r++) {
        float2 dx = __fadd2_rn(st.x[r], nx);
        float2 dy = __fadd2_rn(st.y[r], ny);
        float2 s = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, e2));
        float2 inv = make_float2(mufu_rcp(s.x), mufu_rcp(s.y));
        st.fx[r] = __ffma2_rn(dx, inv, st.fx[r]);
        st.fy[r] = __ffma2_rn(dy, inv, st.fy[r]);
      }
    };
#pragma unroll 4
    for (int k = 0; k < TJ / 2; k++) body(k);
#pragma unroll
    for (int r = 0; r < R; r++) {
      csum_add2(st.cs[r][0], st.fx[r]);
      csum_add2(st.cs[r][1], st.fy[r]);
      st.fx[r] = st.fy[r] = f2(0.f);
    }
  }
  // Off-diagonal block of the Newton's-third-law variant: the i-rows as in tile<>,
  // and for every j the sum over this warp's 32 R rows of the same terms
  // r_ij / s_ij, into colsm[(warp TJ + j) 2 + component] (the j-side term is
  // minus that sum).  Eight j's at a time: per lane 16 partial sums (4 j-pairs x
  // 2 components), reduced over the warp by a butterfly.
  __device__ static void tile_sym(State &st, const unsigned char *smb, const PairArgs &a, float *colsm) {
    const float4 *sm = (const float4 *)smb;
    const float2 e2 = f2((float)a.epsd);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll 4
    for (int k8 = 0; k8 < TJ / 8; k8++) {
      float v[16];
#pragma unroll
      for (int kk = 0; kk < 4; kk++) {
        const float4 X = sm[4 * k8 + kk];
        const float2 nx = make_float2(X.x, X.y), ny = make_float2(X.z, X.w);
        float2 cx = f2(0.f), cy = f2(0.f);
#pragma unroll
        for (int r = 0; r < R; r++) {
          float2 dx = __fadd2_rn(st.x[r], nx);
          float2 dy = __fadd2_rn(st.y[r], ny);
          float2 s = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, e2));
          float2 inv = make_float2(mufu_rcp(s.x), mufu_rcp(s.y));
          st.fx[r] = __ffma2_rn(dx, inv, st.fx[r]);
          st.fy[r] = __ffma2_rn(dy, inv, st.fy[r]);
          cx = __ffma2_rn(dx, inv, cx);
          cy = __ffma2_rn(dy, inv, cy);
        }
        v[4 * kk + 0] = cx.x;
        v[4 * kk + 1] = cx.y;
        v[4 * kk + 2] = cy.x;
        v[4 * kk + 3] = cy.y;
      }
      float sum = butterfly_sum<16, 16>(v, lane);  // over lane bits 4..1
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      if ((lane & 1) == 0) {
        const int vi = lane >> 1;  // value number: 4 kk + 2 component + (j parity)
        const int j = 8 * k8 + 2 * (vi >> 2) + (vi & 1);
        colsm[(w * TJ + j) * 2 + ((vi >> 1) & 1)] = sum;
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      csum_add2(st.cs[r][0], st.fx[r]);
      csum_add2(st.cs[r][1], st.fy[r]);
      st.fx[r] = st.fy[r] = f2(0.f);
    }
  }
  // Diagonal tile kd (columns kd TJ .. kd TJ + TJ - 1 of the tile's own particles)
  // of the Newton's-third-law variant.  Row group r holds rows r NT + tid, so the
  // G = TJ / NT groups from G kd on are the columns' own particles: groups below
  // lie above the diagonal and are evaluated as in tile_sym (row and column sums),
  // the G own groups one-sided as in tile<> (each ordered pair on its row; the self
  // term is exactly zero), and groups above are skipped (their pairs with these
  // columns are above-diagonal pairs of the tile kd' = r / G).  colsm gets every
  // column (zero for kd = 0, where no group lies above).
  template <int KD>
  __device__ static void tile_diag_k(State &st, const unsigned char *smb, const PairArgs &a, float *colsm) {
    constexpr int G = TJ / NT, RS = G * KD, RE = RS + G;
    static_assert(TJ % NT == 0 && RE <= R, "diagonal tile layout");
    const float4 *sm = (const float4 *)smb;
    const float2 e2 = f2((float)a.epsd);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if constexpr (RS == 0) {
      for (int idx = lane; idx < 2 * TJ; idx += 32) colsm[w * TJ * 2 + idx] = 0.f;
#pragma unroll 1
      for (int k = 0; k < TJ / 2; k++) {
        const float4 X = sm[k];
        const float2 nx = make_float2(X.x, X.y), ny = make_float2(X.z, X.w);
#pragma unroll
        for (int r = RS; r < RE; r++) {
          float2 dx = __fadd2_rn(st.x[r], nx);
          float2 dy = __fadd2_rn(st.y[r], ny);
          float2 s = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, e2));
          float2 inv = make_float2(mufu_rcp(s.x), mufu_rcp(s.y));
          st.fx[r] = __ffma2_rn(dx, inv, st.fx[r]);
          st.fy[r] = __ffma2_rn(dy, inv, st.fy[r]);
        }
      }
    } else {
#pragma unroll 1
      for (int k8 = 0; k8 < TJ / 8; k8++) {
        float v[16];
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
          const float4 X = sm[4 * k8 + kk];
          const float2 nx = make_float2(X.x, X.y), ny = make_float2(X.z, X.w);
          float2 cx = f2(0.f), cy = f2(0.f);
#pragma unroll
          for (int r = 0; r < RE; r++) {
            float2 dx = __fadd2_rn(st.x[r], nx);
            float2 dy = __fadd2_rn(st.y[r], ny);
            float2 s = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, e2));
            float2 inv = make_float2(mufu_rcp(s.x), mufu_rcp(s.y));
            st.fx[r] = __ffma2_rn(dx, inv, st.fx[r]);
            st.fy[r] = __ffma2_rn(dy, inv, st.fy[r]);
            if (r < RS) {
              cx = __ffma2_rn(dx, inv, cx);
              cy = __ffma2_rn(dy, inv, cy);
            }
          }
          v[4 * kk + 0] = cx.x;
          v[4 * kk + 1] = cx.y;
          v[4 * kk + 2] = cy.x;
          v[4 * kk + 3] = cy.y;
        }
        float sum = butterfly_sum<16, 16>(v, lane);
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        if ((lane & 1) == 0) {
          const int vi = lane >> 1;
          const int j = 8 * k8 + 2 * (vi >> 2) + (vi & 1);
          colsm[(w * TJ + j) * 2 + ((vi >> 1) & 1)] = sum;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RE; r++) {
      csum_add2(st.cs[r][0], st.fx[r]);
      csum_add2(st.cs[r][1], st.fy[r]);
      st.fx[r] = st.fy[r] = f2(0.f);
    }
  }
  __device__ static void tile_diag(State &st, const unsigned char *smb, const PairArgs &a, float *colsm, int kd) {
    static_assert(NT * R == 4 * TJ, "four column blocks per diagonal tile");
    switch (kd) {
      case 0: tile_diag_k<0>(st, smb, a, colsm); break;
      case 1: tile_diag_k<1>(st, smb, a, colsm); break;
      case 2: tile_diag_k<2>(st, smb, a, colsm); break;
      default: tile_diag_k<3>(st, smb, a, colsm); break;
    }
  }
};

// ------------------------------------------------------------ forward Ring FP64
template <int R_, int TJ_, int MODE>
struct RingF64 {
  static constexpr int THREADS = NT, MINB = 4;
  using ColT = double;
  static constexpr int R = R_, TJ = TJ_, NACC = 1, JB = RecordBytes<MD_RING, false, false>::value;
  static constexpr bool MASK = true;
  static constexpr int NR = R;  // rows finished per thread
  static constexpr int FMT = 0;  // mirror record format
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    double s[R], c[R], a[R], g[R];
    double accd[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = st.accd[r][d];
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const double *m = (const double *)mirror + (i0 + row_of(r)) * 4;
      st.s[r] = m[0];
      st.c[r] = m[1];
      st.a[r] = m[2];
      st.g[r] = m[3];
      st.accd[r][0] = 0.0;
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t i0, int64_t j0) {
    const double2 *sm = (const double2 *)smb;
#pragma unroll 2
    for (int k = 0; k < TJ; k++) {
      const double2 sc = sm[2 * k], ag = sm[2 * k + 1];
#pragma unroll
      for (int r = 0; r < R; r++) {
        double S = fma(st.s[r], sc.y, -(st.c[r] * sc.x));
        double sh = fma(st.a[r], ag.y, -(st.g[r] * ag.x));
        double y = rsqrt_nr(fma(sh, sh, a.epsd));
        double qq = S * y;
        if (DIAG && i0 + row_of(r) == j0 + k) qq = 0.0;
        st.accd[r][0] = fma(qq, y * y, st.accd[r][0]);
      }
    }
  }
  // Off-diagonal block of the Newton's-third-law variant (FP64): the i-rows as in
  // tile<>, and per j the sum over this warp's 32 R rows of the same terms, into
  // colsm[warp TJ + j]; sixteen j's at a time reduced over the warp by a butterfly.
  __device__ static void tile_sym(State &st, const unsigned char *smb, const PairArgs &a, double *colsm) {
    const double2 *sm = (const double2 *)smb;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll 1
    for (int k16 = 0; k16 < TJ / 16; k16++) {
      double v[16];
#pragma unroll
      for (int kk = 0; kk < 16; kk++) {
        const int k = 16 * k16 + kk;
        const double2 sc = sm[2 * k], ag = sm[2 * k + 1];
        double col = 0.0;
#pragma unroll
        for (int r = 0; r < R; r++) {
          double S = fma(st.s[r], sc.y, -(st.c[r] * sc.x));
          double sh = fma(st.a[r], ag.y, -(st.g[r] * ag.x));
          double y = rsqrt_nr(fma(sh, sh, a.epsd));
          double t = S * y * (y * y);
          st.accd[r][0] += t;
          col += t;
        }
        v[kk] = col;
      }
      double sum = butterfly_sum<16, 16>(v, lane);  // over lane bits 4..1
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      if ((lane & 1) == 0) colsm[w * TJ + 16 * k16 + (lane >> 1)] = sum;
    }
  }
};

// ------------------------------------------------------------ forward 2D FP64
template <int R_, int TJ_, int MODE>
struct GravF64 {
  static constexpr int THREADS = NT, MINB = 4;
  using ColT = double;
  static constexpr int R = R_, TJ = TJ_, NACC = 2, JB = RecordBytes<MD_GRAV2D, false, false>::value;
  static constexpr bool MASK = false;
  static constexpr int NR = R;  // rows finished per thread
  static constexpr int FMT = 0;  // mirror record format
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    double x[R], y[R];
    double accd[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = st.accd[r][d];
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const double *m = (const double *)mirror + (i0 + row_of(r)) * 2;
      st.x[r] = m[0];
      st.y[r] = m[1];
      st.accd[r][0] = st.accd[r][1] = 0.0;
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t, int64_t) {
    const double2 *sm = (const double2 *)smb;
#pragma unroll 2
    for (int k = 0; k < TJ; k++) {
      const double2 xy = sm[k];
#pragma unroll
      for (int r = 0; r < R; r++) {
        double dx = st.x[r] - xy.x, dy = st.y[r] - xy.y;
        double inv = rcp_nr(fma(dx, dx, fma(dy, dy, a.epsd)));
        st.accd[r][0] = fma(dx, inv, st.accd[r][0]);
        st.accd[r][1] = fma(dy, inv, st.accd[r][1]);
      }
    }
  }
  // Off-diagonal block of the Newton's-third-law variant (FP64): per j the sums
  // over this warp's rows of the x and y terms into colsm[(warp TJ + j) 2 + d];
  // eight j's (16 values) at a time reduced over the warp by a butterfly.
  __device__ static void tile_sym(State &st, const unsigned char *smb, const PairArgs &a, double *colsm) {
    const double2 *sm = (const double2 *)smb;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll 1
    for (int k8 = 0; k8 < TJ / 8; k8++) {
      double v[16];
#pragma unroll
      for (int kk = 0; kk < 8; kk++) {
        const double2 xy = sm[8 * k8 + kk];
        double cx = 0.0, cy = 0.0;
#pragma unroll
        for (int r = 0; r < R; r++) {
          double dx = st.x[r] - xy.x, dy = st.y[r] - xy.y;
          double inv = rcp_nr(fma(dx, dx, fma(dy, dy, a.epsd)));
          double tx = dx * inv, ty = dy * inv;
          st.accd[r][0] += tx;
          st.accd[r][1] += ty;
          cx += tx;
          cy += ty;
        }
        v[2 * kk] = cx;
        v[2 * kk + 1] = cy;
      }
      double sum = butterfly_sum<16, 16>(v, lane);
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      if ((lane & 1) == 0) {
        const int vi = lane >> 1;  // 2 kk + component
        colsm[(w * TJ + 8 * k8 + (vi >> 1)) * 2 + (vi & 1)] = sum;
      }
    }
  }
};

// ------------------------------------------------------------ forward 3D FP32
// f_i = -(1/N) sum_j r_ij s^(-3/2), s = |r_ij|^2 + eps; per pair 11 FP32 operations
// and one rsqrt.  Accumulators 0, 1, 2 = x, y, z sums of r s^(-3/2).
template <int R_, int TJ_, int MODE, int MINB_ = 4>
struct Grav3DMixed {
  static constexpr int THREADS = NT, MINB = MINB_;  // CTA size and CTAs per SM of the register budget
  using ColT = float;
  static constexpr int R = R_, TJ = TJ_, NACC = 3, JB = RecordBytes<MD_GRAV3D, true, false>::value;
  static constexpr bool MASK = false;
  static constexpr int NR = R;
  static constexpr int FMT = 0;
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    float2 x[R], y[R], z[R], fx[R], fy[R], fz[R];
    CompSum cs[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = csum_total(st.cs[r][d]);
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int64_t i = i0 + row_of(r);
      const float *m = (const float *)mirror + (i >> 1) * 8 + (i & 1);
      st.x[r] = f2(-m[0]);
      st.y[r] = f2(-m[2]);
      st.z[r] = f2(-m[4]);
      st.fx[r] = st.fy[r] = st.fz[r] = f2(0.f);
#pragma unroll
      for (int d = 0; d < NACC; d++) st.cs[r][d] = CompSum{0.f, 0.f};
    }
  }
  __device__ static void flush(State &st) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      csum_add2(st.cs[r][0], st.fx[r]);
      csum_add2(st.cs[r][1], st.fy[r]);
      csum_add2(st.cs[r][2], st.fz[r]);
      st.fx[r] = st.fy[r] = st.fz[r] = f2(0.f);
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t, int64_t) {
    const float4 *sm = (const float4 *)smb;
    const float2 e2 = f2((float)a.epsd);
#pragma unroll 4
    for (int k = 0; k < TJ / 2; k++) {
      const float4 A = sm[2 * k], B = sm[2 * k + 1];
      const float2 nx = make_float2(A.x, A.y), ny = make_float2(A.z, A.w), nz = make_float2(B.x, B.y);
#pragma unroll
      for (int r = 0; r < R; r++) {
        const float2 dx = __fadd2_rn(st.x[r], nx), dy = __fadd2_rn(st.y[r], ny), dz = __fadd2_rn(st.z[r], nz);
        const float2 s = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
        const float2 y = make_float2(mufu_rsqrt(s.x), mufu_rsqrt(s.y));
        const float2 w = __fmul2_rn(__fmul2_rn(y, y), y);
        st.fx[r] = __ffma2_rn(dx, w, st.fx[r]);
        st.fy[r] = __ffma2_rn(dy, w, st.fy[r]);
        st.fz[r] = __ffma2_rn(dz, w, st.fz[r]);
      }
    }
    flush(st);
  }
  // Off-diagonal block of the Newton's-third-law variant: rows as in tile<>, and
  // per j the sums over this warp's 32 R rows of the x, y, z terms into
  // colsm[(warp TJ + j) 3 + d]; four j-pairs at a time, the (x, y) sums reduced by
  // one butterfly of 16 values and the z sums by one of 8.
  __device__ static void tile_sym(State &st, const unsigned char *smb, const PairArgs &a, float *colsm) {
    const float4 *sm = (const float4 *)smb;
    const float2 e2 = f2((float)a.epsd);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll 4
    for (int k8 = 0; k8 < TJ / 8; k8++) {
      float vxy[16], vz[8];
#pragma unroll
      for (int kk = 0; kk < 4; kk++) {
        const int k = 4 * k8 + kk;
        const float4 A = sm[2 * k], B = sm[2 * k + 1];
        const float2 nx = make_float2(A.x, A.y), ny = make_float2(A.z, A.w), nz = make_float2(B.x, B.y);
        float2 cx = f2(0.f), cy = f2(0.f), cz = f2(0.f);
#pragma unroll
        for (int r = 0; r < R; r++) {
          const float2 dx = __fadd2_rn(st.x[r], nx), dy = __fadd2_rn(st.y[r], ny), dz = __fadd2_rn(st.z[r], nz);
          const float2 s = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
          const float2 y = make_float2(mufu_rsqrt(s.x), mufu_rsqrt(s.y));
          const float2 wt = __fmul2_rn(__fmul2_rn(y, y), y);
          st.fx[r] = __ffma2_rn(dx, wt, st.fx[r]);
          st.fy[r] = __ffma2_rn(dy, wt, st.fy[r]);
          st.fz[r] = __ffma2_rn(dz, wt, st.fz[r]);
          cx = __ffma2_rn(dx, wt, cx);
          cy = __ffma2_rn(dy, wt, cy);
          cz = __ffma2_rn(dz, wt, cz);
        }
        vxy[4 * kk + 0] = cx.x;
        vxy[4 * kk + 1] = cx.y;
        vxy[4 * kk + 2] = cy.x;
        vxy[4 * kk + 3] = cy.y;
        vz[2 * kk + 0] = cz.x;
        vz[2 * kk + 1] = cz.y;
      }
      float sxy = butterfly_sum<16, 16>(vxy, lane);  // value lane >> 1 = 4 kk + 2 d + (j parity)
      sxy += __shfl_xor_sync(0xffffffffu, sxy, 1);
      float sz = butterfly_sum<8, 16>(vz, lane);  // value lane >> 2 = 2 kk + (j parity)
      sz += __shfl_xor_sync(0xffffffffu, sz, 2);
      sz += __shfl_xor_sync(0xffffffffu, sz, 1);
      if ((lane & 1) == 0) {
        const int vi = lane >> 1;
        const int j = 8 * k8 + 2 * (vi >> 2) + (vi & 1);
        colsm[(w * TJ + j) * 3 + ((vi >> 1) & 1)] = sxy;
      }
      if ((lane & 3) == 0) {
        const int vi = lane >> 2;
        colsm[(w * TJ + 8 * k8 + vi) * 3 + 2] = sz;
      }
    }
    flush(st);
  }
};

// ------------------------------------------------------------ forward 3D FP64
template <int R_, int TJ_, int MODE>
struct Grav3DF64 {
  static constexpr int THREADS = NT, MINB = 4;
  using ColT = double;
  static constexpr int R = R_, TJ = TJ_, NACC = 3, JB = RecordBytes<MD_GRAV3D, false, false>::value;
  static constexpr bool MASK = false;
  static constexpr int NR = R;
  static constexpr int FMT = 0;
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    double x[R], y[R], z[R];
    double accd[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = st.accd[r][d];
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const double *m = (const double *)mirror + (i0 + row_of(r)) * 4;
      st.x[r] = m[0];
      st.y[r] = m[1];
      st.z[r] = m[2];
      st.accd[r][0] = st.accd[r][1] = st.accd[r][2] = 0.0;
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t, int64_t) {
    const double4_16a *sm = (const double4_16a *)smb;
#pragma unroll 2
    for (int k = 0; k < TJ; k++) {
      const double4_16a o = sm[k];
#pragma unroll
      for (int r = 0; r < R; r++) {
        const double dx = st.x[r] - o.x, dy = st.y[r] - o.y, dz = st.z[r] - o.z;
        const double y = rsqrt_nr(fma(dx, dx, fma(dy, dy, fma(dz, dz, a.epsd))));
        const double w = y * y * y;
        st.accd[r][0] = fma(dx, w, st.accd[r][0]);
        st.accd[r][1] = fma(dy, w, st.accd[r][1]);
        st.accd[r][2] = fma(dz, w, st.accd[r][2]);
      }
    }
  }
  // Newton's-third-law variant: per j the sums over this warp's rows of the x, y,
  // z terms into colsm[(warp TJ + j) 3 + d]; eight j's at a time, (x, y) by a
  // butterfly of 16 values and z by one of 8.
  __device__ static void tile_sym(State &st, const unsigned char *smb, const PairArgs &a, double *colsm) {
    const double4_16a *sm = (const double4_16a *)smb;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll 1
    for (int k8 = 0; k8 < TJ / 8; k8++) {
      double vxy[16], vz[8];
#pragma unroll
      for (int kk = 0; kk < 8; kk++) {
        const double4_16a o = sm[8 * k8 + kk];
        double cx = 0.0, cy = 0.0, cz = 0.0;
#pragma unroll
        for (int r = 0; r < R; r++) {
          const double dx = st.x[r] - o.x, dy = st.y[r] - o.y, dz = st.z[r] - o.z;
          const double y = rsqrt_nr(fma(dx, dx, fma(dy, dy, fma(dz, dz, a.epsd))));
          const double wt = y * y * y;
          const double tx = dx * wt, ty = dy * wt, tz = dz * wt;
          st.accd[r][0] += tx;
          st.accd[r][1] += ty;
          st.accd[r][2] += tz;
          cx += tx;
          cy += ty;
          cz += tz;
        }
        vxy[2 * kk] = cx;
        vxy[2 * kk + 1] = cy;
        vz[kk] = cz;
      }
      double sxy = butterfly_sum<16, 16>(vxy, lane);  // value lane >> 1 = 2 kk + d
      sxy += __shfl_xor_sync(0xffffffffu, sxy, 1);
      double sz = butterfly_sum<8, 16>(vz, lane);  // value lane >> 2 = kk
      sz += __shfl_xor_sync(0xffffffffu, sz, 2);
      sz += __shfl_xor_sync(0xffffffffu, sz, 1);
      if ((lane & 1) == 0) {
        const int vi = lane >> 1;
        colsm[(w * TJ + 8 * k8 + (vi >> 1)) * 3 + (vi & 1)] = sxy;
      }
      if ((lane & 3) == 0) colsm[(w * TJ + 8 * k8 + (lane >> 2)) * 3 + 2] = sz;
    }
  }
};

// ------------------------------------------------------------ forward 1D sheets FP32
// eps = 0: the term of a pair is sign(x_i - x_j), decided on the FP32 positions
// (the FP32 difference of two floats is zero only for equal floats, so its sign is
// their order), summed exactly (integers below 2^24 per tile); eps > 0:
// d / sqrt(d^2 + eps) with one rsqrt.  One accumulator.
template <int R_, int TJ_, int MODE, int MINB_ = 4>
struct SheetMixed {
  static constexpr int THREADS = NT, MINB = MINB_;  // CTA size and CTAs per SM of the register budget
  using ColT = float;
  static constexpr int R = R_, TJ = TJ_, NACC = 1, JB = RecordBytes<MD_SHEET1D, true, false>::value;
  static constexpr bool MASK = false;  // the self term is zero in both forms
  static constexpr int NR = R;
  static constexpr int FMT = 0;
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    float2 x[R], acc[R];
    CompSum cs[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) { out[0] = csum_total(st.cs[r][0]); }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      st.x[r] = f2(-((const float *)mirror)[i0 + row_of(r)]);
      st.acc[r] = f2(0.f);
      st.cs[r][0] = CompSum{0.f, 0.f};
    }
  }
  __device__ static float sgnf(float d) { return (float)(d > 0.f) - (float)(d < 0.f); }
  __device__ static float2 term(float2 xi, float2 nx, float2 e2, bool smooth) {
    const float2 d = __fadd2_rn(xi, nx);
    if (!smooth) return make_float2(sgnf(d.x), sgnf(d.y));
    const float2 s = __ffma2_rn(d, d, e2);
    return __fmul2_rn(d, make_float2(mufu_rsqrt(s.x), mufu_rsqrt(s.y)));
  }
  __device__ static void flush(State &st) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      csum_add2(st.cs[r][0], st.acc[r]);
      st.acc[r] = f2(0.f);
    }
  }
  template <bool SMOOTH>
  __device__ static void body(State &st, const float2 *sm, float2 e2) {
#pragma unroll 4
    for (int k = 0; k < TJ / 2; k++) {
      const float2 nx = sm[k];
#pragma unroll
      for (int r = 0; r < R; r++) st.acc[r] = __fadd2_rn(st.acc[r], term(st.x[r], nx, e2, SMOOTH));
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t, int64_t) {
    const float2 *sm = (const float2 *)smb;
    const float2 e2 = f2((float)a.epsd);
    if (a.epsd > 0.0) body<true>(st, sm, e2);
    else body<false>(st, sm, e2);
    flush(st);
  }
  template <bool SMOOTH>
  __device__ static void body_sym(State &st, const float2 *sm, float2 e2, float *colsm) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll 1
    for (int k8 = 0; k8 < TJ / 16; k8++) {
      float v[16];
#pragma unroll
      for (int kk = 0; kk < 8; kk++) {
        const float2 nx = sm[8 * k8 + kk];
        float2 col = f2(0.f);
#pragma unroll
        for (int r = 0; r < R; r++) {
          const float2 t = term(st.x[r], nx, e2, SMOOTH);
          st.acc[r] = __fadd2_rn(st.acc[r], t);
          col = __fadd2_rn(col, t);
        }
        v[2 * kk] = col.x;
        v[2 * kk + 1] = col.y;
      }
      float sum = butterfly_sum<16, 16>(v, lane);  // value lane >> 1 = 2 kk + (j parity)
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      if ((lane & 1) == 0) colsm[w * TJ + 16 * k8 + (lane >> 1)] = sum;
    }
  }
  // Newton's-third-law variant: the i-rows as in tile<>, and per j the sum over this
  // warp's rows of the same terms into colsm[warp TJ + j]; sixteen j's at a time.
  __device__ static void tile_sym(State &st, const unsigned char *smb, const PairArgs &a, float *colsm) {
    const float2 *sm = (const float2 *)smb;
    const float2 e2 = f2((float)a.epsd);
    if (a.epsd > 0.0) body_sym<true>(st, sm, e2, colsm);
    else body_sym<false>(st, sm, e2, colsm);
    flush(st);
  }
};

// ------------------------------------------------------------ forward 1D sheets FP64
// Records are integer keys of x (sheet_key).  eps = 0: per pair the two comparisons
// k_i > k_j and k_i < k_j on the ALU pipe, counted in integers per tile; eps > 0:
// x from the key, d / sqrt(d^2 + eps) in FP64.
template <int R_, int TJ_, int MODE>
struct SheetF64 {
  static constexpr int THREADS = NT, MINB = 4;
  using ColT = double;
  static constexpr int R = R_, TJ = TJ_, NACC = 1, JB = RecordBytes<MD_SHEET1D, false, false>::value;
  static constexpr bool MASK = false;
  static constexpr int NR = R;
  static constexpr int FMT = 0;
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    long long k[R];
    double accd[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) { out[0] = st.accd[r][0]; }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      st.k[r] = ((const long long *)mirror)[i0 + row_of(r)];
      st.accd[r][0] = 0.0;
    }
  }
  __device__ static int cmp(long long ki, long long kj) { return (int)(ki > kj) - (int)(ki < kj); }
  __device__ static double smooth_term(double xi, long long kj, double eps) {
    const double d = xi - sheet_unkey(kj);
    return d * rsqrt_nr(fma(d, d, eps));
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t, int64_t) {
    const long long *sm = (const long long *)smb;
    if (a.epsd > 0.0) {
      double x[R];
#pragma unroll
      for (int r = 0; r < R; r++) x[r] = sheet_unkey(st.k[r]);
#pragma unroll 2
      for (int k = 0; k < TJ; k++) {
        const long long kj = sm[k];
#pragma unroll
        for (int r = 0; r < R; r++) st.accd[r][0] += smooth_term(x[r], kj, a.epsd);
      }
    } else {
      int acc[R];
#pragma unroll
      for (int r = 0; r < R; r++) acc[r] = 0;
#pragma unroll 4
      for (int k = 0; k < TJ; k++) {
        const long long kj = sm[k];
#pragma unroll
        for (int r = 0; r < R; r++) acc[r] += cmp(st.k[r], kj);
      }
#pragma unroll
      for (int r = 0; r < R; r++) st.accd[r][0] += (double)acc[r];
    }
  }
  __device__ static void tile_sym(State &st, const unsigned char *smb, const PairArgs &a, double *colsm) {
    const long long *sm = (const long long *)smb;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (a.epsd > 0.0) {
      double x[R];
#pragma unroll
      for (int r = 0; r < R; r++) x[r] = sheet_unkey(st.k[r]);
#pragma unroll 1
      for (int k16 = 0; k16 < TJ / 16; k16++) {
        double v[16];
#pragma unroll
        for (int kk = 0; kk < 16; kk++) {
          const long long kj = sm[16 * k16 + kk];
          double col = 0.0;
#pragma unroll
          for (int r = 0; r < R; r++) {
            const double t = smooth_term(x[r], kj, a.epsd);
            st.accd[r][0] += t;
            col += t;
          }
          v[kk] = col;
        }
        double sum = butterfly_sum<16, 16>(v, lane);
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        if ((lane & 1) == 0) colsm[w * TJ + 16 * k16 + (lane >> 1)] = sum;
      }
    } else {
      int acc[R];
#pragma unroll
      for (int r = 0; r < R; r++) acc[r] = 0;
#pragma unroll 1
      for (int k16 = 0; k16 < TJ / 16; k16++) {
        int v[16];
#pragma unroll
        for (int kk = 0; kk < 16; kk++) {
          const long long kj = sm[16 * k16 + kk];
          int col = 0;
#pragma unroll
          for (int r = 0; r < R; r++) {
            const int t = cmp(st.k[r], kj);
            acc[r] += t;
            col += t;
          }
          v[kk] = col;
        }
        int sum = butterfly_sum<16, 16>(v, lane);
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        if ((lane & 1) == 0) colsm[w * TJ + 16 * k16 + (lane >> 1)] = (double)sum;
      }
#pragma unroll
      for (int r = 0; r < R; r++) st.accd[r][0] += (double)acc[r];
    }
  }
};

// ------------------------------------------------------------ adjoint Ring FP32
// accumulators: 0 = sum S dd^-3/2 (force), 1 = sum G w (J v), 2 = sum S dd^-5/2 (d/deps)
template <int R_, int TJ_, int MODE, int MINB_ = 1>
struct RingMixedAdj {
  static constexpr int STREAMK_MINB = MINB_;  // register budget of the one-sided kernel
  static constexpr int R = R_, TJ = TJ_, NACC = 3, JB = RecordBytes<MD_RING, true, true>::value;
  static constexpr bool MASK = true;
  static constexpr int NR = R;  // rows finished per thread
  static constexpr int FMT = 0;  // mirror record format
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    float2 s[R], c[R], a[R], g[R], ns[R], v[R], af[R], aj[R], ae[R];
    CompSum cs[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = csum_total(st.cs[r][d]);
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int64_t i = i0 + row_of(r);
      const float *m = (const float *)mirror + (i >> 1) * 12 + (i & 1);
      st.s[r] = f2(-m[0]);
      st.ns[r] = f2(m[0]);
      st.c[r] = f2(m[2]);
      st.a[r] = f2(-m[4]);
      st.g[r] = f2(m[6]);
      st.v[r] = f2(-m[8]);
      st.af[r] = st.aj[r] = st.ae[r] = f2(0.f);
      for (int d = 0; d < NACC; d++) st.cs[r][d] = CompSum{0.f, 0.f};
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t i0, int64_t j0) {
    const float4 *sm = (const float4 *)smb;
    const float2 he = f2((float)a.epsd), m34 = f2(-0.75f);
#pragma unroll 4
    for (int k = 0; k < TJ / 2; k++) {
      const float4 A = sm[3 * k], B = sm[3 * k + 1], L = sm[3 * k + 2];
      const float2 nsj = make_float2(A.x, A.y), cj = make_float2(A.z, A.w);
      const float2 naj = make_float2(B.x, B.y), gj = make_float2(B.z, B.w);
      const float2 nvj = make_float2(L.x, L.y);
#pragma unroll
      for (int r = 0; r < R; r++) {
        float2 S = __ffma2_rn(st.s[r], cj, __fmul2_rn(st.c[r], nsj));
        float2 C = __ffma2_rn(st.c[r], cj, __fmul2_rn(st.ns[r], nsj));  // cos(theta_i - theta_j)
        float2 sh = __ffma2_rn(st.a[r], gj, __fmul2_rn(st.g[r], naj));
        float2 d = __ffma2_rn(sh, sh, he);
        float2 y = make_float2(mufu_rsqrt(d.x), mufu_rsqrt(d.y));
        float2 y2 = __fmul2_rn(y, y);
        float2 r3 = __fmul2_rn(y2, y);
        float2 r5 = __fmul2_rn(r3, y2);
        if (DIAG) {
          const int64_t i = i0 + row_of(r), j = j0 + 2 * k;
          if (i == j) S.x = 0.f;
          if (i == j + 1) S.y = 0.f;
        }
        st.af[r] = __ffma2_rn(S, r3, st.af[r]);
        st.ae[r] = __ffma2_rn(S, r5, st.ae[r]);
        float2 G = __ffma2_rn(__fmul2_rn(__fmul2_rn(S, S), m34), r5, __fmul2_rn(C, r3));
        st.aj[r] = __ffma2_rn(G, __fadd2_rn(st.v[r], nvj), st.aj[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      csum_add2(st.cs[r][0], st.af[r]);
      csum_add2(st.cs[r][1], st.aj[r]);
      csum_add2(st.cs[r][2], st.ae[r]);
      st.af[r] = st.aj[r] = st.ae[r] = f2(0.f);
    }
  }
};

// ------------------------------------------------------------ adjoint 2D FP32
// accumulators: 0,1 = force (x,y); 2,3 = J v (x,y) without the -2/N factor; 4,5 = d/deps
template <int R_, int TJ_, int MODE, int MINB_ = 1>
struct GravMixedAdj {
  static constexpr int STREAMK_MINB = MINB_;  // register budget of the one-sided kernel
  static constexpr int R = R_, TJ = TJ_, NACC = 6, JB = RecordBytes<MD_GRAV2D, true, true>::value;
  static constexpr bool MASK = false;
  static constexpr int NR = R;  // rows finished per thread
  static constexpr int FMT = 0;  // mirror record format
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    float2 x[R], y[R], vx[R], vy[R], fx[R], fy[R], jx[R], jy[R], ex[R], ey[R];
    CompSum cs[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = csum_total(st.cs[r][d]);
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int64_t i = i0 + row_of(r);
      const float *m = (const float *)mirror + (i >> 1) * 8 + (i & 1);
      st.x[r] = f2(-m[0]);
      st.y[r] = f2(-m[2]);
      st.vx[r] = f2(-m[4]);
      st.vy[r] = f2(-m[6]);
      st.fx[r] = st.fy[r] = st.jx[r] = st.jy[r] = st.ex[r] = st.ey[r] = f2(0.f);
#pragma unroll
      for (int d = 0; d < NACC; d++) st.cs[r][d] = CompSum{0.f, 0.f};
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t, int64_t) {
    const float4 *sm = (const float4 *)smb;
    const float2 e2 = f2((float)a.epsd), m2 = f2(-2.f);
#pragma unroll 4
    for (int k = 0; k < TJ / 2; k++) {
      const float4 X = sm[2 * k], V = sm[2 * k + 1];
      const float2 nx = make_float2(X.x, X.y), ny = make_float2(X.z, X.w);
      const float2 nvx = make_float2(V.x, V.y), nvy = make_float2(V.z, V.w);
#pragma unroll
      for (int r = 0; r < R; r++) {
        float2 dx = __fadd2_rn(st.x[r], nx);
        float2 dy = __fadd2_rn(st.y[r], ny);
        float2 s = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, e2));
        float2 inv = make_float2(mufu_rcp(s.x), mufu_rcp(s.y));
        float2 inv2 = __fmul2_rn(inv, inv);
        float2 wx = __fadd2_rn(st.vx[r], nvx), wy = __fadd2_rn(st.vy[r], nvy);
        float2 m2u = __fmul2_rn(__fmul2_rn(__ffma2_rn(dy, wy, __fmul2_rn(dx, wx)), inv2), m2);
        st.fx[r] = __ffma2_rn(dx, inv, st.fx[r]);
        st.fy[r] = __ffma2_rn(dy, inv, st.fy[r]);
        st.jx[r] = __ffma2_rn(m2u, dx, __ffma2_rn(wx, inv, st.jx[r]));
        st.jy[r] = __ffma2_rn(m2u, dy, __ffma2_rn(wy, inv, st.jy[r]));
        st.ex[r] = __ffma2_rn(dx, inv2, st.ex[r]);
        st.ey[r] = __ffma2_rn(dy, inv2, st.ey[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      csum_add2(st.cs[r][0], st.fx[r]);
      csum_add2(st.cs[r][1], st.fy[r]);
      csum_add2(st.cs[r][2], st.jx[r]);
      csum_add2(st.cs[r][3], st.jy[r]);
      csum_add2(st.cs[r][4], st.ex[r]);
      csum_add2(st.cs[r][5], st.ey[r]);
      st.fx[r] = st.fy[r] = st.jx[r] = st.jy[r] = st.ex[r] = st.ey[r] = f2(0.f);
    }
  }
};

// ------------------------------------------------------------ adjoint 3D FP32
// accumulators: 0-2 = force sums of r s^(-3/2); 3-5 = J w sums of w s^(-3/2) - 3 r (r.w) s^(-5/2)
// (w = lambda_i - lambda_j); 6-8 = d/deps sums of r s^(-5/2)
template <int R_, int TJ_, int MODE, int MINB_ = 1>
struct Grav3DMixedAdj {
  static constexpr int STREAMK_MINB = MINB_;  // register budget of the one-sided kernel
  static constexpr int R = R_, TJ = TJ_, NACC = 9, JB = RecordBytes<MD_GRAV3D, true, true>::value;
  static constexpr bool MASK = false;
  static constexpr int NR = R;
  static constexpr int FMT = 0;
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    float2 x[R], y[R], z[R], vx[R], vy[R], vz[R], acc[R][NACC];
    CompSum cs[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = csum_total(st.cs[r][d]);
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int64_t i = i0 + row_of(r);
      const float *m = (const float *)mirror + (i >> 1) * 12 + (i & 1);
      st.x[r] = f2(-m[0]);
      st.y[r] = f2(-m[2]);
      st.z[r] = f2(-m[4]);
      st.vx[r] = f2(-m[6]);
      st.vy[r] = f2(-m[8]);
      st.vz[r] = f2(-m[10]);
#pragma unroll
      for (int d = 0; d < NACC; d++) {
        st.acc[r][d] = f2(0.f);
        st.cs[r][d] = CompSum{0.f, 0.f};
      }
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t, int64_t) {
    const float4 *sm = (const float4 *)smb;
    const float2 e2 = f2((float)a.epsd), m3 = f2(-3.f);
#pragma unroll 2
    for (int k = 0; k < TJ / 2; k++) {
      const float4 A = sm[3 * k], B = sm[3 * k + 1], C = sm[3 * k + 2];
      const float2 nx = make_float2(A.x, A.y), ny = make_float2(A.z, A.w), nz = make_float2(B.x, B.y);
      const float2 nvx = make_float2(B.z, B.w), nvy = make_float2(C.x, C.y), nvz = make_float2(C.z, C.w);
#pragma unroll
      for (int r = 0; r < R; r++) {
        const float2 dx = __fadd2_rn(st.x[r], nx), dy = __fadd2_rn(st.y[r], ny), dz = __fadd2_rn(st.z[r], nz);
        const float2 s = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
        const float2 y = make_float2(mufu_rsqrt(s.x), mufu_rsqrt(s.y));
        const float2 y2 = __fmul2_rn(y, y);
        const float2 w3 = __fmul2_rn(y2, y), w5 = __fmul2_rn(w3, y2);
        const float2 wx = __fadd2_rn(st.vx[r], nvx), wy = __fadd2_rn(st.vy[r], nvy), wz = __fadd2_rn(st.vz[r], nvz);
        const float2 rw = __ffma2_rn(dx, wx, __ffma2_rn(dy, wy, __fmul2_rn(dz, wz)));
        const float2 t = __fmul2_rn(rw, __fmul2_rn(w5, m3));
        float2 *ac = st.acc[r];
        ac[0] = __ffma2_rn(dx, w3, ac[0]);
        ac[1] = __ffma2_rn(dy, w3, ac[1]);
        ac[2] = __ffma2_rn(dz, w3, ac[2]);
        ac[3] = __ffma2_rn(t, dx, __ffma2_rn(wx, w3, ac[3]));
        ac[4] = __ffma2_rn(t, dy, __ffma2_rn(wy, w3, ac[4]));
        ac[5] = __ffma2_rn(t, dz, __ffma2_rn(wz, w3, ac[5]));
        ac[6] = __ffma2_rn(dx, w5, ac[6]);
        ac[7] = __ffma2_rn(dy, w5, ac[7]);
        ac[8] = __ffma2_rn(dz, w5, ac[8]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
      for (int d = 0; d < NACC; d++) {
        csum_add2(st.cs[r][d], st.acc[r][d]);
        st.acc[r][d] = f2(0.f);
      }
  }
};

// ------------------------------------------------------------ adjoint 3D FP64
template <int R_, int TJ_, int MODE>
struct Grav3DF64Adj {
  static constexpr int R = R_, TJ = TJ_, NACC = 9, JB = RecordBytes<MD_GRAV3D, false, true>::value;
  static constexpr bool MASK = false;
  static constexpr int NR = R;
  static constexpr int FMT = 0;
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    double x[R], y[R], z[R], vx[R], vy[R], vz[R];
    double accd[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = st.accd[r][d];
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const double *m = (const double *)mirror + (i0 + row_of(r)) * 8;
      st.x[r] = m[0];
      st.y[r] = m[1];
      st.z[r] = m[2];
      st.vx[r] = m[3];
      st.vy[r] = m[4];
      st.vz[r] = m[5];
#pragma unroll
      for (int d = 0; d < NACC; d++) st.accd[r][d] = 0.0;
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t, int64_t) {
    const double4_16a *sm = (const double4_16a *)smb;
#pragma unroll 1
    for (int k = 0; k < TJ; k++) {
      const double4_16a P = sm[2 * k], V = sm[2 * k + 1];
#pragma unroll
      for (int r = 0; r < R; r++) {
        const double dx = st.x[r] - P.x, dy = st.y[r] - P.y, dz = st.z[r] - P.z;
        const double y = rsqrt_nr(fma(dx, dx, fma(dy, dy, fma(dz, dz, a.epsd))));
        const double y2 = y * y, w3 = y2 * y, w5 = w3 * y2;
        const double wx = st.vx[r] - P.w, wy = st.vy[r] - V.x, wz = st.vz[r] - V.y;
        const double t = -3.0 * fma(dx, wx, fma(dy, wy, dz * wz)) * w5;
        double *ac = st.accd[r];
        ac[0] = fma(dx, w3, ac[0]);
        ac[1] = fma(dy, w3, ac[1]);
        ac[2] = fma(dz, w3, ac[2]);
        ac[3] = fma(t, dx, fma(wx, w3, ac[3]));
        ac[4] = fma(t, dy, fma(wy, w3, ac[4]));
        ac[5] = fma(t, dz, fma(wz, w3, ac[5]));
        ac[6] = fma(dx, w5, ac[6]);
        ac[7] = fma(dy, w5, ac[7]);
        ac[8] = fma(dz, w5, ac[8]);
      }
    }
  }
};

// ------------------------------------------------------------ adjoint sheets FP32 (eps > 0)
// accumulators: 0 = force sum of d s^(-1/2); 1 = J w sum of s^(-3/2) w (times eps in the
// epilogue); 2 = d/deps sum of d s^(-3/2); s = d^2 + eps
template <int R_, int TJ_, int MODE, int MINB_ = 1>
struct SheetMixedAdj {
  static constexpr int STREAMK_MINB = MINB_;  // register budget of the one-sided kernel
  static constexpr int R = R_, TJ = TJ_, NACC = 3, JB = RecordBytes<MD_SHEET1D, true, true>::value;
  static constexpr bool MASK = false;
  static constexpr int NR = R;
  static constexpr int FMT = 0;
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    float2 x[R], v[R], acc[R][NACC];
    CompSum cs[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = csum_total(st.cs[r][d]);
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int64_t i = i0 + row_of(r);
      const float *m = (const float *)mirror + (i >> 1) * 4 + (i & 1);
      st.x[r] = f2(-m[0]);
      st.v[r] = f2(-m[2]);
#pragma unroll
      for (int d = 0; d < NACC; d++) {
        st.acc[r][d] = f2(0.f);
        st.cs[r][d] = CompSum{0.f, 0.f};
      }
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t, int64_t) {
    const float4 *sm = (const float4 *)smb;
    const float2 e2 = f2((float)a.epsd);
#pragma unroll 2
    for (int k = 0; k < TJ / 2; k++) {
      const float4 A = sm[k];
      const float2 nx = make_float2(A.x, A.y), nv = make_float2(A.z, A.w);
#pragma unroll
      for (int r = 0; r < R; r++) {
        const float2 d = __fadd2_rn(st.x[r], nx);
        const float2 s = __ffma2_rn(d, d, e2);
        const float2 y = make_float2(mufu_rsqrt(s.x), mufu_rsqrt(s.y));
        const float2 w3 = __fmul2_rn(__fmul2_rn(y, y), y);
        st.acc[r][0] = __ffma2_rn(d, y, st.acc[r][0]);
        st.acc[r][1] = __ffma2_rn(w3, __fadd2_rn(st.v[r], nv), st.acc[r][1]);
        st.acc[r][2] = __ffma2_rn(d, w3, st.acc[r][2]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
      for (int d = 0; d < NACC; d++) {
        csum_add2(st.cs[r][d], st.acc[r][d]);
        st.acc[r][d] = f2(0.f);
      }
  }
};

// ------------------------------------------------------------ adjoint sheets FP64 (eps > 0)
template <int R_, int TJ_, int MODE>
struct SheetF64Adj {
  static constexpr int R = R_, TJ = TJ_, NACC = 3, JB = RecordBytes<MD_SHEET1D, false, true>::value;
  static constexpr bool MASK = false;
  static constexpr int NR = R;
  static constexpr int FMT = 0;
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    double x[R], v[R];
    double accd[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = st.accd[r][d];
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const double *m = (const double *)mirror + (i0 + row_of(r)) * 2;
      st.x[r] = m[0];
      st.v[r] = m[1];
      st.accd[r][0] = st.accd[r][1] = st.accd[r][2] = 0.0;
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t, int64_t) {
    const double2 *sm = (const double2 *)smb;
#pragma unroll 2
    for (int k = 0; k < TJ; k++) {
      const double2 o = sm[k];
#pragma unroll
      for (int r = 0; r < R; r++) {
        const double d = st.x[r] - o.x;
        const double y = rsqrt_nr(fma(d, d, a.epsd));
        const double w3 = y * y * y;
        st.accd[r][0] = fma(d, y, st.accd[r][0]);
        st.accd[r][1] = fma(w3, st.v[r] - o.y, st.accd[r][1]);
        st.accd[r][2] = fma(d, w3, st.accd[r][2]);
      }
    }
  }
};

// ------------------------------------------------------------ adjoint Ring FP64
template <int R_, int TJ_, int MODE>
struct RingF64Adj {
  static constexpr int R = R_, TJ = TJ_, NACC = 3, JB = RecordBytes<MD_RING, false, true>::value;
  static constexpr bool MASK = true;
  static constexpr int NR = R;  // rows finished per thread
  static constexpr int FMT = 0;  // mirror record format
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    double s[R], c[R], a[R], g[R], v[R];
    double accd[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = st.accd[r][d];
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const double *m = (const double *)mirror + (i0 + row_of(r)) * 6;
      st.s[r] = m[0];
      st.c[r] = m[1];
      st.a[r] = m[2];
      st.g[r] = m[3];
      st.v[r] = m[4];
      st.accd[r][0] = st.accd[r][1] = st.accd[r][2] = 0.0;
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t i0, int64_t j0) {
    const double2 *sm = (const double2 *)smb;
#pragma unroll 2
    for (int k = 0; k < TJ; k++) {
      const double2 sc = sm[3 * k], ag = sm[3 * k + 1], vv = sm[3 * k + 2];
#pragma unroll
      for (int r = 0; r < R; r++) {
        double S = fma(st.s[r], sc.y, -(st.c[r] * sc.x));
        double C = fma(st.c[r], sc.y, st.s[r] * sc.x);
        double sh = fma(st.a[r], ag.y, -(st.g[r] * ag.x));
        double y = rsqrt_nr(fma(sh, sh, a.epsd));
        double y2 = y * y, r3 = y2 * y, r5 = r3 * y2;
        if (DIAG && i0 + row_of(r) == j0 + k) S = 0.0;
        st.accd[r][0] = fma(S, r3, st.accd[r][0]);
        st.accd[r][2] = fma(S, r5, st.accd[r][2]);
        double G = fma(-0.75 * S * S, r5, C * r3);
        st.accd[r][1] = fma(G, st.v[r] - vv.x, st.accd[r][1]);
      }
    }
  }
};

// ------------------------------------------------------------ adjoint 2D FP64
template <int R_, int TJ_, int MODE>
struct GravF64Adj {
  static constexpr int R = R_, TJ = TJ_, NACC = 6, JB = RecordBytes<MD_GRAV2D, false, true>::value;
  static constexpr bool MASK = false;
  static constexpr int NR = R;  // rows finished per thread
  static constexpr int FMT = 0;  // mirror record format
  __device__ static int row_of(int r) { return r * NT + (int)threadIdx.x; }
  struct State {
    double x[R], y[R], vx[R], vy[R];
    double accd[R][NACC];
  };
  __device__ static void total(const State &st, int r, double *out) {
#pragma unroll
    for (int d = 0; d < NACC; d++) out[d] = st.accd[r][d];
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const double *m = (const double *)mirror + (i0 + row_of(r)) * 4;
      st.x[r] = m[0];
      st.y[r] = m[1];
      st.vx[r] = m[2];
      st.vy[r] = m[3];
#pragma unroll
      for (int d = 0; d < NACC; d++) st.accd[r][d] = 0.0;
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t, int64_t) {
    const double2 *sm = (const double2 *)smb;
#pragma unroll 2
    for (int k = 0; k < TJ; k++) {
      const double2 xy = sm[2 * k], vv = sm[2 * k + 1];
#pragma unroll
      for (int r = 0; r < R; r++) {
        double dx = st.x[r] - xy.x, dy = st.y[r] - xy.y;
        double inv = rcp_nr(fma(dx, dx, fma(dy, dy, a.epsd)));
        double inv2 = inv * inv;
        double wx = st.vx[r] - vv.x, wy = st.vy[r] - vv.y;
        double m2u = -2.0 * fma(dy, wy, dx * wx) * inv2;
        st.accd[r][0] = fma(dx, inv, st.accd[r][0]);
        st.accd[r][1] = fma(dy, inv, st.accd[r][1]);
        st.accd[r][2] = fma(m2u, dx, fma(wx, inv, st.accd[r][2]));
        st.accd[r][3] = fma(m2u, dy, fma(wy, inv, st.accd[r][3]));
        st.accd[r][4] = fma(dx, inv2, st.accd[r][4]);
        st.accd[r][5] = fma(dy, inv2, st.accd[r][5]);
      }
    }
  }
};

// ------------------------------------------------ forward Ring, tensor cores
//
// sin(d) = s_i c_j - c_i s_j and sin(d/2) = a_i g_j - g_i a_j (a, g: sin, cos of
// the half angle) are dot products of length 2, so for a 16 x 8 block of pairs
// each is one warp-level matrix multiply.  The FP32 operands are split into
// TF32 hi + lo parts (round to nearest) and the three significant products
// hi.hi + hi.lo + lo.hi are laid along K (6 of the 8 K slots), which keeps the
// result within a few FP32 ulps.  What is left per pair is 4 FP32 operations
// and one rsqrt:  dd = sh^2 + eps/2,  acc += S * dd^(-3/2).
//   A row i (S):  [s_h, c_h, s_h, c_h, s_l, c_l, 0, 0]
//   B col j (S):  [c_h, -s_h, c_l, -s_l, c_h, -s_h, 0, 0]      (same with a, g for sh)
// The mirror record of the 8 particles of an n-block holds, per lane (g, t) of
// the m16n8k8 B fragment, the pair (B[t][g], B[t+4][g]) for S, then for sh:
// 512 bytes per 8 particles.

__device__ __forceinline__ unsigned tf32_rn(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// hi and lo TF32 parts of x (hi + lo = x to ~2^-22 relative)
__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
  hi = __uint_as_float(tf32_rn(x));
  lo = __uint_as_float(tf32_rn(x - hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%10,%10,%10,%10};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(0.f));
}

// TC record of particle i from FP32 (s, c, a, g); all-zero = padding
__device__ __forceinline__ void write_tc_record(void *mirror, int64_t i, float s, float c, float a, float g) {
  float *m = (float *)mirror + (i >> 3) * 128 + (i & 7) * 8;
  float sh, sl, ch, cl, ah, al, gh, gl;
  tf32_split(s, sh, sl);
  tf32_split(c, ch, cl);
  tf32_split(a, ah, al);
  tf32_split(g, gh, gl);
  // lanes 4g+t of the S fragment, then of the sin(d/2) fragment (64 floats later)
  float2 *S = (float2 *)m, *H = (float2 *)(m + 64);
  S[0] = make_float2(ch, ch);
  S[1] = make_float2(-sh, -sh);
  S[2] = make_float2(cl, 0.f);
  S[3] = make_float2(-sl, 0.f);
  H[0] = make_float2(gh, gh);
  H[1] = make_float2(-ah, -ah);
  H[2] = make_float2(gl, 0.f);
  H[3] = make_float2(-al, 0.f);
}

__device__ __forceinline__ void write_tc_pad(void *mirror, int64_t i) {
  float *m = (float *)mirror + (i >> 3) * 128 + (i & 7) * 8;
#pragma unroll
  for (int k = 0; k < 8; k++) m[k] = m[64 + k] = 0.f;
}

template <int RM_, int TJ_, int MODE, int THREADS_ = NT, int MINB_ = 4>
struct RingTC {
  static constexpr int THREADS = THREADS_;    // CTA size (the one-sided skeletons use NT)
  static constexpr int MINB = MINB_;          // resident CTAs per SM the register budget is set for
  using ColT = float;                         // column partials of the symmetric form
  static constexpr int RM = RM_;              // 16-row m-blocks per warp
  static constexpr int R = RM / 2 > 0 ? RM / 2 : 1;  // TI = THREADS * R = 16 RM rows per warp
  static constexpr int TJ = TJ_, NACC = 1, JB = 64;
  static constexpr bool MASK = true;
  static constexpr int NR = 2 * RM;           // rows g and g+8 of each m-block
  static constexpr int FMT = 1;               // tensor-core fragment records
  static_assert(THREADS * R == 16 * RM * (THREADS / 32), "tile rows: warps x RM m-blocks x 16");
  static_assert(RM % 2 == 0, "m-blocks are dealt to the warps in pairs");
  static constexpr int NW = THREADS / 32;
  // m-block (16 rows) of the tile held as this warp's r-th: the pair p = r / 2 of
  // blocks {2 NW p + w, 2 NW p + 2 NW - 1 - w}, so that every warp's blocks add up to
  // the same number of above-diagonal pairs in a diagonal tile (tile_diag)
  __device__ static int mblock(int r) {
    const int w = threadIdx.x >> 5, p = r >> 1;
    return (r & 1) ? 2 * NW * p + 2 * NW - 1 - w : 2 * NW * p + w;
  }
  __device__ static int mrow(int rr) {        // row offset in the tile of item rr = 2 r + h
    const int g = (threadIdx.x & 31) >> 2;
    return 16 * mblock(rr >> 1) + g + 8 * (rr & 1);
  }
  __device__ static int row_of(int rr) { return (threadIdx.x & 3) == 0 ? mrow(rr) : -1; }
  struct State {
    unsigned aS[RM][4], aH[RM][4];
    float2 acc[RM][2];
    CompSum cs[RM][2];
  };
  __device__ static void total(const State &st, int rr, double *out) {
    double v = csum_total(st.cs[rr >> 1][rr & 1]);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    out[0] = v;
  }
  __device__ static void load(State &st, const void *mirror, int64_t i0) {
    const int t = threadIdx.x & 3;
#pragma unroll
    for (int r = 0; r < RM; r++) {
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int64_t i = i0 + mrow(2 * r + h);
        const float *m = (const float *)mirror + (i >> 3) * 128 + (i & 7) * 8;
        // record lanes: 0 -> (c_h, c_h), 1 -> (-s_h, -s_h), 2 -> (c_l, 0), 3 -> (-s_l, 0)
        const float ch = m[0], sh = -m[2], cl = m[4], sl = -m[6];
        const float gh = m[64], ah = -m[66], gl = m[68], al = -m[70];
        const float s_lo = (t == 0) ? sl : (t == 1) ? cl : 0.f;  // A[row][t+4]
        const float h_lo = (t == 0) ? al : (t == 1) ? gl : 0.f;
        st.aS[r][h] = __float_as_uint((t & 1) ? ch : sh);      // A[row][t]
        st.aS[r][2 + h] = __float_as_uint(s_lo);
        st.aH[r][h] = __float_as_uint((t & 1) ? gh : ah);
        st.aH[r][2 + h] = __float_as_uint(h_lo);
      }
#pragma unroll
      for (int h = 0; h < 2; h++) {
        st.acc[r][h] = f2(0.f);
        st.cs[r][h] = CompSum{0.f, 0.f};
      }
    }
  }
  template <bool DIAG>
  __device__ static void tile(State &st, const unsigned char *smb, const PairArgs &a, int64_t i0, int64_t j0) {
    const float *sm = (const float *)smb;
    const float2 he = f2((float)a.epsd);
    const int lane = threadIdx.x & 31, t = lane & 3;
    // off-diagonal tiles (the one-sided kernel's bulk) unrolled by 4; diagonal tiles,
    // rare in both kernels, by 2: the symmetric kernel measured 2.7% slower with them
    // unrolled by 4 beside its tile_sym (same registers; more code)
#pragma unroll(DIAG ? 2 : 4)
    for (int k = 0; k < TJ / 8; k++) {
      const float2 bs = *(const float2 *)(sm + k * 128 + lane * 2);
      const float2 bh = *(const float2 *)(sm + k * 128 + 64 + lane * 2);
      const unsigned bs0 = __float_as_uint(bs.x), bs1 = __float_as_uint(bs.y);
      const unsigned bh0 = __float_as_uint(bh.x), bh1 = __float_as_uint(bh.y);
#pragma unroll
      for (int r = 0; r < RM; r++) {
        float dS[4], dH[4];
        mma_tf32(dS, st.aS[r], bs0, bs1);
        mma_tf32(dH, st.aH[r], bh0, bh1);
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const float2 S = make_float2(dS[2 * h], dS[2 * h + 1]);   // row g + 8h, columns 2t, 2t+1
          const float2 sh = make_float2(dH[2 * h], dH[2 * h + 1]);
          const float2 d = __ffma2_rn(sh, sh, he);
          const float2 y = make_float2(mufu_rsqrt(d.x), mufu_rsqrt(d.y));
          float2 qq = __fmul2_rn(S, y);
          if (DIAG) {
            const int64_t i = i0 + mrow(2 * r + h), j = j0 + 8 * k + 2 * t;
            if (i == j) qq.x = 0.f;
            if (i == j + 1) qq.y = 0.f;
          }
          st.acc[r][h] = __ffma2_rn(qq, __fmul2_rn(y, y), st.acc[r][h]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RM; r++)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        csum_add2(st.cs[r][h], st.acc[r][h]);
        st.acc[r][h] = f2(0.f);
      }
  }
  // Off-diagonal block of the Newton's-third-law variant: the i-rows as in tile<>,
  // and for every j the sum over this warp's 16 RM rows of the same terms
  // S dd^(-3/2), into colsm[warp TJ + j] (the j-side term is minus that sum, as
  // sin(theta_j - theta_i) = -sin(theta_i - theta_j)).  Per lane and n-block the
  // two columns 2t, 2t+1 are summed over the lane's rows; four n-blocks at a
  // time are then reduced over the 8 lanes g by a butterfly.
  __device__ static void tile_sym(State &st, const unsigned char *smb, const PairArgs &a, float *colsm) {
    const float *sm = (const float *)smb;
    const float2 he = f2((float)a.epsd);
    const int lane = threadIdx.x & 31, t = lane & 3, w = threadIdx.x >> 5;
#pragma unroll 2
    for (int k4 = 0; k4 < TJ / 32; k4++) {
      float v[8];
#pragma unroll
      for (int kk = 0; kk < 4; kk++) {
        const int k = 4 * k4 + kk;
        const float2 bs = *(const float2 *)(sm + k * 128 + lane * 2);
        const float2 bh = *(const float2 *)(sm + k * 128 + 64 + lane * 2);
        const unsigned bs0 = __float_as_uint(bs.x), bs1 = __float_as_uint(bs.y);
        const unsigned bh0 = __float_as_uint(bh.x), bh1 = __float_as_uint(bh.y);
        float2 col = f2(0.f);
#pragma unroll
        for (int r = 0; r < RM; r++) {
          float dS[4], dH[4];
          mma_tf32(dS, st.aS[r], bs0, bs1);
          mma_tf32(dH, st.aH[r], bh0, bh1);
#pragma unroll
          for (int h = 0; h < 2; h++) {
            const float2 S = make_float2(dS[2 * h], dS[2 * h + 1]);
            const float2 sh = make_float2(dH[2 * h], dH[2 * h + 1]);
            const float2 d = __ffma2_rn(sh, sh, he);
            const float2 y = make_float2(mufu_rsqrt(d.x), mufu_rsqrt(d.y));
            const float2 qq = __fmul2_rn(S, y);
            const float2 y2 = __fmul2_rn(y, y);
            st.acc[r][h] = __ffma2_rn(qq, y2, st.acc[r][h]);
            col = __ffma2_rn(qq, y2, col);
          }
        }
        v[2 * kk] = col.x;
        v[2 * kk + 1] = col.y;
      }
      // lane (g, t) ends with n-block 4 k4 + (g >> 1), column 2t + (g & 1)
      const float sum = butterfly_sum<8, 16>(v, lane);
      colsm[w * TJ + 8 * (4 * k4 + (lane >> 3)) + 2 * t + ((lane >> 2) & 1)] = sum;
    }
#pragma unroll
    for (int r = 0; r < RM; r++)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        csum_add2(st.cs[r][h], st.acc[r][h]);
        st.acc[r][h] = f2(0.f);
      }
  }
  // Diagonal tile of the Newton's-third-law variant (TI = TJ: the columns are the
  // tile's own particles).  m-block b (rows 16b .. 16b+15) against n-block k (columns
  // 8k .. 8k+7): k >= 2b + 2 lies above the diagonal and is evaluated as in tile_sym
  // (row and column sums); k = 2b, 2b+1 is the block's own 16 x 16 square, evaluated
  // one-sided as in tile<true> (each ordered pair on its row, the self term masked);
  // k < 2b mirrors an above-diagonal block of another m-block and is skipped.  Every
  // warp's m-blocks (mblock) have the same number of n-blocks to do; colsm gets
  // every column (zero where none of the warp's m-blocks lies above it).
  __device__ static void tile_diag(State &st, const unsigned char *smb, const PairArgs &a, float *colsm, int) {
    static_assert(16 * RM * NW == TJ, "diagonal tiles are square");
    const float *sm = (const float *)smb;
    const float2 he = f2((float)a.epsd);
    const int lane = threadIdx.x & 31, t = lane & 3, w = threadIdx.x >> 5;
    // one pair term: row sum, and the column sum when the pair lies above the diagonal
    auto term = [&](int r, const float (&dS)[4], const float (&dH)[4], float2 &col, bool above, int k) {
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const float2 S = make_float2(dS[2 * h], dS[2 * h + 1]);
        const float2 sh = make_float2(dH[2 * h], dH[2 * h + 1]);
        const float2 d = __ffma2_rn(sh, sh, he);
        const float2 y = make_float2(mufu_rsqrt(d.x), mufu_rsqrt(d.y));
        float2 qq = __fmul2_rn(S, y);
        if (!above) {
          const int i = mrow(2 * r + h), j = 8 * k + 2 * t;
          if (i == j) qq.x = 0.f;
          if (i == j + 1) qq.y = 0.f;
        }
        const float2 y2 = __fmul2_rn(y, y);
        st.acc[r][h] = __ffma2_rn(qq, y2, st.acc[r][h]);
        if (above) col = __ffma2_rn(qq, y2, col);
      }
    };
#pragma unroll 1
    for (int k4 = 0; k4 < TJ / 32; k4++) {
      unsigned b[4][4];
#pragma unroll
      for (int kk = 0; kk < 4; kk++) {
        const int k = 4 * k4 + kk;
        const float2 bs = *(const float2 *)(sm + k * 128 + lane * 2);
        const float2 bh = *(const float2 *)(sm + k * 128 + 64 + lane * 2);
        b[kk][0] = __float_as_uint(bs.x);
        b[kk][1] = __float_as_uint(bs.y);
        b[kk][2] = __float_as_uint(bh.x);
        b[kk][3] = __float_as_uint(bh.y);
      }
      float2 col[4];
#pragma unroll
      for (int kk = 0; kk < 4; kk++) col[kk] = f2(0.f);
#pragma unroll
      for (int r = 0; r < RM; r++) {
        // the m-block's own n-blocks kb, kb + 1 (kb even: both in one group of 4)
        const int kb = 2 * mblock(r);
        if (4 * k4 >= kb + 2) {
          // the whole group lies above the m-block: as tile_sym
#pragma unroll
          for (int kk = 0; kk < 4; kk++) {
            float dS[4], dH[4];
            mma_tf32(dS, st.aS[r], b[kk][0], b[kk][1]);
            mma_tf32(dH, st.aH[r], b[kk][2], b[kk][3]);
            term(r, dS, dH, col[kk], true, 4 * k4 + kk);
          }
        } else if (4 * k4 + 4 > kb) {
          // the group holds the m-block's own square (and, before it, skipped
          // n-blocks or, after it, n-blocks above)
#pragma unroll
          for (int kk = 0; kk < 4; kk++) {
            const int k = 4 * k4 + kk;
            if (k < kb) continue;
            float dS[4], dH[4];
            mma_tf32(dS, st.aS[r], b[kk][0], b[kk][1]);
            mma_tf32(dH, st.aH[r], b[kk][2], b[kk][3]);
            term(r, dS, dH, col[kk], k >= kb + 2, k);
          }
        }
      }
      float v[8];
#pragma unroll
      for (int kk = 0; kk < 4; kk++) {
        v[2 * kk] = col[kk].x;
        v[2 * kk + 1] = col[kk].y;
      }
      const float sum = butterfly_sum<8, 16>(v, lane);
      colsm[w * TJ + 8 * (4 * k4 + (lane >> 3)) + 2 * t + ((lane >> 2) & 1)] = sum;
    }
#pragma unroll
    for (int r = 0; r < RM; r++)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        csum_add2(st.cs[r][h], st.acc[r][h]);
        st.acc[r][h] = f2(0.f);
      }
  }
};

// Record writers by format: FMT 0 = interleaved FP32 / FP64 records above,
// FMT 1 = Ring tensor-core fragment records (FP32 forward stages only).
template <int MODEL, bool MIXED, bool ADJ, int FMT>
__device__ __forceinline__ void write_record_fmt(void *mirror, int64_t i, double x, double y, double vx, double vy) {
  if constexpr (FMT == 1) {
    const float r = (float)reduce_2pi(x);
    float s, c, a, g;
    sincos_small(r, &s, &c);
    sincos_small(0.5f * r, &a, &g);
    write_tc_record(mirror, i, s, c, a, g);
  } else {
    write_record<MODEL, MIXED, ADJ>(mirror, i, x, y, vx, vy);
  }
}
template <int MODEL, bool MIXED, bool ADJ, int FMT>
__device__ __forceinline__ void write_pad_fmt(void *mirror, int64_t i) {
  if constexpr (FMT == 1)
    write_tc_pad(mirror, i);
  else
    write_pad<MODEL, MIXED, ADJ>(mirror, i);
}

// ============================================================ epilogues ====

// Forward stages: kick, drift, new mirror record (or the force alone).
template <int MODEL, bool MIXED, int MODE, int FMT, bool SHARD = false>
__device__ __forceinline__ void finish_forward(const PairArgs &a, int64_t i, const double *acc) {
  constexpr int D = dim_of<MODEL>();
  // state index and leading dimension: global ones, or the shard's local rows
  const int64_t li = SHARD ? i - a.row0 : i;
  const int64_t ld = SHARD ? a.nrow : a.N;
  if (li >= ld) return;
  const double scale = MODEL == MD_RING ? -1.0 / (8.0 * (double)a.N)
                       : MODEL == MD_GRAV3D ? -1.0 / (double)a.N
                                            : -2.0 / (double)a.N;
  double f[D], x[D];
#pragma unroll
  for (int d = 0; d < D; d++) f[d] = MODEL == MD_SHEET1D ? -acc[d] / (double)a.N : scale * acc[d];
  if constexpr (MODE == STAGE_FORCE_ONLY) {
#pragma unroll
    for (int d = 0; d < D; d++) a.fout[d * ld + li] = f[d];
    return;
  } else {
#pragma unroll
    for (int d = 0; d < D; d++) {
      const double pp = fma(a.kick, f[d], a.p[d * ld + li]);
      a.p[d * ld + li] = pp;
      if (MODE == STAGE_KICK_DRIFT) {
        x[d] = fma(a.drift, pp, a.q[d * ld + li]);
        a.q[d * ld + li] = x[d];
      } else {
        a.fout[d * ld + li] = f[d];
      }
    }
  }
  if constexpr (MODE == STAGE_KICK_DRIFT) {
    if constexpr (MODEL == MD_GRAV3D)
      write_record3<MIXED>(a.mirror_out, i, x[0], x[1], x[D - 1]);
    else if constexpr (MODEL == MD_SHEET1D)
      write_record1<MIXED>(a.mirror_out, i, x[0]);
    else
      write_record_fmt<MODEL, MIXED, false, FMT>(a.mirror_out, i, x[0], x[D - 1], 0.0, 0.0);
  }
}

// Reverse stages of md_grad, at the position q_s of one kick (b_adj = a.kick,
// b_undo = a.undo) and the drift that preceded it (a.drift):
//   lambda_q += b_adj J(q_s) lambda_p ;  epsacc += b_adj <lambda_p, df/deps(q_s)>
//   p -= b_undo f(q_s)                          (undo the kick)
//   lambda_p += d lambda_q ;  q -= d p          (adjoint and undo of the drift)
// Force, J v and df/deps of particle i from the reverse-stage accumulators
// (layout of the *Adj policies: [force sums][J w sums][d/deps sums], D each).
template <int MODEL>
__device__ __forceinline__ void adjoint_terms(const PairArgs &a, const double *acc, double *f, double *jv, double *de) {
  constexpr int D = dim_of<MODEL>();
  const double n = (double)a.N;
#pragma unroll
  for (int d = 0; d < D; d++) {
    if (MODEL == MD_RING) {
      f[d] = -acc[0] / (8.0 * n);
      jv[d] = -acc[1] / (8.0 * n);
      de[d] = 3.0 * acc[2] / (32.0 * n);
    } else if (MODEL == MD_GRAV2D) {
      f[d] = -2.0 * acc[d] / n;
      jv[d] = -2.0 * acc[2 + d] / n;
      de[d] = 2.0 * acc[4 + d] / n;
    } else if (MODEL == MD_GRAV3D) {
      f[d] = -acc[d] / n;
      jv[d] = -acc[3 + d] / n;
      de[d] = 1.5 * acc[6 + d] / n;
    } else {  // sheets (eps > 0)
      f[d] = -acc[0] / n;
      jv[d] = -a.epsd * acc[1] / n;
      de[d] = 0.5 * acc[2] / n;
    }
  }
}

// Adjoint record (positions x, lambda_p v) of particle i, per model.
template <int MODEL, bool MIXED>
__device__ __forceinline__ void write_adjoint_record(void *mirror, int64_t i, const double *x, const double *v) {
  constexpr int D = dim_of<MODEL>();
  if constexpr (MODEL == MD_GRAV3D)
    write_record3_adj<MIXED>(mirror, i, x, v);
  else if constexpr (MODEL == MD_SHEET1D)
    write_record1_adj<MIXED>(mirror, i, x[0], v[0]);
  else
    write_record<MODEL, MIXED, true>(mirror, i, x[0], x[D - 1], v[0], v[D - 1]);
}

template <int MODEL, bool MIXED>
__device__ __forceinline__ void finish_adjoint(const PairArgs &a, int64_t i, const double *acc) {
  constexpr int D = dim_of<MODEL>();
  if (i >= a.N) return;
  double f[D], jv[D], de[D];
  adjoint_terms<MODEL>(a, acc, f, jv, de);
  double lq[D], lp[D], x[D], e = 0.0;
#pragma unroll
  for (int d = 0; d < D; d++) {
    lp[d] = a.lp[d * a.N + i];
    lq[d] = fma(a.kick, jv[d], a.lq[d * a.N + i]);
    e = fma(lp[d], de[d], e);
    double pp = fma(-a.undo, f[d], a.p[d * a.N + i]);
    a.p[d * a.N + i] = pp;
    x[d] = a.q[d * a.N + i];
    if (a.drift != 0.0) {
      lp[d] = fma(a.drift, lq[d], lp[d]);
      x[d] = fma(-a.drift, pp, x[d]);
      a.lp[d * a.N + i] = lp[d];
      a.q[d * a.N + i] = x[d];
    }
    a.lq[d * a.N + i] = lq[d];
  }
  a.epsacc[i] = fma(a.kick, e, a.epsacc[i]);
  if (a.drift != 0.0) write_adjoint_record<MODEL, MIXED>(a.mirror_out, i, x, lp);
}

// Tangent stages (forward-mode derivative of the stage map), with a.lq = dq and
// a.lp = dp: p += kick f; dp += kick J dq; then q += drift p; dq += drift dp and
// a new adjoint-format record (q, dq) for the next stage.
template <int MODEL, bool MIXED>
__device__ __forceinline__ void finish_tangent(const PairArgs &a, int64_t i, const double *acc) {
  constexpr int D = dim_of<MODEL>();
  if (i >= a.N) return;
  double f[D], jv[D], de[D], x[D], v[D];
  adjoint_terms<MODEL>(a, acc, f, jv, de);
#pragma unroll
  for (int d = 0; d < D; d++) {
    const double pp = fma(a.kick, f[d], a.p[d * a.N + i]);
    const double dpp = fma(a.kick, jv[d], a.lp[d * a.N + i]);
    a.p[d * a.N + i] = pp;
    a.lp[d * a.N + i] = dpp;
    x[d] = a.q[d * a.N + i];
    v[d] = a.lq[d * a.N + i];
    if (a.drift != 0.0) {
      x[d] = fma(a.drift, pp, x[d]);
      v[d] = fma(a.drift, dpp, v[d]);
      a.q[d * a.N + i] = x[d];
      a.lq[d * a.N + i] = v[d];
    }
  }
  if (a.drift != 0.0) write_adjoint_record<MODEL, MIXED>(a.mirror_out, i, x, v);
}

template <class Pol, int MODEL, bool MIXED, int MODE, bool SHARD = false>
__device__ __forceinline__ void finish(const PairArgs &a, int64_t i, const double *acc) {
  if constexpr (MODE == STAGE_ADJOINT) {
    finish_adjoint<MODEL, MIXED>(a, i, acc);
  } else if constexpr (MODE == STAGE_TANGENT) {
    finish_tangent<MODEL, MIXED>(a, i, acc);
  } else if constexpr (MODEL == MD_SHEET1D && !MIXED) {
    // FP64 sheets at eps = 0: each of the n_jt TJ - N padding records added +1
    const double c0 = a.epsd > 0.0 ? acc[0] : acc[0] - (double)(a.n_jt * Pol::TJ - a.N);
    finish_forward<MODEL, MIXED, MODE, Pol::FMT, SHARD>(a, i, &c0);
  } else {
    finish_forward<MODEL, MIXED, MODE, Pol::FMT, SHARD>(a, i, acc);
  }
}

}  // namespace
