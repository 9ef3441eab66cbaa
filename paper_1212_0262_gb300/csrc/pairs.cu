// Ring and 2D self-gravitating models (Sec. 3.2): direct all-pairs forces fused
// with the integrator's kick and drift.
//
// Tiling (after the tile algorithm of Sec. 3.2 / Fig. 1): an i-tile of
// TI = NT*R particles lives in registers (R per thread); j-tiles of TJ particles
// of a position "mirror" are staged in shared memory with cp.async, double
// buffered.  Every i visits every j (Newton's third law is not used, as in the
// paper).  Work is split stream-K style: the grid is P persistent CTAs, and CTA
// c takes the contiguous range [U c / P, U (c+1) / P) of the U = n_it * n_jt
// (i-tile, j-tile) units in i-major order, so every CTA does the same number of
// pair interactions.  An i-tile covered by several CTAs is finished by the last
// of them to arrive (atomic ticket per i-tile, no waiting), which adds the FP64
// partial sums in CTA order: results are deterministic.
//
// Pair arithmetic.
//   Ring:  f_i = -(1/(2 sqrt2 N)) sum_j sin(d) / (1 - cos d + eps)^(3/2)
//          (minus the gradient of Eq. 1; Eq. 8 with the sign of the Hamiltonian).
//          sin(d) comes from the product form of Eq. 9 on (sin, cos) of each
//          angle; 1 - cos d is taken as 2 sin^2(d/2) from (sin, cos) of the half
//          angles, which avoids the cancellation of Eq. 9's denominator for close
//          pairs.  With dd = sin^2(d/2) + eps/2: f_i = -(1/(8N)) sum S dd^(-3/2).
//   2D:    f_i = -(2/N) sum_j r_ij / (|r_ij|^2 + eps)   (minus the gradient of Eq. 3).
// MIXED: the mirror holds FP32 values, two j's are processed per packed
// f32x2 instruction (FFMA2/FMUL2/FADD2), 1/sqrt and 1/x use the SFU
// (rsqrt.approx / rcp.approx, as the paper uses rsqrt), per-tile sums are FP32
// and are added into FP64 per-particle accumulators once per j-tile
// (Sec. 3.2: FP32 pair force added into a double).  FP64: everything in double,
// with Newton-refined reciprocal square roots and reciprocals.
#include <algorithm>

#include "md_internal.cuh"

namespace {

constexpr int NT = kPairThreads;
constexpr int kPadMultiple = 1024;  // mirror padding: multiple of every TI and TJ

// bytes per particle in the mirror
template <int MODEL, bool MIXED>
struct MirrorFmt {
  static constexpr int bytes = MODEL == MD_RING ? (MIXED ? 16 : 32) : (MIXED ? 8 : 16);
};

struct PairArgs {
  const void *mirror_in;
  void *mirror_out;
  double *q, *p;
  int64_t N;
  int64_t n_it, n_jt, U;
  int P;
  double scale;  // force prefactor (Ring: -1/(8N); 2D: -2/N)
  double epsd;   // Ring: eps/2; 2D: eps
  double kick, drift;
  double *slots;  // [P][2][dim][TI] FP64 partial sums
  unsigned *tickets;
  double *fout;   // STAGE_KICK_ONLY / STAGE_FORCE_ONLY force output (dim*N)
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

// ----------------------------------------------------------- i-side state --

template <int MODEL, bool MIXED, int R>
struct IState;

template <int R>
struct IState<MD_RING, true, R> {
  float2 s[R], c[R], a[R], g[R];  // sin, cos, sin(half), cos(half), each duplicated
  float2 acc[R];
  double accd[R][1];
};
template <int R>
struct IState<MD_GRAV2D, true, R> {
  float2 x[R], y[R];
  float2 fx[R], fy[R];
  double accd[R][2];
};
template <int R>
struct IState<MD_RING, false, R> {
  double s[R], c[R], a[R], g[R];
  double accd[R][1];
};
template <int R>
struct IState<MD_GRAV2D, false, R> {
  double x[R], y[R];
  double accd[R][2];
};

template <int MODEL, bool MIXED, int R>
__device__ __forceinline__ void load_i(IState<MODEL, MIXED, R> &st, const void *mirror, int64_t i0) {
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t i = i0 + (int64_t)r * NT;
    if constexpr (MODEL == MD_RING && MIXED) {
      const float *m = (const float *)mirror + (i >> 1) * 8 + (i & 1);
      float ns = m[0], c = m[2], na = m[4], g = m[6];
      st.s[r] = make_float2(-ns, -ns);
      st.c[r] = make_float2(c, c);
      st.a[r] = make_float2(-na, -na);
      st.g[r] = make_float2(g, g);
      st.acc[r] = make_float2(0.f, 0.f);
      st.accd[r][0] = 0.0;
    } else if constexpr (MODEL == MD_GRAV2D && MIXED) {
      const float *m = (const float *)mirror + (i >> 1) * 4 + (i & 1);
      float nx = m[0], ny = m[2];
      st.x[r] = make_float2(-nx, -nx);
      st.y[r] = make_float2(-ny, -ny);
      st.fx[r] = st.fy[r] = make_float2(0.f, 0.f);
      st.accd[r][0] = st.accd[r][1] = 0.0;
    } else if constexpr (MODEL == MD_RING) {
      const double *m = (const double *)mirror + i * 4;
      st.s[r] = m[0];
      st.c[r] = m[1];
      st.a[r] = m[2];
      st.g[r] = m[3];
      st.accd[r][0] = 0.0;
    } else {
      const double *m = (const double *)mirror + i * 2;
      st.x[r] = m[0];
      st.y[r] = m[1];
      st.accd[r][0] = st.accd[r][1] = 0.0;
    }
  }
}

// ------------------------------------------------------------ tile bodies --

// One unit: all R i's of this thread against the TJ j's staged in smem.
// DIAG: the j-tile overlaps the i-tile (Ring only: the j == i term is masked,
// because the product form leaves a rounding residual there).
template <int MODEL, bool MIXED, int R, int TJ, bool DIAG>
__device__ __forceinline__ void tile_body(IState<MODEL, MIXED, R> &st, const unsigned char *smb,
                                          double epsd, int64_t i0, int64_t j0) {
  if constexpr (MODEL == MD_RING && MIXED) {
    const float4 *sm = (const float4 *)smb;
    const float h = (float)epsd;
    const float2 he = make_float2(h, h);
#pragma unroll 2
    for (int k = 0; k < TJ / 2; k++) {
      const float4 A = sm[2 * k], B = sm[2 * k + 1];
      const float2 nsj = make_float2(A.x, A.y), cj = make_float2(A.z, A.w);
      const float2 naj = make_float2(B.x, B.y), gj = make_float2(B.z, B.w);
#pragma unroll
      for (int r = 0; r < R; r++) {
        float2 t = __fmul2_rn(st.c[r], nsj);
        float2 S = __ffma2_rn(st.s[r], cj, t);       // sin(theta_i - theta_j)
        float2 u = __fmul2_rn(st.g[r], naj);
        float2 sh = __ffma2_rn(st.a[r], gj, u);      // sin((theta_i - theta_j)/2)
        float2 d = __ffma2_rn(sh, sh, he);           // (1 - cos + eps)/2
        float2 y = make_float2(mufu_rsqrt(d.x), mufu_rsqrt(d.y));
        float2 y2 = __fmul2_rn(y, y);
        float2 qq = __fmul2_rn(S, y);
        if (DIAG) {
          const int64_t i = i0 + (int64_t)r * NT, j = j0 + 2 * k;
          if (i == j) qq.x = 0.f;
          if (i == j + 1) qq.y = 0.f;
        }
        st.acc[r] = __ffma2_rn(qq, y2, st.acc[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      st.accd[r][0] += (double)st.acc[r].x + (double)st.acc[r].y;
      st.acc[r] = make_float2(0.f, 0.f);
    }
  } else if constexpr (MODEL == MD_GRAV2D && MIXED) {
    const float4 *sm = (const float4 *)smb;
    const float e = (float)epsd;
    const float2 e2 = make_float2(e, e);
#pragma unroll 2
    for (int k = 0; k < TJ / 2; k++) {
      const float4 X = sm[k];
      const float2 nx = make_float2(X.x, X.y), ny = make_float2(X.z, X.w);
#pragma unroll
      for (int r = 0; r < R; r++) {
        float2 dx = __fadd2_rn(st.x[r], nx);
        float2 dy = __fadd2_rn(st.y[r], ny);
        float2 s = __ffma2_rn(dy, dy, e2);
        s = __ffma2_rn(dx, dx, s);
        float2 inv = make_float2(mufu_rcp(s.x), mufu_rcp(s.y));
        st.fx[r] = __ffma2_rn(dx, inv, st.fx[r]);
        st.fy[r] = __ffma2_rn(dy, inv, st.fy[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
      st.accd[r][0] += (double)st.fx[r].x + (double)st.fx[r].y;
      st.accd[r][1] += (double)st.fy[r].x + (double)st.fy[r].y;
      st.fx[r] = st.fy[r] = make_float2(0.f, 0.f);
    }
  } else if constexpr (MODEL == MD_RING) {
    const double2 *sm = (const double2 *)smb;
#pragma unroll 2
    for (int k = 0; k < TJ; k++) {
      const double2 sc = sm[2 * k], ag = sm[2 * k + 1];
#pragma unroll
      for (int r = 0; r < R; r++) {
        double S = fma(st.s[r], sc.y, -(st.c[r] * sc.x));
        double sh = fma(st.a[r], ag.y, -(st.g[r] * ag.x));
        double d = fma(sh, sh, epsd);
        double y = rsqrt_nr(d);
        double qq = S * y;
        if (DIAG) {
          if (i0 + (int64_t)r * NT == j0 + k) qq = 0.0;
        }
        st.accd[r][0] = fma(qq, y * y, st.accd[r][0]);
      }
    }
  } else {
    const double2 *sm = (const double2 *)smb;
#pragma unroll 2
    for (int k = 0; k < TJ; k++) {
      const double2 xy = sm[k];
#pragma unroll
      for (int r = 0; r < R; r++) {
        double dx = st.x[r] - xy.x, dy = st.y[r] - xy.y;
        double s = fma(dx, dx, fma(dy, dy, epsd));
        double inv = rcp_nr(s);
        st.accd[r][0] = fma(dx, inv, st.accd[r][0]);
        st.accd[r][1] = fma(dy, inv, st.accd[r][1]);
      }
    }
  }
}

// ----------------------------------------------------------- epilogue -----

// Mirror record of particle i at FP64 position(s) (x, y) into `mirror`.
template <int MODEL, bool MIXED>
__device__ __forceinline__ void write_mirror(void *mirror, int64_t i, double x, double y) {
  if constexpr (MODEL == MD_RING) {
    double r = reduce_2pi(x);
    if constexpr (MIXED) {
      float s, c, a, g;
      sincos_small((float)r, &s, &c);
      sincos_small(0.5f * (float)r, &a, &g);
      float *m = (float *)mirror + (i >> 1) * 8 + (i & 1);
      m[0] = -s;
      m[2] = c;
      m[4] = -a;
      m[6] = g;
    } else {
      double s, c, a, g;
      sincos(x, &s, &c);
      sincos(0.5 * r, &a, &g);
      double *m = (double *)mirror + i * 4;
      m[0] = s;
      m[1] = c;
      m[2] = a;
      m[3] = g;
    }
  } else {
    if constexpr (MIXED) {
      float *m = (float *)mirror + (i >> 1) * 4 + (i & 1);
      m[0] = -(float)x;
      m[2] = -(float)y;
    } else {
      double *m = (double *)mirror + i * 2;
      m[0] = x;
      m[1] = y;
    }
  }
}

// Padding record: contributes exactly zero to every force.  Ring: all-zero
// (sin d = 0 with a positive denominator).  2D: so far away that |r|^2 overflows
// to +inf, whose reciprocal is 0 (the FP64 path's Newton steps keep 0).
template <int MODEL, bool MIXED>
__device__ __forceinline__ void write_pad(void *mirror, int64_t i) {
  if constexpr (MODEL == MD_RING) {
    if constexpr (MIXED) {
      float *m = (float *)mirror + (i >> 1) * 8 + (i & 1);
      m[0] = m[2] = m[4] = m[6] = 0.f;
    } else {
      double *m = (double *)mirror + i * 4;
      m[0] = m[1] = m[2] = m[3] = 0.0;
    }
  } else {
    if constexpr (MIXED) {
      float *m = (float *)mirror + (i >> 1) * 4 + (i & 1);
      m[0] = m[2] = -3.0e19f;
    } else {
      double *m = (double *)mirror + i * 2;
      m[0] = m[1] = 1.0e150;
    }
  }
}

template <int MODEL, bool MIXED, int MODE>
__device__ __forceinline__ void finish_particle(const PairArgs &a, int64_t i, const double *f) {
  constexpr int D = MODEL == MD_GRAV2D ? 2 : 1;
  if (i >= a.N) return;
  if (MODE == STAGE_FORCE_ONLY) {
#pragma unroll
    for (int d = 0; d < D; d++) a.fout[d * a.N + i] = f[d];
    return;
  }
  double q[D];
#pragma unroll
  for (int d = 0; d < D; d++) {
    double pp = fma(a.kick, f[d], a.p[d * a.N + i]);
    a.p[d * a.N + i] = pp;
    if (MODE == STAGE_KICK_DRIFT) {
      q[d] = fma(a.drift, pp, a.q[d * a.N + i]);
      a.q[d * a.N + i] = q[d];
    } else {
      a.fout[d * a.N + i] = f[d];
    }
  }
  if (MODE == STAGE_KICK_DRIFT) write_mirror<MODEL, MIXED>(a.mirror_out, i, q[0], D == 2 ? q[D - 1] : 0.0);
}

// ------------------------------------------------------------ the kernel --

template <int MODEL, bool MIXED, int R, int TJ, int MODE>
__global__ void __launch_bounds__(NT) pair_stage_kernel(PairArgs a) {
  constexpr int D = MODEL == MD_GRAV2D ? 2 : 1;
  constexpr int JB = MirrorFmt<MODEL, MIXED>::bytes;
  constexpr int TILE_BYTES = TJ * JB;
  constexpr int CHUNKS = TILE_BYTES / 16;
  constexpr int64_t TI = (int64_t)NT * R;
  __shared__ __align__(16) unsigned char sbuf[2][TILE_BYTES];
  __shared__ bool s_last;

  const int64_t cta = blockIdx.x;
  const int64_t u0 = unit_begin(a.U, a.P, cta), u1 = unit_begin(a.U, a.P, cta + 1);
  if (u0 >= u1) return;
  const int64_t first_row = u0 / a.n_jt;
  const unsigned char *mir = (const unsigned char *)a.mirror_in;

  auto prefetch = [&](int buf, int64_t jt) {
    const unsigned char *src = mir + jt * (int64_t)TILE_BYTES;
    for (int ch = threadIdx.x; ch < CHUNKS; ch += NT) cp_async16(&sbuf[buf][ch * 16], src + ch * 16);
    cp_async_commit();
  };

  IState<MODEL, MIXED, R> st;
  int64_t it = u0 / a.n_jt, jt = u0 % a.n_jt;
  bool row_from_start = (jt == 0);
  int64_t i0 = it * TI + threadIdx.x;
  load_i<MODEL, MIXED, R>(st, a.mirror_in, i0);
  prefetch(0, jt);

  for (int64_t u = u0; u < u1; u++) {
    const int buf = (int)((u - u0) & 1);
    if (u + 1 < u1) {
      prefetch(buf ^ 1, jt + 1 == a.n_jt ? 0 : jt + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int64_t j0 = jt * TJ;
    const bool diag = MODEL == MD_RING && (j0 < it * TI + TI) && (it * TI < j0 + TJ);
    if (diag)
      tile_body<MODEL, MIXED, R, TJ, true>(st, sbuf[buf], a.epsd, i0, j0);
    else
      tile_body<MODEL, MIXED, R, TJ, false>(st, sbuf[buf], a.epsd, i0, j0);
    __syncthreads();
    jt++;
    const bool row_end = (jt == a.n_jt);
    if (row_end || u + 1 == u1) {
      if (row_end && row_from_start) {
        // this CTA covered the whole i-tile: finish it directly
#pragma unroll
        for (int r = 0; r < R; r++) {
          double f[D];
#pragma unroll
          for (int d = 0; d < D; d++) f[d] = a.scale * st.accd[r][d];
          finish_particle<MODEL, MIXED, MODE>(a, i0 + (int64_t)r * NT, f);
        }
      } else {
        // partial coverage: publish, and let the last contributor finish
        const int slot = (it == first_row) ? 0 : 1;
        double *sp = a.slots + ((cta * 2 + slot) * D) * TI;
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
          for (int d = 0; d < D; d++) sp[d * TI + r * NT + threadIdx.x] = st.accd[r][d];
        __threadfence();
        __syncthreads();
        const int64_t cf = cta_of_unit(a.U, a.P, it * a.n_jt);
        const int64_t cl = cta_of_unit(a.U, a.P, (it + 1) * a.n_jt - 1);
        if (threadIdx.x == 0) {
          unsigned n = atomicAdd(&a.tickets[it], 1u) + 1u;
          s_last = (n == (unsigned)(cl - cf + 1));
        }
        __syncthreads();
        if (s_last) {
          __threadfence();
          double tot[R][D];
#pragma unroll
          for (int r = 0; r < R; r++)
#pragma unroll
            for (int d = 0; d < D; d++) tot[r][d] = 0.0;
          for (int64_t c2 = cf; c2 <= cl; c2++) {
            const int64_t fr = unit_begin(a.U, a.P, c2) / a.n_jt;
            const int sl = (it == fr) ? 0 : 1;
            const double *src = a.slots + ((c2 * 2 + sl) * D) * TI;
#pragma unroll
            for (int r = 0; r < R; r++)
#pragma unroll
              for (int d = 0; d < D; d++) tot[r][d] += __ldcg(src + d * TI + r * NT + threadIdx.x);
          }
#pragma unroll
          for (int r = 0; r < R; r++) {
            double f[D];
#pragma unroll
            for (int d = 0; d < D; d++) f[d] = a.scale * tot[r][d];
            finish_particle<MODEL, MIXED, MODE>(a, i0 + (int64_t)r * NT, f);
          }
          if (threadIdx.x == 0) a.tickets[it] = 0u;
        }
      }
      if (row_end && u + 1 < u1) {
        it++;
        jt = 0;
        row_from_start = true;
        i0 = it * TI + threadIdx.x;
        load_i<MODEL, MIXED, R>(st, a.mirror_in, i0);
      }
    }
  }
}

// Whole mirror from the FP64 state, including padding records.
template <int MODEL, bool MIXED>
__global__ void mirror_kernel(const double *__restrict__ q, int64_t N, int64_t Npad, void *m0, void *m1) {
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Npad; i += G) {
    if (i < N) {
      write_mirror<MODEL, MIXED>(m0, i, q[i], MODEL == MD_GRAV2D ? q[N + i] : 0.0);
    } else {
      write_pad<MODEL, MIXED>(m0, i);
      if (m1) write_pad<MODEL, MIXED>(m1, i);
    }
  }
}

// First stage from the cached force: p += kick f; q += drift p; new mirror.
template <int MODEL, bool MIXED>
__global__ void kick_drift_cached_kernel(double *__restrict__ q, double *__restrict__ p,
                                         const double *__restrict__ f, int64_t N, double kick,
                                         double drift, void *mirror_out) {
  constexpr int D = MODEL == MD_GRAV2D ? 2 : 1;
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += G) {
    double x[D];
#pragma unroll
    for (int d = 0; d < D; d++) {
      double pp = fma(kick, f[d * N + i], p[d * N + i]);
      p[d * N + i] = pp;
      x[d] = fma(drift, pp, q[d * N + i]);
      q[d * N + i] = x[d];
    }
    write_mirror<MODEL, MIXED>(mirror_out, i, x[0], x[D - 1]);
  }
}

// ------------------------------------------------------------ host side ---

int64_t padded(int64_t N) { return (N + kPadMultiple - 1) / kPadMultiple * kPadMultiple; }

int ensure_pair_buffers(md_ctx *c, int TI, int P) {
  const int D = c->dim;
  size_t need_slots = (size_t)P * 2 * D * TI * sizeof(double);
  if (need_slots > c->sk_slots_bytes) {
    dev_free(c->sk_slots);
    c->sk_slots = (double *)dev_alloc(need_slots);
    if (!c->sk_slots) {
      c->sk_slots_bytes = 0;
      return set_err(c, MD_ENOMEM, "stream-K slots: %zu bytes", need_slots);
    }
    c->sk_slots_bytes = need_slots;
  }
  size_t n_it = (size_t)((c->N + TI - 1) / TI);
  if (n_it > c->sk_tickets_count) {
    dev_free(c->sk_tickets);
    c->sk_tickets = (unsigned *)dev_alloc(n_it * sizeof(unsigned));
    if (!c->sk_tickets) {
      c->sk_tickets_count = 0;
      return set_err(c, MD_ENOMEM, "stream-K tickets");
    }
    c->sk_tickets_count = n_it;
    MD_CUDA(c, cudaMemsetAsync(c->sk_tickets, 0, n_it * sizeof(unsigned), c->stream));
  }
  return MD_OK;
}

int ensure_mirrors(md_ctx *c) {
  const int64_t Np = padded(c->N);
  const size_t per = c->model == MD_RING ? 32 : 16;  // FP64 record size bounds the FP32 one
  const size_t need = (size_t)Np * per;
  if (need > c->mirror_bytes) {
    for (int b = 0; b < 2; b++) {
      dev_free(c->mirror[b]);
      c->mirror[b] = dev_alloc(need);
      if (!c->mirror[b]) {
        c->mirror_bytes = 0;
        return set_err(c, MD_ENOMEM, "mirror: %zu bytes", need);
      }
    }
    c->mirror_bytes = need;
  }
  return MD_OK;
}

template <int MODEL, bool MIXED, int R, int TJ, int MODE>
int launch_pairs(md_ctx *c, double kick, double drift, double *fout) {
  constexpr int64_t TI = (int64_t)NT * R;
  auto kern = pair_stage_kernel<MODEL, MIXED, R, TJ, MODE>;
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, 0);
  if (occ < 1) occ = 1;
  if (c->pt.ctas_per_sm > 0 && c->pt.ctas_per_sm < occ) occ = c->pt.ctas_per_sm;
  PairArgs a;
  a.N = c->N;
  a.n_it = (c->N + TI - 1) / TI;
  a.n_jt = (c->N + TJ - 1) / TJ;
  a.U = a.n_it * a.n_jt;
  int64_t P = (int64_t)c->nsm * occ;
  if (P > a.U) P = a.U;
  a.P = (int)P;
  int rc = ensure_pair_buffers(c, (int)TI, a.P);
  if (rc) return rc;
  a.mirror_in = c->mirror[c->mirror_cur];
  a.mirror_out = c->mirror[1 - c->mirror_cur];
  a.q = c->q;
  a.p = c->p;
  a.scale = MODEL == MD_RING ? -1.0 / (8.0 * (double)c->N) : -2.0 / (double)c->N;
  a.epsd = MODEL == MD_RING ? 0.5 * c->eps : c->eps;
  a.kick = kick;
  a.drift = drift;
  a.slots = c->sk_slots;
  a.tickets = c->sk_tickets;
  a.fout = fout;
  kern<<<a.P, NT, 0, c->stream>>>(a);
  MD_LAUNCHED(c);
  if (MODE == STAGE_KICK_DRIFT) c->mirror_cur = 1 - c->mirror_cur;
  return MD_OK;
}

template <int MODEL, bool MIXED, int MODE>
int dispatch_r(md_ctx *c, double kick, double drift, double *fout) {
  if constexpr (MIXED) {
    switch (c->pt.r_mixed) {
    case 4: return launch_pairs<MODEL, MIXED, 4, 256, MODE>(c, kick, drift, fout);
    default: return launch_pairs<MODEL, MIXED, 8, 256, MODE>(c, kick, drift, fout);
    }
  } else {
    switch (c->pt.r_fp64) {
    case 4: return launch_pairs<MODEL, MIXED, 4, 128, MODE>(c, kick, drift, fout);
    default: return launch_pairs<MODEL, MIXED, 2, 128, MODE>(c, kick, drift, fout);
    }
  }
}

template <int MODEL, bool MIXED>
int dispatch_mode(md_ctx *c, int mode, double kick, double drift, double *fout) {
  switch (mode) {
  case STAGE_KICK_DRIFT: return dispatch_r<MODEL, MIXED, STAGE_KICK_DRIFT>(c, kick, drift, fout);
  case STAGE_KICK_ONLY: return dispatch_r<MODEL, MIXED, STAGE_KICK_ONLY>(c, kick, drift, fout);
  default: return dispatch_r<MODEL, MIXED, STAGE_FORCE_ONLY>(c, kick, drift, fout);
  }
}

}  // namespace

int mirror_refresh(md_ctx *c) {
  int rc = ensure_mirrors(c);
  if (rc) return rc;
  const int64_t Np = padded(c->N);
  const int threads = 256;
  int64_t blocks = std::min<int64_t>((Np + threads - 1) / threads, (int64_t)c->nsm * 16);
  void *m0 = c->mirror[c->mirror_cur], *m1 = c->mirror[1 - c->mirror_cur];
  const bool mixed = c->prec == MD_MIXED;
  if (c->model == MD_RING) {
    if (mixed) mirror_kernel<MD_RING, true><<<blocks, threads, 0, c->stream>>>(c->q, c->N, Np, m0, m1);
    else mirror_kernel<MD_RING, false><<<blocks, threads, 0, c->stream>>>(c->q, c->N, Np, m0, m1);
  } else {
    if (mixed) mirror_kernel<MD_GRAV2D, true><<<blocks, threads, 0, c->stream>>>(c->q, c->N, Np, m0, m1);
    else mirror_kernel<MD_GRAV2D, false><<<blocks, threads, 0, c->stream>>>(c->q, c->N, Np, m0, m1);
  }
  MD_LAUNCHED(c);
  c->mirror_valid = true;
  c->mirror_prec = c->prec;
  return MD_OK;
}

int pair_stage(md_ctx *c, int mode, double kick, double drift, double *fout) {
  if (!c->mirror_valid || c->mirror_prec != c->prec) {
    int rc = mirror_refresh(c);
    if (rc) return rc;
  }
  const bool mixed = c->prec == MD_MIXED;
  if (c->model == MD_RING)
    return mixed ? dispatch_mode<MD_RING, true>(c, mode, kick, drift, fout)
                 : dispatch_mode<MD_RING, false>(c, mode, kick, drift, fout);
  return mixed ? dispatch_mode<MD_GRAV2D, true>(c, mode, kick, drift, fout)
               : dispatch_mode<MD_GRAV2D, false>(c, mode, kick, drift, fout);
}

int kick_drift_cached(md_ctx *c, double kick, double drift) {
  if (!c->mirror_valid || c->mirror_prec != c->prec) {
    int rc = mirror_refresh(c);
    if (rc) return rc;
  }
  const int threads = 256;
  int64_t blocks = std::min<int64_t>((c->N + threads - 1) / threads, (int64_t)c->nsm * 16);
  void *mo = c->mirror[1 - c->mirror_cur];
  const bool mixed = c->prec == MD_MIXED;
  if (c->model == MD_RING) {
    if (mixed) kick_drift_cached_kernel<MD_RING, true><<<blocks, threads, 0, c->stream>>>(c->q, c->p, c->f, c->N, kick, drift, mo);
    else kick_drift_cached_kernel<MD_RING, false><<<blocks, threads, 0, c->stream>>>(c->q, c->p, c->f, c->N, kick, drift, mo);
  } else {
    if (mixed) kick_drift_cached_kernel<MD_GRAV2D, true><<<blocks, threads, 0, c->stream>>>(c->q, c->p, c->f, c->N, kick, drift, mo);
    else kick_drift_cached_kernel<MD_GRAV2D, false><<<blocks, threads, 0, c->stream>>>(c->q, c->p, c->f, c->N, kick, drift, mo);
  }
  MD_LAUNCHED(c);
  c->mirror_cur = 1 - c->mirror_cur;
  return MD_OK;
}
