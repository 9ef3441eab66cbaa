// HMF model (Sec. 3.1): one fused, memory-bound pass per integrator stage.
//
// The force of Eq. 6 needs the magnetization of Eq. 7 of the *current* angles.
// Each stage kernel reads the sums (sum cos, sum sin) that the previous stage
// left behind, and per particle
//     f = cos(theta) My - sin(theta) Mx                  (Eq. 6)
//     p += kick * f ;  theta += drift * p                (Sec. 3 step list)
//     accumulate cos(theta_new), sin(theta_new)          (Eq. 7 for the next stage)
// so the state is read once and written once per stage (32 B per particle).
// The paper stores sin and cos in global memory and reloads them.  The mixed
// path recomputes them instead (FP32 polynomials are cheaper than 32 B more
// traffic); the FP64 path is bound by the FP64 pipe (an FP64 sincos is tens of
// DFMA at 2.3 per SM per clock), so it keeps (cos, sin) of the current angles in
// a buffer, as the paper does, and computes one FP64 sincos per particle-stage
// instead of two.
//
// Consecutive stages sweep the particles in opposite directions: the last part of
// a stage's writes is still in L2 when the next stage starts on it.
//
// Reduction: per-thread sums, warp shuffles and a block tree give one FP64
// partial per CTA; the last CTA to finish (atomic ticket, no waiting) adds the
// partials in CTA order, so the result is deterministic.
#include <math.h>

#include <mutex>

#include "md_internal.cuh"
#include "sincos_fp64.cuh"

namespace {

constexpr int kMaxDevicesTab = 64;

constexpr int NT = kStreamThreads;
constexpr int UNROLL = 2;  // double2 loads of theta and of p in flight per thread
// Mixed sums: a thread adds at most kFlush angles' cosines and sines in FP32 before moving
// them into its FP64 partial, so their rounding does not grow with N / (threads).
constexpr int kFlush = 256;

// ------------------------------------------------ FP64 sine and cosine ------
//
// Table-driven (sincos_fp64.cuh): theta = k pi/2048 + r, a 4096-entry FP64 table of
// (sin, cos)(k pi/2048) in dynamic shared memory (64 KB) of the kernels that use it,
// k and the terms of sin r and cos r below 2^-33 in FP32, 8 FP64 operations per angle;
// |theta| >= 2^20, infinities and NaN use sincos.
constexpr int kTabN = sc64::kTabN;
constexpr int kTabBytes = kTabN * (int)sizeof(double2);

__device__ double2 g_sincos_tab[kTabN];  // (sin, cos)(k pi / 2048), k = 0 .. 4095

__device__ __forceinline__ void sincos_tab(double th, const double2 *__restrict__ tab, double *sp, double *cp) {
  sc64::sincos_tab(th, tab, sp, cp);
}

// The table into shared memory (every thread of the CTA takes part).
__device__ __forceinline__ void load_sincos_tab(double2 *sm) {
  for (int k = threadIdx.x; k < kTabN; k += blockDim.x) sm[k] = g_sincos_tab[k];
  __syncthreads();
}

// c 2^52 rounded to the nearest integer (halves up in magnitude), for |c| <= 1, from
// the bits of c with integer instructions only; 0 for zero, subnormal or non-finite c.
// The FP64 stages add their cosines and sines in this fixed point (exactly, on the
// integer pipe) and move the per-thread sums into FP64 every kFlush angles.
__device__ __forceinline__ long long fix52(double c) {
  const long long b = __double_as_longlong(c);
  const int e = (int)(b >> 52) & 0x7ff;
  const int sh = 1023 - e;  // c 2^52 = significand >> sh
  const long long m = (b & 0x000fffffffffffffLL) | 0x0010000000000000LL;
  const long long v = (sh < 0 || sh > 53) ? 0LL : (m + ((1LL << sh) >> 1)) >> sh;
  return b < 0 ? -v : v;
}

struct HmfArgs {
  double *q, *p;
  int64_t N;
  double invN;
  const double *m_in;  // (sum cos, sum sin) of the current angles
  double kick, drift;
  double *partials;  // 2 per CTA
  double *m_out;     // (sum cos, sum sin) of the new angles
  unsigned *ticket;
  double *fout;  // STAGE_FORCE_ONLY output
  double2 *cs;   // FP64 path: (cos, sin) of the current angles, rewritten by drifts
  int rev;       // sweep the particles from the top end down
  int nsum;      // row shard: m_in holds nsum (sum cos, sum sin) pairs, one per rank
};

// FP64 mean-field force cos(th) My - sin(th) Mx (Eq. 6): one product and one FMA.  A lone
// particle's force, its own self-term, is exactly zero (N = 1: My = sin th, Mx = cos th),
// which the FMA would leave as a rounding residual of the product.
__device__ __forceinline__ double hmf_force_fp64(double c, double s, double mx, double my, double invN) {
  return invN == 1.0 ? 0.0 : fma(c, my, -(s * mx));
}

// One particle of a stage.  MIXED: FP64 state update, FP32 sine/cosine of the
// FP64-range-reduced angle; the new angle's reduced value is carried in FP32.
template <bool MIXED, int MODE>
__device__ __forceinline__ void hmf_particle(double &th, double &pp, const HmfArgs &a, float mxf,
                                             float myf, double mx, double my, float dtf, float &acf,
                                             float &asf, long long &aci, long long &asi, int64_t i,
                                             const double2 *tab) {
  if (MIXED) {
    // Only the kick and the drift use the FP64 pipe (two DFMA per particle):
    // range reduction and float<->double conversions move bits on the integer
    // pipe, and the sines and cosines are FP32 polynomials.
    float r = reduce_2pi_f(th);
    float s, c;
    sincos_small(r, &s, &c);
    float f = __fsub_rn(__fmul_rn(c, myf), __fmul_rn(s, mxf));
    if (MODE == STAGE_FORCE_ONLY) {
      a.fout[i] = f2d_bits(f);
      return;
    }
    pp = fma(a.kick, f2d_bits(f), pp);
    if (MODE == STAGE_KICK_DRIFT) {
      th = fma(a.drift, pp, th);
      float r2 = fmaf(dtf, d2f_trunc_bits(pp), r);
      sincos_small(r2, &s, &c);
      acf += c;
      asf += s;
    }
  } else {
    const double2 cs = a.cs[i];
    const double f = hmf_force_fp64(cs.x, cs.y, mx, my, a.invN);
    if (MODE == STAGE_FORCE_ONLY) {
      a.fout[i] = f;
      return;
    }
    pp = fma(a.kick, f, pp);
    if (MODE == STAGE_KICK_DRIFT) {
      th = fma(a.drift, pp, th);
      double s, c;
      sincos_tab(th, tab, &s, &c);
      a.cs[i] = make_double2(c, s);
      aci += fix52(c);
      asi += fix52(s);
    }
  }
}

// Grid finish: write this CTA's partial; the last CTA sums all partials in order.
__device__ __forceinline__ void grid_finish(double sc, double ss, double *partials, double *m_out,
                                            unsigned *ticket) {
  __shared__ double2 red[NT / 32];
  __shared__ bool last;
  double2 b = block_sum2<NT>(sc, ss, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = b.x;
    partials[2 * blockIdx.x + 1] = b.y;
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double c0 = 0.0, c1 = 0.0;
  for (int j = threadIdx.x; j < (int)gridDim.x; j += NT) {
    c0 += __ldcg(partials + 2 * j);
    c1 += __ldcg(partials + 2 * j + 1);
  }
  __syncthreads();
  double2 t = block_sum2<NT>(c0, c1, red);
  if (threadIdx.x == 0) {
    m_out[0] = t.x;
    m_out[1] = t.y;
    *ticket = 0u;
  }
}

// SHARD: the magnetization is the sum of every rank's pair in m_in, added in rank
// order (the same value on every rank), over the whole system's N (invN).
template <bool MIXED, int MODE, bool SHARD = false>
__global__ void __launch_bounds__(NT) hmf_stage_kernel(HmfArgs a) {
  double sx = a.m_in[0], sy = a.m_in[1];
  if constexpr (SHARD)
    for (int r = 1; r < a.nsum; r++) {
      sx += a.m_in[2 * r];
      sy += a.m_in[2 * r + 1];
    }
  const double mx = sx * a.invN, my = sy * a.invN;
  extern __shared__ double2 tab[];  // FP64 kick-drift stages: the sine/cosine table (kTabBytes)
  if constexpr (!MIXED && MODE == STAGE_KICK_DRIFT) load_sincos_tab(tab);
  const float mxf = (float)mx, myf = (float)my, dtf = (float)a.drift;
  float acf = 0.f, asf = 0.f;
  long long aci = 0, asi = 0;
  double acd = 0.0, asd = 0.0;
  const int64_t npairs = a.N >> 1;
  const int64_t G = (int64_t)gridDim.x * NT;
  const int64_t t0 = (int64_t)blockIdx.x * NT + threadIdx.x;
  double2 *q2 = reinterpret_cast<double2 *>(a.q);
  double2 *p2 = reinterpret_cast<double2 *>(a.p);
  // blocks of kFlush / 2 double2 pairs per thread; the FP32 sums move into FP64 after each
  // block (a counter tested inside the loop instead made the stage a fifth slower)
  const int64_t block = (int64_t)(kFlush / (2 * UNROLL)) * UNROLL * G;
  for (int64_t kb = t0; kb < npairs; kb += block) {
  const int64_t kend = kb + block < npairs ? kb + block : npairs;
  for (int64_t k = kb; k < kend; k += UNROLL * G) {
    double2 qv[UNROLL], pv[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; u++) {
      const int64_t kk = k + u * G;
      const int64_t ix = a.rev ? npairs - 1 - kk : kk;
      if (kk < npairs) {
        qv[u] = q2[ix];
        pv[u] = p2[ix];
      }
    }
#pragma unroll
    for (int u = 0; u < UNROLL; u++) {
      const int64_t kk = k + u * G;
      const int64_t ix = a.rev ? npairs - 1 - kk : kk;
      if (kk < npairs) {
        hmf_particle<MIXED, MODE>(qv[u].x, pv[u].x, a, mxf, myf, mx, my, dtf, acf, asf, aci, asi, 2 * ix, tab);
        hmf_particle<MIXED, MODE>(qv[u].y, pv[u].y, a, mxf, myf, mx, my, dtf, acf, asf, aci, asi, 2 * ix + 1, tab);
        if (MODE == STAGE_KICK_DRIFT) q2[ix] = qv[u];
        if (MODE != STAGE_FORCE_ONLY) p2[ix] = pv[u];
      }
    }
  }
  if constexpr (MIXED && MODE == STAGE_KICK_DRIFT) {
    acd += (double)acf;
    asd += (double)asf;
    acf = asf = 0.f;
  }
  if constexpr (!MIXED && MODE == STAGE_KICK_DRIFT) {
    acd += (double)aci * 0x1p-52;
    asd += (double)asi * 0x1p-52;
    aci = asi = 0;
  }
  }
  if ((a.N & 1) && t0 == 0) {
    int64_t i = a.N - 1;
    double th = a.q[i], pp = a.p[i];
    hmf_particle<MIXED, MODE>(th, pp, a, mxf, myf, mx, my, dtf, acf, asf, aci, asi, i, tab);
    if (MODE == STAGE_KICK_DRIFT) a.q[i] = th;
    if (MODE != STAGE_FORCE_ONLY) a.p[i] = pp;
  }
  if (MODE == STAGE_KICK_DRIFT) {
    if (MIXED) {  // the odd last particle, if any
      acd += (double)acf;
      asd += (double)asf;
    } else {
      acd += (double)aci * 0x1p-52;
      asd += (double)asi * 0x1p-52;
    }
    grid_finish(acd, asd, a.partials, a.m_out, a.ticket);
  }
}

// (sum cos, sum sin) of the given angles.  MIXED: FP32 sine/cosine after FP64
// range reduction, FP32 per-thread sums; otherwise FP64 throughout.
// FP64: use_tab selects the table-driven sine and cosine of the FP64 stages (the table
// in kTabBytes of dynamic shared memory) over sincos; cs_out (may be NULL) also gets
// (cos, sin) of every angle.
template <bool MIXED>
__global__ void __launch_bounds__(NT) hmf_sums_kernel(const double *__restrict__ q, int64_t N,
                                                      double *partials, double *m_out, unsigned *ticket,
                                                      double2 *cs_out, int use_tab) {
  extern __shared__ double2 tab[];
  if (!MIXED && use_tab) load_sincos_tab(tab);  // use_tab is the same for the whole grid
  float acf = 0.f, asf = 0.f;
  double acd = 0.0, asd = 0.0;
  const int64_t G = (int64_t)gridDim.x * NT;
  const int64_t block = (int64_t)kFlush * G;  // kFlush angles per thread, then the FP64 move
  for (int64_t ib = (int64_t)blockIdx.x * NT + threadIdx.x; ib < N; ib += block) {
  const int64_t iend = ib + block < N ? ib + block : N;
  for (int64_t i = ib; i < iend; i += G) {
    double th = q[i];
    if (MIXED) {
      float s, c;
      sincos_small(reduce_2pi_f(th), &s, &c);
      acf += c;
      asf += s;
    } else {
      double s, c;
      if (use_tab)
        sincos_tab(th, tab, &s, &c);
      else
        sincos(th, &s, &c);
      if (cs_out) cs_out[i] = make_double2(c, s);
      acd += c;
      asd += s;
    }
  }
  if (MIXED) {
    acd += (double)acf;
    asd += (double)asf;
    acf = asf = 0.f;
  }
  }
  grid_finish(acd, asd, partials, m_out, ticket);
}

// Grid of a streaming kernel: CTAs per SM = the occupancy limit, or `cap` when
// given (0: none), or the tuning key when set.
int grid_for(md_ctx *c, const void *kern, int64_t work_items, int cap = 0, size_t dyn_smem = 0) {
  int lim = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lim, kern, NT, dyn_smem);
  int occ = (cap > 0 && cap < lim) ? cap : lim;
  if (c->ht.ctas_per_sm > 0) occ = c->ht.ctas_per_sm < lim ? c->ht.ctas_per_sm : lim;
  int64_t g = (int64_t)c->nsm * (occ > 0 ? occ : 1);
  int64_t need = (work_items + NT - 1) / NT;
  if (need < 1) need = 1;
  if (g > need) g = need;
  if (g > c->hmf_grid_max) g = c->hmf_grid_max;
  return (int)g;
}

template <bool MIXED, int MODE>
int launch_stage(md_ctx *c, double kick, double drift, double *fout) {
  HmfArgs a;
  a.q = c->q;
  a.p = c->p;
  a.N = c->N;
  a.invN = 1.0 / (double)c->N;
  a.m_in = c->hmf_m + 2 * c->hmf_cur;
  a.kick = kick;
  a.drift = drift;
  a.partials = c->hmf_partials;
  a.m_out = c->hmf_m + 2 * (1 - c->hmf_cur);
  a.ticket = c->hmf_ticket;
  a.fout = fout;
  a.cs = (double2 *)c->hmf_cs;
  // Consecutive stages sweep the state in opposite directions, so a stage starts on
  // the lines the previous one wrote last, which are still in L2 (dirty lines that
  // are overwritten before eviction are never written back either).
  a.rev = c->hmf_rev;
  a.nsum = 1;
  c->hmf_rev ^= 1;
  auto kern = hmf_stage_kernel<MIXED, MODE>;
  const size_t dyn = (!MIXED && MODE == STAGE_KICK_DRIFT) ? kTabBytes : 0;
  // Mixed stages: 4 CTAs of 256 threads per SM measured fastest on GB300 at N = 5e7
  // (0.252 ms per stage; 0.269 at 3, 0.307 at 2 and 0.271 at 5, the register limit).
  int g = grid_for(c, (const void *)kern, (c->N + 1) / 2 / UNROLL + 1, MIXED ? 4 : 0, dyn);
  kern<<<g, NT, dyn, c->stream>>>(a);
  MD_LAUNCHED(c);
  if (MODE == STAGE_KICK_DRIFT) c->hmf_cur = 1 - c->hmf_cur;
  return MD_OK;
}

}  // namespace

// The sine/cosine table of this device (made on the host in long double, rounded to
// double) and the shared-memory attribute of the kernels that hold it: set up once per
// device, and again if (probe) a read of one entry finds the device copy gone (a device
// reset drops both).  Synchronous; not to be called inside a stream capture.
int hmf_sincos_table(md_ctx *c, bool probe) {
  static std::mutex mu;
  static bool done[kMaxDevicesTab] = {};
  static double2 t[kTabN];
  if (c->device < 0 || c->device >= kMaxDevicesTab) return set_err(c, MD_EINVAL, "device %d", c->device);
  std::lock_guard<std::mutex> lk(mu);
  if (done[c->device]) {
    if (!probe) return MD_OK;
    double2 e1;
    MD_CUDA(c, cudaMemcpyFromSymbol(&e1, g_sincos_tab, sizeof e1, sizeof(double2)));
    if (e1.x == t[1].x && e1.y == t[1].y) return MD_OK;
    done[c->device] = false;
  }
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < kTabN; k++) {
    const long double x = (long double)k * pi / (long double)(kTabN / 2);
    t[k] = make_double2((double)sinl(x), (double)cosl(x));
  }
  MD_CUDA(c, cudaMemcpyToSymbol(g_sincos_tab, t, sizeof t));
  // the kernels that hold the table in dynamic shared memory (64 KB, above the 48 KB default)
  MD_CUDA(c, cudaFuncSetAttribute(hmf_stage_kernel<false, STAGE_KICK_DRIFT, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kTabBytes));
  MD_CUDA(c, cudaFuncSetAttribute(hmf_stage_kernel<false, STAGE_KICK_DRIFT, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kTabBytes));
  MD_CUDA(c, cudaFuncSetAttribute(hmf_sums_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTabBytes));
  done[c->device] = true;
  return MD_OK;
}

// FP64 (sum cos, sum sin) of q[0..N) into device out2, with caller-supplied
// partials (>= grid_cap doubles x 2) and a zeroed ticket.
void hmf_sums_raw(cudaStream_t st, int nsm, int grid_cap, const double *q, int64_t N, double *partials,
                  double *out2, unsigned *ticket) {
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hmf_sums_kernel<false>, NT, 0);
  int64_t g = (int64_t)nsm * (occ > 0 ? occ : 1);
  const int64_t need = (N + NT - 1) / NT;
  if (g > need) g = need;
  if (g > grid_cap) g = grid_cap;
  if (g < 1) g = 1;
  hmf_sums_kernel<false><<<(int)g, NT, 0, st>>>(q, N, partials, out2, ticket, nullptr, 0);
}

int hmf_sums_fp64_of(md_ctx *c, const double *q, double *d_out2) {
  int rc = hmf_sincos_table(c, false);  // HMF contexts have it already; Ring ones (md_magnetization) may not
  if (rc) return rc;
  auto kern = hmf_sums_kernel<false>;
  int g = grid_for(c, (const void *)kern, c->N, 0, kTabBytes);
  kern<<<g, NT, kTabBytes, c->stream>>>(q, c->N, c->hmf_partials, d_out2, c->hmf_ticket, nullptr, 1);
  MD_LAUNCHED(c);
  return MD_OK;
}

int hmf_sums_fp64(md_ctx *c, double *d_out2) { return hmf_sums_fp64_of(c, c->q, d_out2); }

// Sums of the current angles into the current magnetization slot.
int hmf_prime(md_ctx *c) {
  double *out = c->hmf_m + 2 * c->hmf_cur;
  if (c->prec == MD_MIXED) {
    auto kern = hmf_sums_kernel<true>;
    int g = grid_for(c, (const void *)kern, c->N);
    kern<<<g, NT, 0, c->stream>>>(c->q, c->N, c->hmf_partials, out, c->hmf_ticket, nullptr, 0);
    MD_LAUNCHED(c);
  } else {
    // FP64: the sums and the (cos, sin) buffer the FP64 stages read
    const size_t need = sizeof(double2) * (size_t)c->N;
    if (need > c->hmf_cs_bytes) {
      dev_free(c->hmf_cs);
      c->hmf_cs = (double *)dev_alloc(need);
      c->hmf_cs_bytes = c->hmf_cs ? need : 0;
      if (!c->hmf_cs) return set_err(c, MD_ENOMEM, "HMF (cos, sin) buffer: %zu bytes", need);
    }
    auto kern = hmf_sums_kernel<false>;
    int g = grid_for(c, (const void *)kern, c->N, 0, kTabBytes);
    kern<<<g, NT, kTabBytes, c->stream>>>(c->q, c->N, c->hmf_partials, out, c->hmf_ticket, (double2 *)c->hmf_cs, 1);
    MD_LAUNCHED(c);
  }
  c->hmf_m_valid = true;
  c->hmf_m_prec = c->prec;
  return MD_OK;
}

// ------------------------------------------------------------ row shards ---
//
// A row shard (md_shard_*) holds rows [row0, row0 + N) of a system of n_total
// particles.  Its stages read the magnetization from every rank's partial sums
// (shard_sums[cur][rank], in rank order) and write the sums of their own new angles
// to shard_sums[1 - cur][rank]; the exchange between stages copies the other ranks'
// pairs in (Sec. 3.1, last paragraph: partial magnetizations per GPU, summed).

int hmf_shard_prime(md_ctx *c) {
  const size_t sums_bytes = sizeof(double) * 4 * (size_t)c->shard_nranks;
  if (!c->shard_sums) {
    c->shard_sums = (double *)dev_alloc(sums_bytes);
    if (!c->shard_sums) return set_err(c, MD_ENOMEM, "HMF shard sums: %zu bytes", sums_bytes);
  }
  MD_CUDA(c, cudaMemsetAsync(c->shard_sums, 0, sums_bytes, c->stream));
  c->shard_cur = 0;
  double *out = c->shard_sums + 2 * c->shard_rank;
  if (c->prec == MD_MIXED) {
    auto kern = hmf_sums_kernel<true>;
    int g = grid_for(c, (const void *)kern, c->N);
    kern<<<g, NT, 0, c->stream>>>(c->q, c->N, c->hmf_partials, out, c->hmf_ticket, nullptr, 0);
  } else {
    const size_t need = sizeof(double2) * (size_t)c->N;
    if (need > c->hmf_cs_bytes) {
      dev_free(c->hmf_cs);
      c->hmf_cs = (double *)dev_alloc(need);
      c->hmf_cs_bytes = c->hmf_cs ? need : 0;
      if (!c->hmf_cs) return set_err(c, MD_ENOMEM, "HMF (cos, sin) buffer: %zu bytes", need);
    }
    auto kern = hmf_sums_kernel<false>;
    int g = grid_for(c, (const void *)kern, c->N, 0, kTabBytes);
    kern<<<g, NT, kTabBytes, c->stream>>>(c->q, c->N, c->hmf_partials, out, c->hmf_ticket, (double2 *)c->hmf_cs, 1);
  }
  MD_LAUNCHED(c);
  c->hmf_m_valid = false;  // md_step's own sums are not kept on a shard
  return MD_OK;
}

namespace {
template <bool MIXED, int MODE>
int launch_shard_stage(md_ctx *c, double kick, double drift, double *fout) {
  const int P = c->shard_nranks;
  HmfArgs a;
  a.q = c->q;
  a.p = c->p;
  a.N = c->N;
  a.invN = 1.0 / (double)c->n_total;
  a.m_in = c->shard_sums + 2 * P * c->shard_cur;
  a.nsum = P;
  a.kick = kick;
  a.drift = drift;
  a.partials = c->hmf_partials;
  a.m_out = c->shard_sums + 2 * (P * (1 - c->shard_cur) + c->shard_rank);
  a.ticket = c->hmf_ticket;
  a.fout = fout;
  a.cs = (double2 *)c->hmf_cs;
  a.rev = c->hmf_rev;
  c->hmf_rev ^= 1;
  auto kern = hmf_stage_kernel<MIXED, MODE, true>;
  const size_t dyn = (!MIXED && MODE == STAGE_KICK_DRIFT) ? kTabBytes : 0;
  int g = grid_for(c, (const void *)kern, (c->N + 1) / 2 / UNROLL + 1, MIXED ? 4 : 0, dyn);
  kern<<<g, NT, dyn, c->stream>>>(a);
  MD_LAUNCHED(c);
  if (MODE == STAGE_KICK_DRIFT) c->shard_cur = 1 - c->shard_cur;
  return MD_OK;
}
}  // namespace

int hmf_shard_stage(md_ctx *c, int mode, double kick, double drift, double *fout) {
  const bool mixed = c->prec == MD_MIXED;
  if (mode == STAGE_FORCE_ONLY)
    return mixed ? launch_shard_stage<true, STAGE_FORCE_ONLY>(c, 0.0, 0.0, fout)
                 : launch_shard_stage<false, STAGE_FORCE_ONLY>(c, 0.0, 0.0, fout);
  return mixed ? launch_shard_stage<true, STAGE_KICK_DRIFT>(c, kick, drift, nullptr)
               : launch_shard_stage<false, STAGE_KICK_DRIFT>(c, kick, drift, nullptr);
}

int hmf_stage(md_ctx *c, int mode, double kick, double drift, double *fout) {
  if (!c->hmf_m_valid || c->hmf_m_prec != c->prec) {
    int rc = hmf_prime(c);
    if (rc) return rc;
  }
  const bool mixed = c->prec == MD_MIXED;
  switch (mode) {
  case STAGE_KICK_DRIFT:
    return mixed ? launch_stage<true, STAGE_KICK_DRIFT>(c, kick, drift, fout)
                 : launch_stage<false, STAGE_KICK_DRIFT>(c, kick, drift, fout);
  case STAGE_KICK_ONLY:
    return mixed ? launch_stage<true, STAGE_KICK_ONLY>(c, kick, drift, fout)
                 : launch_stage<false, STAGE_KICK_ONLY>(c, kick, drift, fout);
  default:
    return mixed ? launch_stage<true, STAGE_FORCE_ONLY>(c, kick, drift, fout)
                 : launch_stage<false, STAGE_FORCE_ONLY>(c, kick, drift, fout);
  }
}

// ---------------------------------------------------------------- adjoint --
//
// Reverse stages of md_grad for HMF.  With Eqs. 6-7, J = df/dtheta gives
//   (J v)_i = -(sin t_i My + cos t_i Mx) v_i + cos t_i A + sin t_i B,
//   A = (1/N) sum cos t_k v_k,  B = (1/N) sum sin t_k v_k,
// so each reverse stage needs the four sums (sum cos, sum sin, sum cos v,
// sum sin v) of the current angles and lambda_p, which the previous reverse
// stage leaves behind (same deterministic grid finish as the forward).

namespace {

struct HmfAdjArgs {
  double *q, *p, *lq, *lp;
  int64_t N;
  double invN;
  const double *s_in;  // 4 sums of the current (theta, lambda_p)
  double b_adj, b_undo, drift;
  double *partials;  // 4 per CTA
  double *s_out;
  unsigned *ticket;
};

__device__ __forceinline__ void grid_finish4(double v0, double v1, double v2, double v3, double *partials,
                                             double *out, unsigned *ticket) {
  __shared__ double2 red[NT / 32];
  __shared__ bool last;
  double2 b01 = block_sum2<NT>(v0, v1, red);
  __syncthreads();
  double2 b23 = block_sum2<NT>(v2, v3, red);
  if (threadIdx.x == 0) {
    partials[4 * blockIdx.x] = b01.x;
    partials[4 * blockIdx.x + 1] = b01.y;
    partials[4 * blockIdx.x + 2] = b23.x;
    partials[4 * blockIdx.x + 3] = b23.y;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double c[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < (int)gridDim.x; j += NT)
#pragma unroll
    for (int k = 0; k < 4; k++) c[k] += __ldcg(partials + 4 * j + k);
  __syncthreads();
  double2 t01 = block_sum2<NT>(c[0], c[1], red);
  __syncthreads();
  double2 t23 = block_sum2<NT>(c[2], c[3], red);
  if (threadIdx.x == 0) {
    out[0] = t01.x;
    out[1] = t01.y;
    out[2] = t23.x;
    out[3] = t23.y;
    *ticket = 0u;
  }
}

template <bool MIXED>
__device__ __forceinline__ void sc_of(double th, double &s, double &c) {
  if (MIXED) {
    float sf, cf;
    sincos_small(reduce_2pi_f(th), &sf, &cf);
    s = f2d_bits(sf);
    c = f2d_bits(cf);
  } else {
    sincos(th, &s, &c);
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(NT) hmf_adj_sums_kernel(const double *__restrict__ q, const double *__restrict__ lp,
                                                          int64_t N, double *partials, double *out, unsigned *ticket) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  const int64_t G = (int64_t)gridDim.x * NT;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < N; i += G) {
    double s, c;
    sc_of<MIXED>(q[i], s, c);
    const double v = lp[i];
    a0 += c;
    a1 += s;
    a2 = fma(c, v, a2);
    a3 = fma(s, v, a3);
  }
  grid_finish4(a0, a1, a2, a3, partials, out, ticket);
}

template <bool MIXED>
__global__ void __launch_bounds__(NT) hmf_adj_stage_kernel(HmfAdjArgs a) {
  const double mx = a.s_in[0] * a.invN, my = a.s_in[1] * a.invN;
  const double A = a.s_in[2] * a.invN, B = a.s_in[3] * a.invN;
  const float mxf = (float)mx, myf = (float)my;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  const int64_t G = (int64_t)gridDim.x * NT;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.N; i += G) {
    double th = a.q[i], pp = a.p[i], lq = a.lq[i], lp = a.lp[i];
    double s, c, f;
    sc_of<MIXED>(th, s, c);
    if (MIXED)  // the same FP32 force as the forward stage, so the reversal undoes it
      f = f2d_bits(__fsub_rn(__fmul_rn((float)c, myf), __fmul_rn((float)s, mxf)));
    else
      f = hmf_force_fp64(c, s, mx, my, a.invN);
    const double jv = fma(-fma(s, my, c * mx), lp, fma(c, A, s * B));
    lq = fma(a.b_adj, jv, lq);
    pp = fma(-a.b_undo, f, pp);
    if (a.drift != 0.0) {
      lp = fma(a.drift, lq, lp);
      th = fma(-a.drift, pp, th);
      sc_of<MIXED>(th, s, c);
      a0 += c;
      a1 += s;
      a2 = fma(c, lp, a2);
      a3 = fma(s, lp, a3);
      a.q[i] = th;
      a.lp[i] = lp;
    }
    a.p[i] = pp;
    a.lq[i] = lq;
  }
  if (a.drift != 0.0) grid_finish4(a0, a1, a2, a3, a.partials, a.s_out, a.ticket);
}

// lambda_q of the |M| observable: d|M|/dtheta_i = (My cos t_i - Mx sin t_i) / (N |M|).
__global__ void hmf_mag_terminal_kernel(const double *__restrict__ q, int64_t N, double cx, double cy,
                                        double *__restrict__ lq) {
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += G) {
    double s, c;
    sincos(q[i], &s, &c);
    lq[i] = fma(cx, c, -cy * s);
  }
}

}  // namespace

// Four sums of the current (theta, lambda_p) into the current adjoint slot.
int hmf_adjoint_prime(md_ctx *c, const double *lp, double *sums) {
  const int g = grid_for(c, (const void *)hmf_adj_sums_kernel<true>, c->N);
  if (c->prec == MD_MIXED)
    hmf_adj_sums_kernel<true><<<g, NT, 0, c->stream>>>(c->q, lp, c->N, c->hmf_partials, sums, c->hmf_ticket);
  else
    hmf_adj_sums_kernel<false><<<g, NT, 0, c->stream>>>(c->q, lp, c->N, c->hmf_partials, sums, c->hmf_ticket);
  MD_LAUNCHED(c);
  return MD_OK;
}

int hmf_adjoint_stage(md_ctx *c, double b_adj, double b_undo, double drift, double *lq, double *lp,
                      const double *s_in, double *s_out) {
  HmfAdjArgs a;
  a.q = c->q;
  a.p = c->p;
  a.lq = lq;
  a.lp = lp;
  a.N = c->N;
  a.invN = 1.0 / (double)c->N;
  a.s_in = s_in;
  a.b_adj = b_adj;
  a.b_undo = b_undo;
  a.drift = drift;
  a.partials = c->hmf_partials;
  a.s_out = s_out;
  a.ticket = c->hmf_ticket;
  const int g = grid_for(c, (const void *)hmf_adj_stage_kernel<false>, c->N);
  if (c->prec == MD_MIXED)
    hmf_adj_stage_kernel<true><<<g, NT, 0, c->stream>>>(a);
  else
    hmf_adj_stage_kernel<false><<<g, NT, 0, c->stream>>>(a);
  MD_LAUNCHED(c);
  return MD_OK;
}

int hmf_magnetization_terminal(md_ctx *c, double cx, double cy, double *lq) {
  int64_t b = (c->N + 255) / 256;
  if (b > (int64_t)c->nsm * 16) b = (int64_t)c->nsm * 16;
  hmf_mag_terminal_kernel<<<(int)b, 256, 0, c->stream>>>(c->q, c->N, cx, cy, lq);
  MD_LAUNCHED(c);
  return MD_OK;
}

// ---------------------------------------------------------------- tangent --
//
// Forward tangent (linearised) dynamics for HMF:  p += kick f, dp += kick J dq,
// then theta += drift p, dq += drift dp, with (J dq)_i from the four sums of the
// current (theta, dq) as in the adjoint above.

namespace {

template <bool MIXED>
__global__ void __launch_bounds__(NT) hmf_tangent_stage_kernel(HmfAdjArgs a) {
  const double mx = a.s_in[0] * a.invN, my = a.s_in[1] * a.invN;
  const double A = a.s_in[2] * a.invN, B = a.s_in[3] * a.invN;
  const float mxf = (float)mx, myf = (float)my;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  const int64_t G = (int64_t)gridDim.x * NT;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.N; i += G) {
    double th = a.q[i], pp = a.p[i], dq = a.lq[i], dp = a.lp[i];
    double s, c, f;
    sc_of<MIXED>(th, s, c);
    if (MIXED)
      f = f2d_bits(__fsub_rn(__fmul_rn((float)c, myf), __fmul_rn((float)s, mxf)));
    else
      f = hmf_force_fp64(c, s, mx, my, a.invN);
    const double jv = fma(-fma(s, my, c * mx), dq, fma(c, A, s * B));
    pp = fma(a.b_adj, f, pp);
    dp = fma(a.b_adj, jv, dp);
    if (a.drift != 0.0) {
      th = fma(a.drift, pp, th);
      dq = fma(a.drift, dp, dq);
      sc_of<MIXED>(th, s, c);
      a0 += c;
      a1 += s;
      a2 = fma(c, dq, a2);
      a3 = fma(s, dq, a3);
      a.q[i] = th;
      a.lq[i] = dq;
    }
    a.p[i] = pp;
    a.lp[i] = dp;
  }
  if (a.drift != 0.0) grid_finish4(a0, a1, a2, a3, a.partials, a.s_out, a.ticket);
}

}  // namespace

int hmf_tangent_stage(md_ctx *c, double kick, double drift, double *dq, double *dp, const double *s_in,
                      double *s_out) {
  HmfAdjArgs a;
  a.q = c->q;
  a.p = c->p;
  a.lq = dq;
  a.lp = dp;
  a.N = c->N;
  a.invN = 1.0 / (double)c->N;
  a.s_in = s_in;
  a.b_adj = kick;
  a.b_undo = 0.0;
  a.drift = drift;
  a.partials = c->hmf_partials;
  a.s_out = s_out;
  a.ticket = c->hmf_ticket;
  const int g = grid_for(c, (const void *)hmf_tangent_stage_kernel<false>, c->N);
  if (c->prec == MD_MIXED)
    hmf_tangent_stage_kernel<true><<<g, NT, 0, c->stream>>>(a);
  else
    hmf_tangent_stage_kernel<false><<<g, NT, 0, c->stream>>>(a);
  MD_LAUNCHED(c);
  return MD_OK;
}
