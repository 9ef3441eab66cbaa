// Batched ensembles of independent Ring / 2D systems of uneven N.
//
// Each integrator stage of every system in the ensemble is one persistent
// launch.  The grid is split into a Ring part and a 2D part (the two models
// have different pair arithmetic); within a part, the (system, i-tile, j-tile)
// units of all its systems form one linear range that is split stream-K style
// across the part's CTAs, so every CTA does the same number of pair
// interactions whatever the spread of N (work per system grows as N^2).  Rows
// (i-tiles) covered by several CTAs are finished by the last contributor, as
// in the single-system kernel.  The Ring/2D split, the register blocking R and
// the CTAs per SM are chosen by md_batch_autotune, which times candidate
// configurations on force-only launches (state untouched).  md_batch_step
// replays a CUDA graph holding a block of steps.
//
// Mixed precision runs, by default, the Newton's-third-law form of each part
// (every unordered pair of a system once, as the single-system stages in
// sym.cu): one pair launch per part, each over the whole GPU, walking the
// triangular (system, i-tile, j-tile) units of its systems stream-K style and
// writing row and column partials (diagonal units too: their above-diagonal
// blocks are evaluated once, with column sums), then one finish launch with a CTA
// per (system, tile, chunk of column-partial rows: 128 for the Ring part's
// 256-output tiles, 32 for the 2D part's 2048) that sums them in a fixed order and
// runs the epilogue; the grid holds only the chunks each tile has (tile t sums the
// rows 0 .. t, ceil((t + 1) / chunk) chunks).  (The one-sided form shares one launch
// between the parts, split by md_batch_set_tuning's `split`.)
#include <algorithm>
#include <vector>

#include "pairs_impl.cuh"

namespace {

constexpr int kGraphSteps = 10;  // even: three mirror flips per step keep the parity
// Record bytes of the systems one wave of the Newton's-third-law pair phase works on.
constexpr int64_t kWaveRecordBytes = 32ll << 20;
// Virtual CTAs per CTA of the Newton's-third-law pair phase, at least (2 measured 0.4%
// faster than 4 and 2% faster than 3 on the 256-system mix).
constexpr int kMinWaves = 2;

struct SysDesc {
  double *q, *p, *f;
  const unsigned char *mir[2];
  int64_t N, n_it, n_jt;
  int64_t ubeg;  // first unit of the system in its part
  int64_t rbeg;  // first row (i-tile) of the system in its part
  int64_t fbeg;  // symmetric form: first finish CTA of the system in its part
  int64_t nfin;  // symmetric form: finish CTAs of the system (chunks of all its tiles)
  double epsd, dt;
};

struct PartArgs {
  const SysDesc *sys;
  int nsys;
  int64_t U;
  int P;
  int cur;
  double b, d;
  double *slots;
  unsigned *tickets;
  // symmetric form
  int waves;         // virtual CTAs per physical CTA: P = waves x grid
  unsigned *next;    // next virtual CTA to take (the finish kernel sets it back to 0)
  int m;             // TI / TJ of the part
  int64_t nfin;      // finish CTAs of the part
  double *rowfull;   // [rows][NACC][TI]
  float *colslot;    // [U][TJ][NACC]
  double *chunks;    // [nfin][TI][NACC]
};

// index of the system whose unit range holds u (binary search on ubeg)
__device__ __forceinline__ int sys_of_unit(const PartArgs &A, int64_t u) {
  int lo = 0, hi = A.nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (A.sys[mid].ubeg <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int64_t row_of_unit(const PartArgs &A, int64_t u) {
  const SysDesc &S = A.sys[sys_of_unit(A, u)];
  return S.rbeg + (u - S.ubeg) / S.n_jt;
}

__device__ __forceinline__ PairArgs view(const PartArgs &A, const SysDesc &S) {
  PairArgs v{};
  v.mirror_in = S.mir[A.cur];
  v.mirror_out = (void *)S.mir[1 - A.cur];
  v.q = S.q;
  v.p = S.p;
  v.fout = S.f;
  v.N = S.N;
  v.epsd = S.epsd;
  v.kick = A.b * S.dt;
  v.drift = A.d * S.dt;
  return v;
}

// Not inlined: the Ring and 2D parts then get separate register allocations.
template <class Pol, int MODEL, bool MIXED, int MODE>
__device__ __noinline__ void batch_part(const PartArgs &A, int64_t cta) {
  constexpr int R = Pol::R, TJ = Pol::TJ, NACC = Pol::NACC;
  constexpr int TILE_BYTES = TJ * Pol::JB;
  constexpr int CHUNKS = TILE_BYTES / 16;
  constexpr int64_t TI = (int64_t)NT * R;
  __shared__ __align__(16) unsigned char sbuf[2][TILE_BYTES];
  __shared__ bool s_last;

  const int64_t u0 = unit_begin(A.U, A.P, cta), u1 = unit_begin(A.U, A.P, cta + 1);
  if (u0 >= u1) return;
  const int64_t first_row = row_of_unit(A, u0);
  int s = sys_of_unit(A, u0);
  int64_t it = (u0 - A.sys[s].ubeg) / A.sys[s].n_jt, jt = (u0 - A.sys[s].ubeg) % A.sys[s].n_jt;
  bool row_from_start = (jt == 0);

  auto prefetch = [&](int buf, int sp, int64_t jtp) {
    const unsigned char *src = A.sys[sp].mir[A.cur] + jtp * (int64_t)TILE_BYTES;
    for (int ch = threadIdx.x; ch < CHUNKS; ch += NT) cp_async16(&sbuf[buf][ch * 16], src + ch * 16);
    cp_async_commit();
  };

  typename Pol::State st;
  PairArgs v = view(A, A.sys[s]);
  int64_t i0 = it * TI;  // tile base; each thread's rows come from Pol::row_of
  Pol::load(st, v.mirror_in, i0);
  prefetch(0, s, jt);

  for (int64_t u = u0; u < u1; u++) {
    const int buf = (int)((u - u0) & 1);
    if (u + 1 < u1) {
      int sn = s;
      int64_t jn = jt + 1;
      if (jn == A.sys[s].n_jt) {
        jn = 0;
        if (it + 1 == A.sys[s].n_it) sn = s + 1;
      }
      prefetch(buf ^ 1, sn, jn);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int64_t j0 = jt * TJ;
    const bool diag = Pol::MASK && (j0 < it * TI + TI) && (it * TI < j0 + TJ);
    if (diag)
      Pol::template tile<true>(st, sbuf[buf], v, i0, j0);
    else
      Pol::template tile<false>(st, sbuf[buf], v, i0, j0);
    __syncthreads();
    jt++;
    const bool row_end = (jt == A.sys[s].n_jt);
    if (row_end || u + 1 == u1) {
      const int64_t row = A.sys[s].rbeg + it;
      if (row_end && row_from_start) {
#pragma unroll
        for (int r = 0; r < Pol::NR; r++) {
          double ex[NACC];
          Pol::total(st, r, ex);
          const int lr = Pol::row_of(r);  // row offset in the tile, -1: another lane's
          if (lr >= 0) finish<Pol, MODEL, MIXED, MODE>(v, i0 + lr, ex);
        }
      } else {
        const int slot = (row == first_row) ? 0 : 1;
        double *sp = A.slots + ((cta * 2 + slot) * NACC) * TI;
#pragma unroll
        for (int r = 0; r < Pol::NR; r++) {
          double ex[NACC];
          Pol::total(st, r, ex);
          const int lr = Pol::row_of(r);  // row offset in the tile, -1: another lane's
          if (lr >= 0)
#pragma unroll
            for (int d = 0; d < NACC; d++) sp[d * TI + lr] = ex[d];
        }
        __threadfence();
        __syncthreads();
        const int64_t ub = A.sys[s].ubeg + it * A.sys[s].n_jt;
        const int64_t cf = cta_of_unit(A.U, A.P, ub);
        const int64_t cl = cta_of_unit(A.U, A.P, ub + A.sys[s].n_jt - 1);
        if (threadIdx.x == 0) {
          unsigned cnt = atomicAdd(&A.tickets[row], 1u) + 1u;
          s_last = (cnt == (unsigned)(cl - cf + 1));
        }
        __syncthreads();
        if (s_last) {
          __threadfence();
          double tot[Pol::NR][NACC];
#pragma unroll
          for (int r = 0; r < Pol::NR; r++)
#pragma unroll
            for (int d = 0; d < NACC; d++) tot[r][d] = 0.0;
          for (int64_t c2 = cf; c2 <= cl; c2++) {
            const int sl = (row == row_of_unit(A, unit_begin(A.U, A.P, c2))) ? 0 : 1;
            const double *src = A.slots + ((c2 * 2 + sl) * NACC) * TI;
#pragma unroll
            for (int r = 0; r < Pol::NR; r++) {
              const int lr = Pol::row_of(r);  // row offset in the tile, -1: another lane's
              if (lr >= 0)
#pragma unroll
                for (int d = 0; d < NACC; d++) tot[r][d] += __ldcg(src + d * TI + lr);
            }
          }
#pragma unroll
          for (int r = 0; r < Pol::NR; r++) {
            const int lr = Pol::row_of(r);  // row offset in the tile, -1: another lane's
            if (lr >= 0) finish<Pol, MODEL, MIXED, MODE>(v, i0 + lr, tot[r]);
          }
          if (threadIdx.x == 0) A.tickets[row] = 0u;
        }
      }
      if (row_end && u + 1 < u1) {
        it++;
        jt = 0;
        row_from_start = true;
        if (it == A.sys[s].n_it) {
          s++;
          it = 0;
          v = view(A, A.sys[s]);
        }
        i0 = it * TI;
        Pol::load(st, v.mirror_in, i0);
      }
    }
  }
}

template <class PolR, class PolG, bool MIXED, int MODE>
__global__ void __launch_bounds__(NT) batch_kernel(PartArgs ring, PartArgs grav) {
  if ((int)blockIdx.x < ring.P)
    batch_part<PolR, MD_RING, MIXED, MODE>(ring, blockIdx.x);
  else
    batch_part<PolG, MD_GRAV2D, MIXED, MODE>(grav, (int64_t)blockIdx.x - ring.P);
}

// ------------------------------------------------- Newton's-third-law form --

constexpr int kFinishThreadsB = 256;

// Column-partial rows per finish CTA, by the tile's outputs (TI NACC): longer chunks
// where a CTA has fewer outputs to sum, twice the single-system finish's, as the
// ensemble's tiles have few rows above them (small systems) and the finish phase is
// bound by its CTA count rather than by its loads.
__host__ __device__ constexpr int chunk_rows(int64_t outputs) { return outputs <= 256 ? 128 : outputs <= 512 ? 64 : 32; }

// Finish CTAs: tile t sums the column partials of its units (I, t m .. t m + m - 1)
// for I = 0 .. t (its own diagonal units included: their above-diagonal blocks) in
// ceil((t + 1) / ch) chunks of ch rows I.  CTAs of tiles 0 .. T-1:
// sum_{s=1}^{T} ceil(s / ch) = ch q (q + 1) / 2 + r (q + 1) with T = q ch + r.
__host__ __device__ __forceinline__ int64_t fin_prefix(int64_t T, int ch) {
  const int64_t q = T / ch, r = T % ch;
  return (int64_t)ch * q * (q + 1) / 2 + r * (q + 1);
}

// The tile whose chunks hold finish CTA f of a system of n_it tiles: the largest T
// with fin_prefix(T) <= f.
__device__ __forceinline__ int64_t fin_tile(int64_t f, int64_t n_it, int ch) {
  int64_t lo = 0, hi = n_it - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (fin_prefix(mid, ch) <= f) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// (system, local row) of part-local unit u in the triangular layout
__device__ __forceinline__ void sym_locate(const PartArgs &A, int64_t u, int &s, int64_t &it, int64_t &jt) {
  s = sys_of_unit(A, u);
  const SysDesc &S = A.sys[s];
  const int64_t lu = u - S.ubeg;
  it = sym_row_of_unit(lu, S.n_it, S.n_jt, A.m);
  jt = (int64_t)A.m * it + (lu - sym_rowstart(it, S.n_jt, A.m));
}

// Pair phase of one part: the part's CTAs walk its triangular units (systems
// one after the other), write the row partials of the rows they cover and the
// column partial of every unit (a diagonal unit's: the sums of its above-diagonal
// blocks, Pol::tile_diag, which evaluates each unordered pair of the tile's own
// particles once, off the 16 x 16 (Ring) or 256 x 256 (2D) squares on the
// diagonal).  smem: the j-tile double buffer, then the per-warp column sums.
template <class Pol>
__device__ __forceinline__ void batch_sym_pairs(const PartArgs &A, int64_t cta, unsigned char *smem) {
  constexpr int TJ = Pol::TJ, NACC = Pol::NACC, NW = NT / 32;
  constexpr int TILE_BYTES = TJ * Pol::JB;
  constexpr int CHUNKS = TILE_BYTES / 16;
  constexpr int64_t TI = (int64_t)NT * Pol::R;
  unsigned char *sbuf0 = smem, *sbuf1 = smem + TILE_BYTES;
  float *colsm = (float *)(smem + 2 * TILE_BYTES);
  const int64_t u0 = unit_begin(A.U, A.P, cta), u1 = unit_begin(A.U, A.P, cta + 1);
  if (u0 >= u1) return;
  const int m = A.m;
  int s;
  int64_t it, jt;
  sym_locate(A, u0, s, it, jt);
  const int64_t first_row = A.sys[s].rbeg + it;
  bool row_from_start = (jt == (int64_t)m * it);
  auto prefetch = [&](unsigned char *buf, int sp, int64_t jtp) {
    const unsigned char *src = A.sys[sp].mir[A.cur] + jtp * (int64_t)TILE_BYTES;
    for (int ch = threadIdx.x; ch < CHUNKS; ch += NT) cp_async16(buf + ch * 16, src + ch * 16);
    cp_async_commit();
  };
  typename Pol::State st;
  PairArgs v = view(A, A.sys[s]);
  int64_t i0 = it * TI;
  Pol::load(st, v.mirror_in, i0);
  prefetch(sbuf0, s, jt);
  for (int64_t u = u0; u < u1; u++) {
    unsigned char *buf = ((u - u0) & 1) ? sbuf1 : sbuf0;
    const SysDesc &S = A.sys[s];
    const bool row_end = (jt + 1 == S.n_jt);
    const bool sys_end = row_end && (it + 1 == S.n_it);
    const int s_next = sys_end ? s + 1 : s;
    const int64_t jt_next = sys_end ? 0 : row_end ? (int64_t)m * (it + 1) : jt + 1;
    if (u + 1 < u1) {
      prefetch(((u - u0) & 1) ? sbuf0 : sbuf1, s_next, jt_next);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const bool diag = jt < (int64_t)m * (it + 1);
    if (diag) Pol::tile_diag(st, buf, v, colsm, (int)(jt - (int64_t)m * it));
    else Pol::tile_sym(st, buf, v, colsm);
    __syncthreads();
    {
      float *dst = A.colslot + u * (int64_t)(TJ * NACC);
      for (int idx = threadIdx.x; idx < TJ * NACC; idx += NT) {
        float x = colsm[idx];
#pragma unroll
        for (int w = 1; w < NW; w++) x += colsm[w * TJ * NACC + idx];
        dst[idx] = x;
      }
    }
    if (row_end || u + 1 == u1) {
      const int64_t row = S.rbeg + it;
      double *sp = (row_end && row_from_start) ? A.rowfull + row * NACC * TI
                                               : A.slots + ((cta * 2 + (row == first_row ? 0 : 1)) * NACC) * TI;
#pragma unroll
      for (int r = 0; r < Pol::NR; r++) {
        double ex[NACC];
        Pol::total(st, r, ex);
        const int lr = Pol::row_of(r);  // row offset in the tile, -1: another lane's
        if (lr >= 0)
#pragma unroll
          for (int d = 0; d < NACC; d++) sp[d * TI + lr] = ex[d];
      }
      if (row_end && u + 1 < u1) {
        row_from_start = true;
        if (sys_end) {
          s++;
          it = 0;
          v = view(A, A.sys[s]);
        } else {
          it++;
        }
        i0 = it * TI;
        Pol::load(st, v.mirror_in, i0);
      }
    }
    jt = jt_next;
  }
}

// index of the system whose finish-CTA range holds f (binary search on fbeg)
__device__ __forceinline__ int sys_of_fin(const PartArgs &A, int64_t f) {
  int lo = 0, hi = A.nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (A.sys[mid].fbeg <= f) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Finish phase of one part, CTA f: chunk c of tile T of system s (as in sym.cu).
template <class Pol, int MODEL, int MODE>
__device__ __noinline__ void batch_sym_finish(const PartArgs &A, int64_t f) {
  constexpr int NACC = Pol::NACC, TJ = Pol::TJ;
  constexpr int64_t TI = (int64_t)NT * Pol::R;
  constexpr int OUT = (int)TI * NACC;
  __shared__ bool s_last;
  constexpr int CH = chunk_rows(OUT);
  const int s = sys_of_fin(A, f);
  const SysDesc &S = A.sys[s];
  const int64_t lf = f - S.fbeg;
  const int64_t T = fin_tile(lf, S.n_it, CH), tbeg = fin_prefix(T, CH);
  const int c = (int)(lf - tbeg);
  const int nch = (int)(T / CH + 1);
  const int m = A.m;
  const int64_t I_lo = (int64_t)c * CH, I_hi = min(T + 1, I_lo + CH);
  double *chunk = A.chunks + (S.fbeg + tbeg) * OUT;
  for (int o = threadIdx.x; o < OUT; o += kFinishThreadsB) {
    const int jsub = o / (TJ * NACC), rest = o % (TJ * NACC);
    CompSum cs{0.f, 0.f};
    // unit (I2, T m + jsub) advances by n_jt - m (I2 + 1) from I2 to I2 + 1
    int64_t off = (S.ubeg + sym_rowstart(I_lo, S.n_jt, m) + (T * m + jsub - (int64_t)m * I_lo)) * (TJ * NACC) + rest;
    int64_t step = (S.n_jt - (int64_t)m * (I_lo + 1)) * (TJ * NACC);
    const int64_t dstep = (int64_t)m * (TJ * NACC);
#pragma unroll 8
    for (int64_t I2 = I_lo; I2 < I_hi; I2++) {
      csum_add(cs, __ldcg(A.colslot + off));
      off += step;
      step -= dstep;
    }
    chunk[(int64_t)c * OUT + o] = csum_total(cs);
  }
  __threadfence();
  __syncthreads();
  const int64_t row = S.rbeg + T;
  if (threadIdx.x == 0) s_last = atomicAdd(&A.tickets[row], 1u) + 1u == (unsigned)nch;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int64_t cf = cta_of_unit(A.U, A.P, S.ubeg + sym_rowstart(T, S.n_jt, m));
  const int64_t cl = cta_of_unit(A.U, A.P, S.ubeg + sym_rowstart(T + 1, S.n_jt, m) - 1);
  const PairArgs v = view(A, S);
  for (int lr = threadIdx.x; lr < TI; lr += kFinishThreadsB) {
    const int64_t i = T * TI + lr;
    if (i >= S.N) break;
    double tot[NACC];
    if (cf == cl) {
#pragma unroll
      for (int d = 0; d < NACC; d++) tot[d] = __ldcg(A.rowfull + (row * NACC + d) * TI + lr);
    } else {
#pragma unroll
      for (int d = 0; d < NACC; d++) tot[d] = 0.0;
      for (int64_t c2 = cf; c2 <= cl; c2++) {
        int s2;
        int64_t it2, jt2;
        sym_locate(A, unit_begin(A.U, A.P, c2), s2, it2, jt2);
        const double *src = A.slots + ((c2 * 2 + (row == A.sys[s2].rbeg + it2 ? 0 : 1)) * NACC) * TI;
#pragma unroll
        for (int d = 0; d < NACC; d++) tot[d] += __ldcg(src + d * TI + lr);
      }
    }
    for (int c2 = 0; c2 < nch; c2++)
#pragma unroll
      for (int d = 0; d < NACC; d++) tot[d] -= __ldcg(chunk + (int64_t)c2 * OUT + lr * NACC + d);
    finish<Pol, MODEL, true, MODE>(v, i, tot);
  }
  if (threadIdx.x == 0) A.tickets[row] = 0u;
}

template <class Pol>
constexpr int sym_smem_bytes() {
  return 2 * Pol::TJ * Pol::JB + (NT / 32) * Pol::TJ * Pol::NACC * 4;
}

// One launch per part, each sized by its own occupancy (the parts' systems are
// disjoint, so the launches simply follow each other on the stream).
// The part's P = waves x gridDim.x stream-K ranges are virtual CTAs, which the CTAs
// take in increasing order from an atomic counter: a CTA that the SM's warp
// schedulers served faster takes more of them (the CTAs sharing an SM progress
// unevenly, and with a static split the SM's last CTA ran alone at the end), and at
// any time all CTAs work in about the same 1/waves of the unit list (the same few
// systems), whose j-records then stay in L2.
template <class Pol>
__global__ void __launch_bounds__(NT, Pol::MINB) batch_sym_pairs_kernel(PartArgs part) {
  __shared__ __align__(16) unsigned char smem[sym_smem_bytes<Pol>()];
  __shared__ unsigned s_vc;
  for (;;) {
    if (threadIdx.x == 0) s_vc = atomicAdd(part.next, 1u);
    __syncthreads();
    const unsigned vc = s_vc;
    __syncthreads();
    if (vc >= (unsigned)part.P) break;
    batch_sym_pairs<Pol>(part, (int64_t)vc, smem);
  }
}

template <class PolR, class PolG, int MODE>
__global__ void __launch_bounds__(kFinishThreadsB) batch_sym_finish_kernel(PartArgs ring, PartArgs grav) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *ring.next = *grav.next = 0u;  // the pair kernels have ended
  if ((int64_t)blockIdx.x < ring.nfin)
    batch_sym_finish<PolR, MD_RING, MODE>(ring, blockIdx.x);
  else
    batch_sym_finish<PolG, MD_GRAV2D, MODE>(grav, (int64_t)blockIdx.x - ring.nfin);
}

struct Config {
  int r = 0;            // i-particles per thread of the one-sided kernels (mixed: 4 or 8;
                        // FP64: 2); 0: Newton's-third-law kernels (mixed only)
  double split = 0.5;   // fraction of CTAs given to the Ring part
  int ctas_per_sm = 0;  // 0: occupancy limit
};

}  // namespace

struct md_batch {
  std::vector<md_ctx *> ctx;
  std::vector<int> model;
  int nsys = 0, prec = MD_MIXED, nsm = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int cur = 0;
  bool mirrors_valid = false;
  Config cfg;
  SysDesc *d_sys = nullptr;  // Ring descriptors, then 2D descriptors
  size_t d_sys_count = 0;
  double *slots = nullptr;
  size_t slots_bytes = 0;
  unsigned *tickets = nullptr;
  size_t tickets_count = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_key[2] = {-1, -1};
  int64_t graph_launches[2] = {0, 0};
  // unit / row layout uploaded for tile shapes and form (layout_key)
  int64_t layout_key[7] = {-1, -1, -1, -1, -1, -1, -1};
  int64_t Ur = 0, Ug = 0, rows_r = 0, rows_g = 0, nfin_r = 0, nfin_g = 0;
  int64_t rec_bytes_r = 0, rec_bytes_g = 0;  // forward-record bytes of each part's systems
  int nr = 0;
  int mirror_sym = -1;  // form the mirrors were written for (Ring records differ)
  double *rowfull = nullptr;  // Newton's-third-law form: row partials, column partials, chunk sums
  size_t rowfull_bytes = 0;
  float *colslot = nullptr;
  size_t colslot_bytes = 0;
  double *chunks = nullptr;
  size_t chunks_bytes = 0;
  std::vector<std::pair<const void *, int>> occ_cache;  // occupancy per kernel, queried outside captures
  int64_t launches = 0;
  std::string err;
};

namespace {

int berr(md_batch *b, int code, const char *fmt, const char *what) {
  char buf[512];
  snprintf(buf, sizeof buf, fmt, what);
  b->err = buf;
  set_err(nullptr, code, "%s", buf);
  return code;
}

#define B_CUDA(b, call)                                                             \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return berr((b), MD_ECUDA, #call ": %s", cudaGetErrorString(e_)); \
  } while (0)

void drop_graphs(md_batch *b) {
  for (int k = 0; k < 2; k++) {
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    b->graph[k] = nullptr;
    b->graph_key[k] = -1;
  }
}

// Descriptors and the unit / row layout of both parts: tile sizes (TI, TJ) per
// part, and the one-sided (rectangular unit table) or symmetric (triangular,
// n_jt = m n_it) form.
int build_layout(md_batch *b, const int64_t TI[2], const int64_t TJ[2], const int nacc[2], bool sym,
                 std::vector<SysDesc> &hs) {
  hs.clear();
  b->Ur = b->Ug = b->rows_r = b->rows_g = b->nfin_r = b->nfin_g = 0;
  b->rec_bytes_r = b->rec_bytes_g = 0;
  b->nr = 0;
  for (int pass = 0; pass < 2; pass++) {
    const int want = pass == 0 ? MD_RING : MD_GRAV2D;
    const int64_t ti = TI[pass], tj = TJ[pass], m = ti / tj;
    for (int s = 0; s < b->nsys; s++) {
      if (b->model[s] != want) continue;
      md_ctx *c = b->ctx[s];
      SysDesc d;
      d.q = c->q;
      d.p = c->p;
      d.f = c->f;
      d.mir[0] = (const unsigned char *)c->mirror[0];
      d.mir[1] = (const unsigned char *)c->mirror[1];
      d.N = c->N;
      d.n_it = (c->N + ti - 1) / ti;
      d.n_jt = sym ? m * d.n_it : (c->N + tj - 1) / tj;
      d.epsd = want == MD_RING ? 0.5 * c->eps : c->eps;
      d.dt = c->dt;
      d.nfin = fin_prefix(d.n_it, chunk_rows(ti * nacc[pass]));
      int64_t &U = pass == 0 ? b->Ur : b->Ug;
      int64_t &rows = pass == 0 ? b->rows_r : b->rows_g;
      int64_t &nfin = pass == 0 ? b->nfin_r : b->nfin_g;
      d.ubeg = U;
      d.rbeg = rows;
      d.fbeg = nfin;
      U += sym ? sym_rowstart(d.n_it, d.n_jt, (int)m) : d.n_it * d.n_jt;
      rows += d.n_it;
      nfin += d.nfin;
      // forward records: Ring tensor-core fragments (symmetric form) or interleaved FP32
      (pass == 0 ? b->rec_bytes_r : b->rec_bytes_g) += c->N * (pass == 0 ? (sym ? 64 : 16) : 8);
      hs.push_back(d);
      if (pass == 0) b->nr++;
    }
  }
  return MD_OK;
}

// Upload the layout for (TI, TJ, form) unless it is the current one.  Never runs
// inside a stream capture: the first step of md_batch_step and every autotune
// trial run uncaptured first.
int ensure_layout(md_batch *b, const int64_t TI[2], const int64_t TJ[2], const int nacc[2], bool sym) {
  const int64_t key[7] = {TI[0], TJ[0], TI[1], TJ[1], sym ? 1 : 0, nacc[0], nacc[1]};
  if (std::equal(key, key + 7, b->layout_key)) return MD_OK;
  std::vector<SysDesc> hs;
  build_layout(b, TI, TJ, nacc, sym, hs);
  if (hs.size() > b->d_sys_count) {
    dev_free(b->d_sys);
    b->d_sys = (SysDesc *)dev_alloc(hs.size() * sizeof(SysDesc));
    if (!b->d_sys) return berr(b, MD_ENOMEM, "%s", "batch descriptors");
    b->d_sys_count = hs.size();
  }
  B_CUDA(b, cudaStreamSynchronize(b->stream));  // no launch may still read the old layout
  B_CUDA(b, cudaMemcpy(b->d_sys, hs.data(), hs.size() * sizeof(SysDesc), cudaMemcpyHostToDevice));
  std::copy(key, key + 7, b->layout_key);
  return MD_OK;
}

template <class T>
int grow(md_batch *b, T *&ptr, size_t &have, size_t need, const char *what) {
  if (need <= have) return MD_OK;
  dev_free(ptr);
  ptr = (T *)dev_alloc(need);
  have = ptr ? need : 0;
  return ptr ? MD_OK : berr(b, MD_ENOMEM, "%s", what);
}

int ensure_tickets(md_batch *b) {
  // a ticket per row of both parts, then the two parts' virtual-CTA counters
  const size_t nt = (size_t)(b->rows_r + b->rows_g) + 2;
  if (nt > b->tickets_count) {
    dev_free(b->tickets);
    b->tickets = (unsigned *)dev_alloc(nt * sizeof(unsigned));
    if (!b->tickets) return berr(b, MD_ENOMEM, "%s", "batch tickets");
    b->tickets_count = nt;
    B_CUDA(b, cudaMemsetAsync(b->tickets, 0, nt * sizeof(unsigned), b->stream));
  }
  return MD_OK;
}

int occupancy(md_batch *b, const void *kern) {
  int occ = 0;
  for (const auto &kv : b->occ_cache)
    if (kv.first == kern) occ = kv.second;
  if (occ == 0) {
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, 0);
    if (occ < 1) occ = 1;
    b->occ_cache.push_back({kern, occ});
  }
  if (b->cfg.ctas_per_sm > 0 && b->cfg.ctas_per_sm < occ) occ = b->cfg.ctas_per_sm;
  return occ;
}

// CTAs of the Ring and 2D parts out of P, by the configured split
void split_ctas(const md_batch *b, int64_t P, int64_t &Pr, int64_t &Pg) {
  const int64_t Ur = b->Ur, Ug = b->Ug;
  Pr = Pg = 0;
  if (Ur > 0 && Ug > 0) {
    Pr = (int64_t)(b->cfg.split * (double)P + 0.5);
    if (Pr < 1) Pr = 1;
    if (Pr > P - 1) Pr = P - 1;
    Pg = P - Pr;
  } else if (Ur > 0) {
    Pr = P;
  } else {
    Pg = P;
  }
  if (Pr > Ur) Pr = Ur;
  if (Pg > Ug) Pg = Ug;
}

template <class PolR, class PolG, int MODE>
int launch_batch_sym(md_batch *b, double bc, double dc) {
  constexpr int64_t TIr = (int64_t)NT * PolR::R, TIg = (int64_t)NT * PolG::R;
  constexpr int NAr = PolR::NACC, NAg = PolG::NACC;
  const int64_t TI[2] = {TIr, TIg}, TJ[2] = {PolR::TJ, PolG::TJ};
  const int nacc[2] = {NAr, NAg};
  int rc = ensure_layout(b, TI, TJ, nacc, true);
  if (rc) return rc;
  // full GPU for each part in turn: CTA counts from each kernel's own occupancy
  auto kern_r = batch_sym_pairs_kernel<PolR>;
  auto kern_g = batch_sym_pairs_kernel<PolG>;
  const int occ_r = occupancy(b, (const void *)kern_r), occ_g = occupancy(b, (const void *)kern_g);
  const int64_t Gr = std::min<int64_t>((int64_t)b->nsm * occ_r, b->Ur);
  const int64_t Gg = std::min<int64_t>((int64_t)b->nsm * occ_g, b->Ug);
  // waves: the part's j-records over about a quarter of L2 (129 MB), and at least
  // kMinWaves virtual CTAs per CTA to even out the CTAs' uneven progress; at least 16
  // units per virtual CTA
  auto waves_of = [&](int64_t rec_bytes, int64_t U, int64_t G) -> int {
    int64_t w = std::max<int64_t>(kMinWaves, (rec_bytes + kWaveRecordBytes - 1) / kWaveRecordBytes);
    if (w > U / (16 * (G > 0 ? G : 1))) w = U / (16 * (G > 0 ? G : 1));
    return (int)std::max<int64_t>(1, std::min<int64_t>(w, 16));
  };
  const int Wr = waves_of(b->rec_bytes_r, b->Ur, Gr), Wg = waves_of(b->rec_bytes_g, b->Ug, Gg);
  const int64_t Pr = Gr * Wr, Pg = Gg * Wg;  // virtual CTAs
  const size_t slot_r = (size_t)Pr * 2 * NAr * TIr, slot_g = (size_t)Pg * 2 * NAg * TIg;
  const size_t row_r = (size_t)b->rows_r * NAr * TIr, row_g = (size_t)b->rows_g * NAg * TIg;
  const size_t col_r = (size_t)b->Ur * PolR::TJ * NAr, col_g = (size_t)b->Ug * PolG::TJ * NAg;
  const size_t ch_r = (size_t)b->nfin_r * TIr * NAr, ch_g = (size_t)b->nfin_g * TIg * NAg;
  if ((rc = grow(b, b->slots, b->slots_bytes, (slot_r + slot_g) * sizeof(double), "batch slots")) ||
      (rc = grow(b, b->rowfull, b->rowfull_bytes, (row_r + row_g) * sizeof(double), "batch row partials")) ||
      (rc = grow(b, b->colslot, b->colslot_bytes, (col_r + col_g) * sizeof(float), "batch column partials")) ||
      (rc = grow(b, b->chunks, b->chunks_bytes, (ch_r + ch_g) * sizeof(double), "batch chunk sums")) ||
      (rc = ensure_tickets(b)))
    return rc;
  PartArgs ar{}, ag{};
  ar.sys = b->d_sys;
  ar.nsys = b->nr;
  ar.U = b->Ur;
  ar.P = (int)Pr;
  ar.waves = Wr;
  ar.next = b->tickets + b->rows_r + b->rows_g;
  ar.m = (int)(TIr / PolR::TJ);
  ar.nfin = b->nfin_r;
  ar.slots = b->slots;
  ar.rowfull = b->rowfull;
  ar.colslot = b->colslot;
  ar.chunks = b->chunks;
  ar.tickets = b->tickets;
  ag.sys = b->d_sys + b->nr;
  ag.nsys = b->nsys - b->nr;
  ag.U = b->Ug;
  ag.P = (int)Pg;
  ag.waves = Wg;
  ag.next = ar.next + 1;
  ag.m = (int)(TIg / PolG::TJ);
  ag.nfin = b->nfin_g;
  ag.slots = b->slots + slot_r;
  ag.rowfull = b->rowfull + row_r;
  ag.colslot = b->colslot + col_r;
  ag.chunks = b->chunks + ch_r;
  ag.tickets = b->tickets + b->rows_r;
  ar.cur = ag.cur = b->cur;
  ar.b = ag.b = bc;
  ar.d = ag.d = dc;
  if (Gr > 0) {
    kern_r<<<(int)Gr, NT, 0, b->stream>>>(ar);
    b->launches++;
  }
  if (Gg > 0) {
    kern_g<<<(int)Gg, NT, 0, b->stream>>>(ag);
    b->launches++;
  }
  batch_sym_finish_kernel<PolR, PolG, MODE><<<(unsigned)(b->nfin_r + b->nfin_g), kFinishThreadsB, 0, b->stream>>>(ar, ag);
  b->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return berr(b, MD_ECUDA, "batch launch: %s", cudaGetErrorString(e));
  if (MODE == STAGE_KICK_DRIFT) b->cur = 1 - b->cur;
  return MD_OK;
}

template <class PolR, class PolG, bool MIXED, int MODE>
int launch_batch(md_batch *b, double bc, double dc) {
  constexpr int64_t TI = (int64_t)NT * PolR::R;
  static_assert(PolR::R == PolG::R && PolR::TJ == PolG::TJ, "parts share the tile shape");
  const int64_t TIs[2] = {TI, TI}, TJs[2] = {PolR::TJ, PolG::TJ};
  const int naccs[2] = {PolR::NACC, PolG::NACC};
  int rc = ensure_layout(b, TIs, TJs, naccs, false);
  if (rc) return rc;
  auto kern = batch_kernel<PolR, PolG, MIXED, MODE>;
  const int occ = occupancy(b, (const void *)kern);
  int64_t Pr, Pg;
  split_ctas(b, (int64_t)b->nsm * occ, Pr, Pg);
  const size_t slot_r = (size_t)Pr * 2 * PolR::NACC * TI, slot_g = (size_t)Pg * 2 * PolG::NACC * TI;
  if ((rc = grow(b, b->slots, b->slots_bytes, (slot_r + slot_g) * sizeof(double), "batch slots")) ||
      (rc = ensure_tickets(b)))
    return rc;
  PartArgs ar{}, ag{};
  ar.sys = b->d_sys;
  ar.nsys = b->nr;
  ar.U = b->Ur;
  ar.P = (int)Pr;
  ag.sys = b->d_sys + b->nr;
  ag.nsys = b->nsys - b->nr;
  ag.U = b->Ug;
  ag.P = (int)Pg;
  ar.cur = ag.cur = b->cur;
  ar.b = ag.b = bc;
  ar.d = ag.d = dc;
  ar.slots = b->slots;
  ag.slots = b->slots + slot_r;
  ar.tickets = b->tickets;
  ag.tickets = b->tickets + b->rows_r;
  kern<<<(int)(Pr + Pg), NT, 0, b->stream>>>(ar, ag);
  b->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return berr(b, MD_ECUDA, "batch launch: %s", cudaGetErrorString(e));
  if (MODE == STAGE_KICK_DRIFT) b->cur = 1 - b->cur;
  return MD_OK;
}

bool sym_form(const md_batch *b) { return b->prec == MD_MIXED && b->cfg.r == 0; }

template <bool MIXED, int MODE>
int dispatch(md_batch *b, double bc, double dc) {
  if constexpr (MIXED) {
    if (b->cfg.r == 0) return launch_batch_sym<RingTC<4, 256, MODE>, GravMixed<8, 256, MODE>, MODE>(b, bc, dc);
    if (b->cfg.r == 4)
      return launch_batch<RingMixed<4, 256, MODE>, GravMixed<4, 256, MODE>, true, MODE>(b, bc, dc);
    return launch_batch<RingMixed<8, 256, MODE>, GravMixed<8, 256, MODE>, true, MODE>(b, bc, dc);
  } else {
    return launch_batch<RingF64<2, 128, MODE>, GravF64<2, 128, MODE>, false, MODE>(b, bc, dc);
  }
}

int refresh_mirrors(md_batch *b);

int stage(md_batch *b, int mode, double bc, double dc) {
  if (!b->mirrors_valid || b->mirror_sym != (sym_form(b) ? 1 : 0)) {
    b->mirrors_valid = false;
    int rc = refresh_mirrors(b);
    if (rc) return rc;
  }
  const bool mixed = b->prec == MD_MIXED;
  switch (mode) {
  case STAGE_KICK_DRIFT: return mixed ? dispatch<true, STAGE_KICK_DRIFT>(b, bc, dc) : dispatch<false, STAGE_KICK_DRIFT>(b, bc, dc);
  case STAGE_KICK_ONLY: return mixed ? dispatch<true, STAGE_KICK_ONLY>(b, bc, dc) : dispatch<false, STAGE_KICK_ONLY>(b, bc, dc);
  default: return mixed ? dispatch<true, STAGE_FORCE_ONLY>(b, bc, dc) : dispatch<false, STAGE_FORCE_ONLY>(b, bc, dc);
  }
}

int refresh_mirrors(md_batch *b) {
  const int sym = sym_form(b) ? 1 : 0;
  if (b->mirrors_valid && b->mirror_sym == sym) return MD_OK;
  for (md_ctx *c : b->ctx) {
    c->prec = b->prec;
    c->pt.ring_tc = sym;  // symmetric form: tensor-core Ring records; one-sided: interleaved
    c->mirror_cur = b->cur;
    int rc = mirror_refresh(c);
    if (rc) return berr(b, rc, "%s", c->err.c_str());
  }
  b->mirrors_valid = true;
  b->mirror_sym = sym;
  return MD_OK;
}

}  // namespace

extern "C" {

md_batch *md_batch_init(int nsys, const int *model, const int64_t *N, const double *eps, const double *dt,
                        const uint64_t *seed) {
  if (nsys < 1 || !model || !N || !eps || !dt || !seed) {
    set_err(nullptr, MD_EINVAL, "md_batch_init: need nsys >= 1 and non-NULL arrays");
    return nullptr;
  }
  for (int s = 0; s < nsys; s++)
    if (model[s] != MD_RING && model[s] != MD_GRAV2D) {
      set_err(nullptr, MD_EINVAL, "md_batch_init: system %d: only MD_RING and MD_GRAV2D systems batch", s);
      return nullptr;
    }
  md_batch *b = new (std::nothrow) md_batch();
  if (!b) {
    set_err(nullptr, MD_ENOMEM, "md_batch_init: host allocation");
    return nullptr;
  }
  b->nsys = nsys;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_err(nullptr, MD_ECUDA, "md_batch_init: device setup: %s", cudaGetErrorString(cudaGetLastError()));
    delete b;
    return nullptr;
  }
  b->own_stream = true;
  double work_r = 0.0, work_g = 0.0;
  for (int s = 0; s < nsys; s++) {
    md_ctx *c = md_init(model[s], N[s], eps[s], dt[s], seed[s]);
    if (!c) {
      std::string m = md_last_error(nullptr);
      md_batch_free(b);
      set_err(nullptr, MD_EINVAL, "md_batch_init: system %d: %s", s, m.c_str());
      return nullptr;
    }
    if (md_set_stream(c, b->stream) != MD_OK) {
      md_free(c);
      md_batch_free(b);
      set_err(nullptr, MD_ECUDA, "md_batch_init: stream");
      return nullptr;
    }
    c->prec = MD_MIXED;
    b->ctx.push_back(c);
    b->model.push_back(model[s]);
    (model[s] == MD_RING ? work_r : work_g) += (double)N[s] * (double)N[s];
  }
  // first split: pair counts weighted by the measured single-system costs per pair
  // (Ring / 2D about 1.07 on GB300); md_batch_autotune refines it
  const double wr = 1.07 * work_r, wg = work_g;
  b->cfg.split = (wr + wg) > 0.0 ? wr / (wr + wg) : 0.5;
  return b;
}

void md_batch_free(md_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  for (md_ctx *c : b->ctx) {
    c->stream = nullptr;
    c->own_stream = false;
    md_free(c);
  }
  dev_free(b->d_sys);
  dev_free(b->slots);
  dev_free(b->tickets);
  dev_free(b->rowfull);
  dev_free(b->colslot);
  dev_free(b->chunks);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char *md_batch_last_error(const md_batch *b) { return b ? b->err.c_str() : md_last_error(nullptr); }

int64_t md_batch_launch_count(const md_batch *b) {
  if (!b) return 0;
  int64_t n = b->launches;
  for (const md_ctx *c : b->ctx) n += c->launches;
  return n;
}

int md_batch_set_precision(md_batch *b, int prec) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  if (prec != MD_FP64 && prec != MD_MIXED) return berr(b, MD_EINVAL, "%s", "unknown precision");
  if (prec != b->prec) {
    b->prec = prec;
    b->mirrors_valid = false;
    drop_graphs(b);
  }
  return MD_OK;
}

int md_batch_set_stream(md_batch *b, void *stream) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  if (b->own_stream) cudaStreamDestroy(b->stream);
  b->stream = (cudaStream_t)stream;
  b->own_stream = false;
  for (md_ctx *c : b->ctx) c->stream = b->stream;
  drop_graphs(b);
  return MD_OK;
}

int md_batch_set_tuning(md_batch *b, int r, double split, int ctas_per_sm) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  if ((r != 0 && r != 4 && r != 8) || !(split > 0.0 && split < 1.0) || ctas_per_sm < 0 || ctas_per_sm > 16)
    return berr(b, MD_EINVAL, "%s", "md_batch_set_tuning: need r in {0, 4, 8}, 0 < split < 1, 0 <= ctas_per_sm <= 16");
  b->cfg.r = r;
  b->cfg.split = split;
  b->cfg.ctas_per_sm = ctas_per_sm;
  drop_graphs(b);
  return MD_OK;
}

int md_batch_get_tuning(const md_batch *b, int *r, double *split, int *ctas_per_sm) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  if (r) *r = b->cfg.r;
  if (split) *split = b->cfg.split;
  if (ctas_per_sm) *ctas_per_sm = b->cfg.ctas_per_sm;
  return MD_OK;
}

int md_batch_autotune(md_batch *b, double *best_ms) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  int rc = refresh_mirrors(b);
  if (rc) return rc;
  const Config base = b->cfg;
  std::vector<Config> cand;
  const int rs[3] = {0, 8, 4};
  const double fs[5] = {0.90, 0.95, 1.0, 1.05, 1.10};
  const int cps[2] = {0, 3};
  for (int r : rs)
    for (double f : fs)
      for (int cp : cps) {
        if (b->prec != MD_MIXED && r != rs[0]) continue;
        Config c = base;
        c.r = b->prec == MD_MIXED ? r : base.r;
        c.split = base.split * f > 0.98 ? 0.98 : base.split * f;
        c.ctas_per_sm = cp;
        cand.push_back(c);
      }
  cudaEvent_t e0, e1;
  B_CUDA(b, cudaEventCreate(&e0));
  B_CUDA(b, cudaEventCreate(&e1));
  float best = 1e30f;
  Config pick = base;
  for (const Config &c : cand) {
    b->cfg = c;
    if ((rc = stage(b, STAGE_FORCE_ONLY, 0.0, 0.0))) break;  // warm-up (allocations)
    B_CUDA(b, cudaEventRecord(e0, b->stream));
    if ((rc = stage(b, STAGE_FORCE_ONLY, 0.0, 0.0))) break;
    B_CUDA(b, cudaEventRecord(e1, b->stream));
    B_CUDA(b, cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->cfg = pick;
  drop_graphs(b);
  if (best_ms) *best_ms = best;
  return rc;
}

int md_batch_step(md_batch *b, int64_t nsteps) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  if (nsteps < 0) return berr(b, MD_EINVAL, "%s", "md_batch_step: nsteps < 0");
  if (nsteps == 0) return MD_OK;
  int rc = refresh_mirrors(b);
  if (rc) return rc;
  double k[4];
  yoshida_coefficients(k);
  const double B0 = k[0], B1 = k[1], D0 = k[2], D1 = k[3];
  // first step (uncaptured: it also makes every buffer the graph will use)
  if ((rc = stage(b, STAGE_KICK_DRIFT, B0, D0)) || (rc = stage(b, STAGE_KICK_DRIFT, B1, D1)) ||
      (rc = stage(b, STAGE_KICK_DRIFT, B1, D0)))
    return rc;
  int64_t left = nsteps - 1;
  // capture only on a capturable stream that is not being captured already
  bool graphs = b->stream != nullptr && b->stream != cudaStreamLegacy && b->stream != cudaStreamPerThread;
  if (graphs) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    graphs = cudaStreamIsCapturing(b->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
    cudaGetLastError();
  }
  while (graphs && left >= kGraphSteps) {
    const int key = b->cur;
    if (b->graph_key[key] != key || !b->graph[key]) {
      cudaGraph_t g;
      B_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      const int64_t l0 = b->launches;
      for (int s = 0; s < kGraphSteps && !rc; s++) {
        if (!rc) rc = stage(b, STAGE_KICK_DRIFT, 2.0 * B0, D0);
        if (!rc) rc = stage(b, STAGE_KICK_DRIFT, B1, D1);
        if (!rc) rc = stage(b, STAGE_KICK_DRIFT, B1, D0);
      }
      cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
      if (rc) return rc;
      if (ee != cudaSuccess) return berr(b, MD_ECUDA, "graph capture: %s", cudaGetErrorString(ee));
      b->graph_launches[key] = b->launches - l0;
      b->launches = l0;  // captured, not launched
      B_CUDA(b, cudaGraphInstantiate(&b->graph[key], g, 0));
      cudaGraphDestroy(g);
      b->graph_key[key] = key;
    }
    B_CUDA(b, cudaGraphLaunch(b->graph[key], b->stream));
    b->launches += b->graph_launches[key];
    left -= kGraphSteps;
  }
  for (; left > 0; left--) {
    if ((rc = stage(b, STAGE_KICK_DRIFT, 2.0 * B0, D0)) || (rc = stage(b, STAGE_KICK_DRIFT, B1, D1)) ||
        (rc = stage(b, STAGE_KICK_DRIFT, B1, D0)))
      return rc;
  }
  rc = stage(b, STAGE_KICK_ONLY, B0, 0.0);
  for (md_ctx *c : b->ctx) {
    c->mirror_cur = b->cur;
    c->fsal_valid = false;
  }
  return rc;
}

int md_batch_force(md_batch *b, double *const *f) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  if (!f) return berr(b, MD_EINVAL, "%s", "md_batch_force: NULL array of outputs");
  int rc = stage(b, STAGE_FORCE_ONLY, 0.0, 0.0);  // every system, the launches md_batch_step runs
  if (rc) return rc;
  for (int s = 0; s < b->nsys; s++) {
    md_ctx *c = b->ctx[s];
    c->fsal_valid = false;  // c->f now holds this force, not a cached one of md_step
    if (f[s])
      B_CUDA(b, cudaMemcpyAsync(f[s], c->f, sizeof(double) * (size_t)(c->dim * c->N), cudaMemcpyDeviceToHost,
                                b->stream));
  }
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  return MD_OK;
}

int md_batch_energy(md_batch *b, double *K, double *V) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  for (int s = 0; s < b->nsys; s++) {
    double k = 0.0, v = 0.0;
    int rc = md_energy(b->ctx[s], &k, &v);
    if (rc) return berr(b, rc, "%s", b->ctx[s]->err.c_str());
    if (K) K[s] = k;
    if (V) V[s] = v;
  }
  return MD_OK;
}

int md_batch_get_state(md_batch *b, int s, double *q, double *p) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  if (s < 0 || s >= b->nsys) return berr(b, MD_EINVAL, "%s", "system index out of range");
  int rc = md_get_state(b->ctx[s], q, p);
  return rc ? berr(b, rc, "%s", b->ctx[s]->err.c_str()) : MD_OK;
}

int md_batch_set_state(md_batch *b, int s, const double *q, const double *p) {
  if (!b) return set_err(nullptr, MD_EINVAL, "NULL batch");
  if (s < 0 || s >= b->nsys) return berr(b, MD_EINVAL, "%s", "system index out of range");
  int rc = md_set_state(b->ctx[s], q, p);
  b->mirrors_valid = false;
  return rc ? berr(b, rc, "%s", b->ctx[s]->err.c_str()) : MD_OK;
}

}  // extern "C"
