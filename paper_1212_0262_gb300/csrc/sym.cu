// Newton's-third-law variant of the Ring and 2D force stages: every
// unordered pair is evaluated once and its term added to both particles.  The
// paper evaluates every ordered pair (Sec. 3.2, tile algorithm) and leaves this
// variant out; it is one of the extensions its conclusion names.
//
// The summands are antisymmetric: with q_ij the term of particle i's sum,
//   Ring:  q_ij = S_ij dd_ij^(-3/2),  S_ji = -S_ij (sine of the opposite angle),
//          dd_ji = dd_ij (sin^2 of the half angle is even);
//   2D:    q_ij = r_ij / (|r_ij|^2 + eps),  r_ji = -r_ij;
// so f_j receives -q_ij from the evaluation of (i, j).
//
// Units.  i-tiles of TI = m TJ particles (m = TI/TJ), j-tiles of TJ.  Row I of
// the unit table holds the j-tiles J = m I .. n_jt - 1 (n_jt = m n_it), so
// rowstart(I) = I n_jt - m I (I - 1) / 2 and U = rowstart(n_it).  A unit whose
// j-tile lies inside its i-tile (J < m (I + 1), "diagonal") holds pairs of the
// tile's own particles: the FP32 Ring and 2D policies (tile_diag) evaluate the
// pairs above the diagonal once, as below, and only the squares on the diagonal
// (16 x 16 for Ring, 256 x 256 for 2D) for the i-rows alone; the other policies
// evaluate the whole TI x TJ block for the i-rows only, self pairs masked.  Every
// other unit evaluates its block once: the i-rows accumulate in registers across
// the CTA's consecutive units of the row (as in the one-sided kernel), and the sums over
// the block's i-rows for each of its TJ j's (warp butterflies, then the warps in
// a fixed order through shared memory) are stored as that unit's column partial
// (FP32, [U][TJ][NACC]).
//
// Pair phase (sym_pairs_kernel, stream-K).  Virtual CTA c (taken by the
// persistent CTAs in increasing order, take_vcta) covers units
// [U c / P, U (c+1) / P) in row-major order and writes the row partials of the
// rows it covers (rowfull[T] when it covered all of row T, else the one-sided
// kernel's two slots per virtual CTA) and the column partial of each off-diagonal
// unit (and of each diagonal one, with tile_diag).
//
// Finish phase (sym_finish_kernel).  Tile T needs its row partials and the
// column partials of the units (I', J), J in tile T, I' < T (I' <= T with
// tile_diag).  One CTA per
// (tile, chunk of sym_chunk rows I') sums a chunk's column partials per particle
// and component (compensated FP32, then one double); the last chunk of a tile to
// arrive (atomic ticket, no waiting) adds the row partials in CTA order and the
// chunk sums in chunk order, and runs the stage epilogue (kick, drift, new mirror
// record) for the tile's particles.  Every sum has a fixed order, so results are
// deterministic.  The finish phase spreads the O(N^2 / TJ) column reads over the
// whole GPU; finishing a tile inside the pair kernel instead serialised them on
// the few CTAs that cover the many short rows at the end of the order.
// Column partials take U TJ NACC floats: beyond kSymMaxColBytes the one-sided
// kernel runs instead.
#include <mutex>

#include "pairs_impl.cuh"

namespace {

constexpr size_t kSymMaxColBytes = (size_t)16 << 30;  // Ring and 2D at N = 1e6 fit

struct SymArgs {
  int m;             // TI / TJ
  int nc;            // chunk slots per tile in the finish phase
  double *rowfull;   // [n_it][NACC][TI] row partials of rows covered by one CTA
  void *colslot;     // [U][TJ][NACC] column partials of the units (Pol::ColT:
                     // FP32 for the mixed policies, FP64 for the FP64 ones)
  double *chunks;    // [n_it][nc][TI][NACC] chunk sums of the column partials
};

// CTAs of the pair kernel that cover part of row T: [cf, cl].
__device__ __forceinline__ void sym_row_ctas(const PairArgs &a, const SymArgs &s, int64_t T, int64_t &cf,
                                             int64_t &cl) {
  cf = cta_of_unit(a.U, a.P, sym_rowstart(T, a.n_jt, s.m));
  cl = cta_of_unit(a.U, a.P, sym_rowstart(T + 1, a.n_jt, s.m) - 1);
}

// Pair phase: every unit's block, row partials per CTA segment, column partials per unit.
template <class Pol>
__global__ void __launch_bounds__(Pol::THREADS, Pol::MINB) sym_pairs_kernel(PairArgs a, SymArgs s) {
  constexpr int THR = Pol::THREADS, NW = THR / 32;
  constexpr int TJ = Pol::TJ, NACC = Pol::NACC;
  constexpr int TILE_BYTES = TJ * Pol::JB;
  constexpr int CHUNKS = TILE_BYTES / 16;
  constexpr int64_t TI = (int64_t)THR * Pol::R;
  static_assert(TILE_BYTES % 16 == 0, "tile must be a whole number of 16-byte chunks");
  static_assert(TI % TJ == 0, "i-tiles must be whole numbers of j-tiles");
  using ColT = typename Pol::ColT;
  constexpr bool DIAG_SYM = HasDiagSym<Pol>::value;
  __shared__ __align__(16) unsigned char sbuf[2][TILE_BYTES];
  __shared__ __align__(16) unsigned char colraw[NW * TJ * NACC * sizeof(ColT)];
  ColT *colsm = (ColT *)colraw;
  __shared__ unsigned s_vc;
  const int m = s.m;
  const unsigned char *mir = (const unsigned char *)a.mirror_in;
  auto prefetch = [&](int buf, int64_t jt) {
    const unsigned char *src = mir + jt * (int64_t)TILE_BYTES;
    for (int ch = threadIdx.x; ch < CHUNKS; ch += THR) cp_async16(&sbuf[buf][ch * 16], src + ch * 16);
    cp_async_commit();
  };

  for (;;) {
    const int64_t cta = take_vcta(a.sched, s_vc);  // virtual CTA: its range and slots
    if (cta >= a.P) break;
    const int64_t u0 = unit_begin(a.U, a.P, cta), u1 = unit_begin(a.U, a.P, cta + 1);
    if (u0 >= u1) continue;

    typename Pol::State st;
    int64_t it = sym_row_of_unit(u0, a.n_it, a.n_jt, m);
    const int64_t first_row = it;
    int64_t jt = (int64_t)m * it + (u0 - sym_rowstart(it, a.n_jt, m));
    bool row_from_start = (jt == (int64_t)m * it);
    int64_t i0 = it * TI;
    Pol::load(st, a.mirror_in, i0);
    prefetch(0, jt);

    for (int64_t u = u0; u < u1; u++) {
      const int buf = (int)((u - u0) & 1);
      const bool row_end = (jt + 1 == a.n_jt);
      const int64_t next_jt = row_end ? (int64_t)m * (it + 1) : jt + 1;
      if (u + 1 < u1) {
        prefetch(buf ^ 1, next_jt);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const bool diag = jt < (int64_t)m * (it + 1);
      if (!diag) Pol::tile_sym(st, sbuf[buf], a, colsm);
      else if constexpr (DIAG_SYM) Pol::tile_diag(st, sbuf[buf], a, colsm, (int)(jt - (int64_t)m * it));
      else Pol::template tile<true>(st, sbuf[buf], a, i0, jt * TJ);
      __syncthreads();
      if (!diag || DIAG_SYM) {
        // column partial of this unit: the warps' sums in a fixed order (colsm is
        // rewritten only after the next unit's first barrier)
        ColT *dst = (ColT *)s.colslot + u * (int64_t)(TJ * NACC);
        for (int idx = threadIdx.x; idx < TJ * NACC; idx += THR) {
          ColT v = colsm[idx];
  #pragma unroll
          for (int w = 1; w < NW; w++) v += colsm[w * TJ * NACC + idx];
          dst[idx] = v;
        }
      }
      if (row_end || u + 1 == u1) {
        // this CTA's part of row it
        double *sp = (row_end && row_from_start)
                         ? s.rowfull + it * NACC * TI
                         : a.slots + ((cta * 2 + (it == first_row ? 0 : 1)) * NACC) * TI;
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
          it++;
          row_from_start = true;
          i0 = it * TI;
          Pol::load(st, a.mirror_in, i0);
        }
      }
      jt = next_jt;
    }
  }
  vcta_done(a.sched);
}

// Finish phase, one CTA per (tile T, chunk c of sym_chunk rows I' < T, or I' <= T
// with tile_diag): the chunk's column partials summed per particle and component
// (compensated FP32) into one double; the last chunk of the tile to arrive (atomic
// ticket, no waiting) adds the row partials (CTA order) and the chunk sums (chunk
// order) and runs the stage epilogue.  A tile with no rows I' has one empty chunk.
constexpr int kFinishThreads = 256;

// Column-partial rows per finish CTA: about 16K loads per CTA whatever the tile's
// output count (Ring FP32 tiles have 256 outputs, 2D 2048).
template <class Pol>
constexpr int sym_chunk() {
  constexpr int out = Pol::THREADS * Pol::R * Pol::NACC;
  return out <= 256 ? 64 : out <= 512 ? 32 : 16;
}

template <class Pol, int MODEL, bool MIXED, int MODE>
__global__ void __launch_bounds__(kFinishThreads) sym_finish_kernel(PairArgs a, SymArgs s) {
  constexpr int NACC = Pol::NACC, TJ = Pol::TJ;
  constexpr int64_t TI = (int64_t)Pol::THREADS * Pol::R;
  constexpr int OUT = (int)TI * NACC;  // outputs of a tile: (particle, component)
  __shared__ bool s_last;
  const int64_t T = blockIdx.x / s.nc;
  const int c = (int)(blockIdx.x % s.nc);
  constexpr int CH = sym_chunk<Pol>();
  const int64_t rows = T + (HasDiagSym<Pol>::value ? 1 : 0);  // column-partial rows I of tile T
  const int nch = rows == 0 ? 1 : (int)((rows + CH - 1) / CH);
  if (c >= nch) return;
  const int m = s.m;
  const int64_t I_lo = (int64_t)c * CH, I_hi = min(rows, I_lo + CH);
  double *chunk = s.chunks + (T * s.nc) * OUT;
  using ColT = typename Pol::ColT;
  const ColT *col = (const ColT *)s.colslot;
  for (int o = threadIdx.x; o < OUT; o += kFinishThreads) {
    const int jsub = o / (TJ * NACC), rest = o % (TJ * NACC);
    CompSum cs{0.f, 0.f};  // FP32 column partials: compensated FP32 sum
    double sd = 0.0;       // FP64 column partials
    // unit (I2, T m + jsub) = rowstart(I2) + T m + jsub - m I2; from I2 to I2 + 1 it
    // advances by the length of row I2 minus m, i.e. n_jt - m (I2 + 1)
    int64_t off = (sym_rowstart(I_lo, a.n_jt, m) + (T * m + jsub - (int64_t)m * I_lo)) * (TJ * NACC) + rest;
    int64_t step = (a.n_jt - (int64_t)m * (I_lo + 1)) * (TJ * NACC);
    const int64_t dstep = (int64_t)m * (TJ * NACC);
#pragma unroll 8
    for (int64_t I2 = I_lo; I2 < I_hi; I2++) {
      if constexpr (sizeof(ColT) == 4) csum_add(cs, __ldcg(col + off));
      else sd += __ldcg(col + off);
      off += step;
      step -= dstep;
    }
    chunk[(int64_t)c * OUT + o] = sizeof(ColT) == 4 ? csum_total(cs) : sd;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&a.tickets[T], 1u) + 1u == (unsigned)nch;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  int64_t cf, cl;
  sym_row_ctas(a, s, T, cf, cl);
  for (int lr = threadIdx.x; lr < TI; lr += kFinishThreads) {
    const int64_t i = T * TI + lr;
    if (i >= a.N) break;
    double tot[NACC];
    if (cf == cl) {
#pragma unroll
      for (int d = 0; d < NACC; d++) tot[d] = __ldcg(s.rowfull + (T * NACC + d) * TI + lr);
    } else {
#pragma unroll
      for (int d = 0; d < NACC; d++) tot[d] = 0.0;
      for (int64_t c2 = cf; c2 <= cl; c2++) {
        const int64_t fr = sym_row_of_unit(unit_begin(a.U, a.P, c2), a.n_it, a.n_jt, m);
        const double *src = a.slots + ((c2 * 2 + (T == fr ? 0 : 1)) * NACC) * TI;
#pragma unroll
        for (int d = 0; d < NACC; d++) tot[d] += __ldcg(src + d * TI + lr);
      }
    }
    // output o = (lr / TJ) TJ NACC + (lr % TJ) NACC + d = lr NACC + d
    for (int c2 = 0; c2 < nch; c2++)
#pragma unroll
      for (int d = 0; d < NACC; d++) tot[d] -= __ldcg(chunk + (int64_t)c2 * OUT + lr * NACC + d);
    finish<Pol, MODEL, MIXED, MODE>(a, i, tot);
  }
  if (threadIdx.x == 0) a.tickets[T] = 0u;
}

// ------------------------------------------------------------ host side ---

template <class Pol, int MODEL, bool MIXED, int MODE>
int launch_sym(md_ctx *c, PairArgs a) {
  constexpr int THR = Pol::THREADS;
  constexpr int64_t TI = (int64_t)THR * Pol::R;
  constexpr int TJ = Pol::TJ, NACC = Pol::NACC;
  auto kern = sym_pairs_kernel<Pol>;
  // the grid is sized for the occupancy limit: make the shared-memory carveout allow it
  // (once per kernel, on the first call, which runs before any stream capture)
  static std::once_flag carveout_once;
  std::call_once(carveout_once, [&] {
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  });
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, THR, 0);
  if (occ < 1) occ = 1;
  if (c->pt.ctas_per_sm > 0 && c->pt.ctas_per_sm < occ) occ = c->pt.ctas_per_sm;
  SymArgs s{};
  s.m = (int)(TI / TJ);
  a.N = c->N;
  a.n_it = (c->N + TI - 1) / TI;
  a.n_jt = s.m * a.n_it;
  a.U = sym_rowstart(a.n_it, a.n_jt, s.m);
  const int64_t G = std::min<int64_t>((int64_t)c->nsm * occ, a.U);  // CTAs
  // virtual CTAs per CTA, measured at the bench sizes (sweeps of 1-16 show sharp dips at
  // single values, 4 for these two among them): 8 for the Ring tensor-core kernel, 3 for
  // the FP64 3D kernel, 4 for the others
  const int kv = c->pt.vcta > 0 ? c->pt.vcta : Pol::FMT == 1 ? 8 : (MODEL == MD_GRAV3D && !MIXED) ? 3 : 4;
  a.P = (int)vcta_count(G, a.U, kv);
  int rc = ensure_pair_buffers(c, (int)TI, a.P, NACC);
  if (rc) return rc;
  const int64_t max_rows = a.n_it - 1 + (HasDiagSym<Pol>::value ? 1 : 0);  // of the last tile
  s.nc = (int)std::max<int64_t>(1, (max_rows + sym_chunk<Pol>() - 1) / sym_chunk<Pol>());
  const size_t need_row = (size_t)a.n_it * NACC * TI * sizeof(double);
  const size_t need_col = (size_t)a.U * TJ * NACC * sizeof(typename Pol::ColT);
  const size_t need_chunk = (size_t)a.n_it * s.nc * NACC * TI * sizeof(double);
  if (need_row > c->sym_rowfull_bytes) {
    dev_free(c->sym_rowfull);
    c->sym_rowfull = (double *)dev_alloc(need_row);
    c->sym_rowfull_bytes = c->sym_rowfull ? need_row : 0;
    if (!c->sym_rowfull) return set_err(c, MD_ENOMEM, "symmetric row partials: %zu bytes", need_row);
  }
  if (need_col > c->sym_colslot_bytes) {
    dev_free(c->sym_colslot);
    c->sym_colslot = dev_alloc(need_col);
    c->sym_colslot_bytes = c->sym_colslot ? need_col : 0;
    if (!c->sym_colslot) return set_err(c, MD_ENOMEM, "symmetric column partials: %zu bytes", need_col);
  }
  if (need_chunk > c->sym_chunk_bytes) {
    dev_free(c->sym_chunks);
    c->sym_chunks = (double *)dev_alloc(need_chunk);
    c->sym_chunk_bytes = c->sym_chunks ? need_chunk : 0;
    if (!c->sym_chunks) return set_err(c, MD_ENOMEM, "symmetric chunk sums: %zu bytes", need_chunk);
  }
  s.rowfull = c->sym_rowfull;
  s.colslot = c->sym_colslot;
  s.chunks = c->sym_chunks;
  a.mirror_in = c->mirror[c->mirror_cur];
  a.mirror_out = c->mirror[1 - c->mirror_cur];
  a.q = c->q;
  a.p = c->p;
  a.epsd = MODEL == MD_RING ? 0.5 * c->eps : c->eps;  // 2D, 3D, sheets: eps
  a.slots = c->sk_slots;
  a.tickets = c->sk_tickets;
  a.sched = pair_sched(c);
  kern<<<(int)G, THR, 0, c->stream>>>(a, s);
  MD_LAUNCHED(c);
  sym_finish_kernel<Pol, MODEL, MIXED, MODE><<<a.n_it * s.nc, kFinishThreads, 0, c->stream>>>(a, s);
  MD_LAUNCHED(c);
  if (MODE == STAGE_KICK_DRIFT) c->mirror_cur = 1 - c->mirror_cur;
  return MD_OK;
}

template <int MODEL, bool MIXED, int MODE>
int sym_dispatch(md_ctx *c, PairArgs a) {
  if constexpr (MODEL == MD_GRAV3D) {
    if constexpr (MIXED) return launch_sym<Grav3DMixed<4, 256, MODE>, MODEL, true, MODE>(c, a);
    else return launch_sym<Grav3DF64<4, 128, MODE>, MODEL, false, MODE>(c, a);
  } else if constexpr (MODEL == MD_SHEET1D) {
    // registers for 5 CTAs per SM (96, no spills): 1.4% faster than for 4 at N = 262,144
    if constexpr (MIXED) return launch_sym<SheetMixed<8, 256, MODE, 5>, MODEL, true, MODE>(c, a);
    else return launch_sym<SheetF64<4, 128, MODE>, MODEL, false, MODE>(c, a);
  } else if constexpr (!MIXED) {
    // 4 rows per thread: the column butterflies' FP64 adds are shared by twice the pairs
    if constexpr (MODEL == MD_RING) return launch_sym<RingF64<4, 128, MODE>, MODEL, false, MODE>(c, a);
    else return launch_sym<GravF64<4, 128, MODE>, MODEL, false, MODE>(c, a);
  } else if constexpr (MODEL == MD_RING) {
    return launch_sym<RingTC<4, 256, MODE>, MODEL, true, MODE>(c, a);
  } else {
    return launch_sym<GravMixed<8, 256, MODE>, MODEL, true, MODE>(c, a);
  }
}

template <int MODEL, bool MIXED>
int sym_mode(md_ctx *c, int mode, PairArgs a) {
  switch (mode) {
  case STAGE_KICK_DRIFT: return sym_dispatch<MODEL, MIXED, STAGE_KICK_DRIFT>(c, a);
  case STAGE_KICK_ONLY: return sym_dispatch<MODEL, MIXED, STAGE_KICK_ONLY>(c, a);
  default: return sym_dispatch<MODEL, MIXED, STAGE_FORCE_ONLY>(c, a);
  }
}

}  // namespace

// Column partials need U TJ NACC floats, U ~ N^2 / (2 TI TJ): the variant runs
// while they fit in kSymMaxColBytes.
bool sym_applies(const md_ctx *c) {
  if (!c->pt.symmetric) return false;
  int64_t TI, TJ, nacc = c->dim, colbytes;
  if (c->model == MD_HMF) return false;
  if (c->prec == MD_FP64) {
    if (c->pt.r_fp64 != 2) return false;
    TI = 512, TJ = 128, colbytes = 8;
  } else if (c->model == MD_GRAV3D) {
    TI = 512, TJ = 256, colbytes = 4;
  } else if (c->model == MD_SHEET1D) {
    TI = 1024, TJ = 256, colbytes = 4;
  } else if (c->model == MD_RING) {
    if (!c->pt.ring_tc || c->pt.ring_tc == 2 || c->pt.r_mixed == 4) return false;
    TI = 256, TJ = 256, colbytes = 4;
  } else if (c->model == MD_GRAV2D) {
    if (c->pt.r_mixed == 4) return false;
    TI = 1024, TJ = 256, colbytes = 4;
  } else {
    return false;
  }
  const int64_t m = TI / TJ, n_it = (c->N + TI - 1) / TI, n_jt = m * n_it;
  const int64_t U = n_it * n_jt - m * n_it * (n_it - 1) / 2;
  return (size_t)U * TJ * nacc * colbytes <= kSymMaxColBytes;
}

int sym_pair_stage(md_ctx *c, int mode, double kick, double drift, double *fout) {
  PairArgs a{};
  a.kick = kick;
  a.drift = drift;
  a.fout = fout;
  const bool mixed = c->prec == MD_MIXED;
  if (c->model == MD_RING) return mixed ? sym_mode<MD_RING, true>(c, mode, a) : sym_mode<MD_RING, false>(c, mode, a);
  if (c->model == MD_GRAV3D)
    return mixed ? sym_mode<MD_GRAV3D, true>(c, mode, a) : sym_mode<MD_GRAV3D, false>(c, mode, a);
  if (c->model == MD_SHEET1D)
    return mixed ? sym_mode<MD_SHEET1D, true>(c, mode, a) : sym_mode<MD_SHEET1D, false>(c, mode, a);
  return mixed ? sym_mode<MD_GRAV2D, true>(c, mode, a) : sym_mode<MD_GRAV2D, false>(c, mode, a);
}
