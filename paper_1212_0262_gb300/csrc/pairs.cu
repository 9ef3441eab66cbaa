// Ring and 2D self-gravitating models (Sec. 3.2): direct all-pairs forces fused
// with the integrator's kick and drift, and the reverse (adjoint) stages of
// md_grad.
//
// Tiling (after the tile algorithm of Sec. 3.2 / Fig. 1): an i-tile of
// TI = NT*R particles lives in registers (R per thread); j-tiles of TJ particles
// of a position "mirror" are staged in shared memory with cp.async, double
// buffered.  Every i visits every j (Newton's third law is not used, as in the
// paper).  Work is split stream-K style: the U = n_it * n_jt (i-tile, j-tile)
// units in i-major order form P contiguous ranges [U c / P, U (c+1) / P)
// ("virtual CTAs", about four per resident CTA), which the persistent CTAs take
// in increasing order from an atomic counter (take_vcta), so every range holds the
// same number of pair interactions and a CTA that its SM served faster takes more
// ranges.  An i-tile covered by several ranges is finished by the last of them to
// arrive (atomic ticket per i-tile, no waiting), which adds the FP64 partial sums
// in range order: results are deterministic.
//
// Pair arithmetic (d = theta_i - theta_j, r = r_i - r_j):
//   Ring:  f_i = -(1/(2 sqrt2 N)) sum_j sin d / (1 - cos d + eps)^(3/2)
//          (minus the gradient of Eq. 1; Eq. 8 with the sign of the Hamiltonian).
//          sin d comes from the product form of Eq. 9 on (sin, cos) of each
//          angle; 1 - cos d is taken as 2 sin^2(d/2) from (sin, cos) of the half
//          angles, which avoids the cancellation of Eq. 9's denominator for close
//          pairs.  With dd = sin^2(d/2) + eps/2:  f_i = -(1/(8N)) sum S dd^(-3/2).
//   2D:    f_i = -(2/N) sum_j r / (|r|^2 + eps)   (minus the gradient of Eq. 3).
// Adjoint stages add, in the same pass, J(q) v (J = df/dq, v = lambda_p) and
// df/deps:
//   Ring:  (Jv)_i = -(1/(8N)) sum [C dd^(-3/2) - (3/4) S^2 dd^(-5/2)] (v_i - v_j),
//          df_i/deps = (3/(32N)) sum S dd^(-5/2)          (C = cos d)
//   2D:    (Jv)_i = -(2/N) sum [w/s - 2 r (r.w)/s^2],  w = v_i - v_j, s = |r|^2 + eps,
//          df_i/deps = (2/N) sum r / s^2
//   3D:    (Jv)_i = -(1/N) sum [w s^(-3/2) - 3 r (r.w) s^(-5/2)],
//          df_i/deps = (3/(2N)) sum r s^(-5/2)
//   sheets (eps > 0, f_i = -(1/N) sum d s^(-1/2), s = d^2 + eps):
//          (Jv)_i = -(eps/N) sum s^(-3/2) w,  df_i/deps = (1/(2N)) sum d s^(-3/2)
// MIXED: the mirror holds FP32 values, two j's are processed per packed
// f32x2 instruction (FFMA2/FMUL2/FADD2), 1/sqrt and 1/x use the SFU
// (rsqrt.approx / rcp.approx, as the paper uses rsqrt), per-tile sums are FP32
// and are added into FP64 per-particle accumulators once per j-tile
// (Sec. 3.2: FP32 pair force added into a double).  FP64: everything in double,
// with Newton-refined reciprocal square roots and reciprocals.
#include "pairs_impl.cuh"

namespace {

// ============================================================ skeleton =====

// SHARD: the i-tiles cover the rows [a.row0, a.row0 + a.nrow) of a row shard (a.n_it
// tiles of them) against every j of the global mirror; a.row0 is a multiple of TI.
template <class Pol, int MODEL, bool MIXED, int MODE, bool SHARD = false>
__global__ void __launch_bounds__(NT, StreamkMinBlocks<Pol>::value) streamk_kernel(PairArgs a) {
  constexpr int R = Pol::R, TJ = Pol::TJ, NACC = Pol::NACC;
  constexpr int TILE_BYTES = TJ * Pol::JB;
  constexpr int CHUNKS = TILE_BYTES / 16;
  constexpr int64_t TI = (int64_t)NT * R;
  static_assert(TILE_BYTES % 16 == 0, "tile must be a whole number of 16-byte chunks");
  __shared__ __align__(16) unsigned char sbuf[2][TILE_BYTES];
  __shared__ bool s_last;
  __shared__ unsigned s_vc;
  const unsigned char *mir = (const unsigned char *)a.mirror_in;

  auto prefetch = [&](int buf, int64_t jt) {
    const unsigned char *src = mir + jt * (int64_t)TILE_BYTES;
    for (int ch = threadIdx.x; ch < CHUNKS; ch += NT) cp_async16(&sbuf[buf][ch * 16], src + ch * 16);
    cp_async_commit();
  };

  for (;;) {
    const int64_t cta = take_vcta(a.sched, s_vc);  // virtual CTA: its range, slots and tickets
    if (cta >= a.P) break;
    const int64_t u0 = unit_begin(a.U, a.P, cta), u1 = unit_begin(a.U, a.P, cta + 1);
    if (u0 >= u1) continue;
    const int64_t first_row = u0 / a.n_jt;

    typename Pol::State st;
    int64_t it = u0 / a.n_jt, jt = u0 % a.n_jt;
    bool row_from_start = (jt == 0);
    const int64_t ibase = SHARD ? a.row0 : 0;
    int64_t i0 = ibase + it * TI;  // tile base; each thread's rows come from Pol::row_of
    Pol::load(st, a.mirror_in, i0);
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
      const bool diag = Pol::MASK && (j0 < i0 + TI) && (i0 < j0 + TJ);
      if (diag)
        Pol::template tile<true>(st, sbuf[buf], a, i0, j0);
      else
        Pol::template tile<false>(st, sbuf[buf], a, i0, j0);
      __syncthreads();
      jt++;
      const bool row_end = (jt == a.n_jt);
      if (row_end || u + 1 == u1) {
        if (row_end && row_from_start) {
          // this CTA covered the whole i-tile: finish it directly
  #pragma unroll
          for (int r = 0; r < Pol::NR; r++) {
            double ex[NACC];
            Pol::total(st, r, ex);
            const int lr = Pol::row_of(r);  // row offset in the tile, -1: another lane's
            if (lr >= 0) finish<Pol, MODEL, MIXED, MODE, SHARD>(a, i0 + lr, ex);
          }
        } else {
          // partial coverage: publish, and let the last contributor finish
          const int slot = (it == first_row) ? 0 : 1;
          double *sp = a.slots + ((cta * 2 + slot) * NACC) * TI;
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
          const int64_t cf = cta_of_unit(a.U, a.P, it * a.n_jt);
          const int64_t cl = cta_of_unit(a.U, a.P, (it + 1) * a.n_jt - 1);
          if (threadIdx.x == 0) {
            unsigned cnt = atomicAdd(&a.tickets[it], 1u) + 1u;
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
              const int64_t fr = unit_begin(a.U, a.P, c2) / a.n_jt;
              const int sl = (it == fr) ? 0 : 1;
              const double *src = a.slots + ((c2 * 2 + sl) * NACC) * TI;
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
              if (lr >= 0) finish<Pol, MODEL, MIXED, MODE, SHARD>(a, i0 + lr, tot[r]);
            }
            if (threadIdx.x == 0) a.tickets[it] = 0u;
          }
        }
        if (row_end && u + 1 < u1) {
          it++;
          jt = 0;
          row_from_start = true;
          i0 = ibase + it * TI;
          Pol::load(st, a.mirror_in, i0);
        }
      }
    }
  }
  vcta_done(a.sched);
}

// Whole mirror from the FP64 state (and lambda_p for adjoint records), padding
// records in both buffers.
template <int MODEL, bool MIXED, bool ADJ, int FMT>
__global__ void mirror_kernel(const double *__restrict__ q, const double *__restrict__ lp, int64_t N, int64_t Npad,
                              void *m0, void *m1, double eps = 0.0) {
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Npad; i += G) {
    if constexpr (MODEL == MD_SHEET1D) {
      if constexpr (ADJ) {
        const double x = i < N ? q[i] : sheet_pad(eps, MIXED);
        const double v = i < N ? lp[i] : 0.0;
        write_record1_adj<MIXED>(m0, i, x, v);
        if (i >= N && m1) write_record1_adj<MIXED>(m1, i, x, v);
      } else if (i < N) {
        write_record1<MIXED>(m0, i, q[i]);
      } else {
        write_pad1<MIXED>(m0, i, eps);
        if (m1) write_pad1<MIXED>(m1, i, eps);
      }
      continue;
    }
    if constexpr (MODEL == MD_GRAV3D && ADJ) {
      // pads far away (their terms vanish in the pair kernels), lambda_p = 0
      double x[3], v[3];
#pragma unroll
      for (int d = 0; d < 3; d++) {
        x[d] = i < N ? q[d * N + i] : (MIXED ? 3.0e19 : 1.0e150);
        v[d] = i < N ? lp[d * N + i] : 0.0;
      }
      write_record3_adj<MIXED>(m0, i, x, v);
      if (i >= N && m1) write_record3_adj<MIXED>(m1, i, x, v);
      continue;
    }
    if constexpr (MODEL == MD_GRAV3D) {
      if (i < N) {
        write_record3<MIXED>(m0, i, q[i], q[N + i], q[2 * N + i]);
      } else {
        write_pad3<MIXED>(m0, i);
        if (m1) write_pad3<MIXED>(m1, i);
      }
      continue;
    }
    if (i < N) {
      const double y = MODEL == MD_GRAV2D ? q[N + i] : 0.0;
      const double vx = ADJ ? lp[i] : 0.0, vy = (ADJ && MODEL == MD_GRAV2D) ? lp[N + i] : 0.0;
      write_record_fmt<MODEL, MIXED, ADJ, FMT>(m0, i, q[i], y, vx, vy);
    } else {
      write_pad_fmt<MODEL, MIXED, ADJ, FMT>(m0, i);
      if (m1) write_pad_fmt<MODEL, MIXED, ADJ, FMT>(m1, i);
    }
  }
}

// First stage from the cached force: p += kick f; q += drift p; new mirror.
template <int MODEL, bool MIXED, int FMT>
__global__ void kick_drift_cached_kernel(double *__restrict__ q, double *__restrict__ p,
                                         const double *__restrict__ f, int64_t N, double kick,
                                         double drift, void *mirror_out) {
  constexpr int D = dim_of<MODEL>();
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
    if constexpr (MODEL == MD_GRAV3D)
      write_record3<MIXED>(mirror_out, i, x[0], x[1], x[D - 1]);
    else if constexpr (MODEL == MD_SHEET1D)
      write_record1<MIXED>(mirror_out, i, x[0]);
    else
      write_record_fmt<MODEL, MIXED, false, FMT>(mirror_out, i, x[0], x[D - 1], 0.0, 0.0);
  }
}

// ------------------------------------------------------------ host side ---

// The Ring FP32 forward path uses the tensor-core records and policy.
bool ring_tc(const md_ctx *c) { return c->model == MD_RING && c->prec == MD_MIXED && c->pt.ring_tc; }


// Mirror record format of the forward stages: 0 interleaved, 1 Ring tensor-core
// fragments.
int mirror_format(const md_ctx *c) { return ring_tc(c) ? 1 : 0; }

int64_t padded(int64_t N) { return (N + kPadMultiple - 1) / kPadMultiple * kPadMultiple; }

int ensure_mirrors(md_ctx *c, bool adj) {
  const int64_t Np = padded(c->n_total);  // a row shard keeps the whole system's mirror
  // the FP64 record bounds the FP32 one
  const size_t per = c->model == MD_RING      ? (adj ? 48 : 64)  // Ring forward: tensor-core record
                     : c->model == MD_GRAV3D  ? (adj ? 64 : 32)
                     : c->model == MD_SHEET1D ? (adj ? 16 : 8)
                                              : (adj ? 32 : 16);
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

template <class Pol, int MODEL, bool MIXED, int MODE>
int launch_streamk(md_ctx *c, PairArgs a) {
  constexpr int64_t TI = (int64_t)NT * Pol::R;
  auto kern = streamk_kernel<Pol, MODEL, MIXED, MODE>;
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, 0);
  if (occ < 1) occ = 1;
  if (c->pt.ctas_per_sm > 0 && c->pt.ctas_per_sm < occ) occ = c->pt.ctas_per_sm;
  a.N = c->N;
  a.n_it = (c->N + TI - 1) / TI;
  a.n_jt = (c->N + Pol::TJ - 1) / Pol::TJ;
  a.U = a.n_it * a.n_jt;
  const int64_t G = std::min<int64_t>((int64_t)c->nsm * occ, a.U);  // CTAs
  a.P = (int)vcta_count(G, a.U, c->pt.vcta > 0 ? c->pt.vcta : 4);  // virtual CTAs
  int rc = ensure_pair_buffers(c, (int)TI, a.P, Pol::NACC);
  if (rc) return rc;
  a.sched = pair_sched(c);
  a.mirror_in = c->mirror[c->mirror_cur];
  a.mirror_out = c->mirror[1 - c->mirror_cur];
  a.q = c->q;
  a.p = c->p;
  a.epsd = MODEL == MD_RING ? 0.5 * c->eps : c->eps;
  a.slots = c->sk_slots;
  a.tickets = c->sk_tickets;
  kern<<<(int)G, NT, 0, c->stream>>>(a);
  MD_LAUNCHED(c);
  if (MODE == STAGE_KICK_DRIFT || ((MODE == STAGE_ADJOINT || MODE == STAGE_TANGENT) && a.drift != 0.0))
    c->mirror_cur = 1 - c->mirror_cur;
  return MD_OK;
}

template <int MODEL, bool MIXED, int MODE>
int dispatch_forward(md_ctx *c, PairArgs a) {
  if constexpr (MODEL == MD_GRAV3D) {
    if constexpr (MIXED) return launch_streamk<Grav3DMixed<4, 256, MODE>, MODEL, MIXED, MODE>(c, a);
    else return launch_streamk<Grav3DF64<2, 128, MODE>, MODEL, MIXED, MODE>(c, a);
  } else if constexpr (MODEL == MD_SHEET1D) {
    if constexpr (MIXED) return launch_streamk<SheetMixed<8, 256, MODE>, MODEL, MIXED, MODE>(c, a);
    else return launch_streamk<SheetF64<2, 128, MODE>, MODEL, MIXED, MODE>(c, a);
  } else if constexpr (MIXED) {
    if (c->pt.r_mixed == 4) {
      if constexpr (MODEL == MD_RING) return launch_streamk<RingMixed<4, 256, MODE>, MODEL, MIXED, MODE>(c, a);
      else return launch_streamk<GravMixed<4, 256, MODE>, MODEL, MIXED, MODE>(c, a);
    }
    if constexpr (MODEL == MD_RING) {
      if (ring_tc(c)) {
        if (c->pt.ring_tc == 2) return launch_streamk<RingTC<2, 256, MODE>, MODEL, MIXED, MODE>(c, a);
        return launch_streamk<RingTC<4, 256, MODE>, MODEL, MIXED, MODE>(c, a);
      }
      return launch_streamk<RingMixed<8, 256, MODE>, MODEL, MIXED, MODE>(c, a);
    } else {
      return launch_streamk<GravMixed<8, 256, MODE>, MODEL, MIXED, MODE>(c, a);
    }
  } else {
    if (c->pt.r_fp64 == 4) {
      if constexpr (MODEL == MD_RING) return launch_streamk<RingF64<4, 128, MODE>, MODEL, MIXED, MODE>(c, a);
      else return launch_streamk<GravF64<4, 128, MODE>, MODEL, MIXED, MODE>(c, a);
    }
    if constexpr (MODEL == MD_RING) return launch_streamk<RingF64<2, 128, MODE>, MODEL, MIXED, MODE>(c, a);
    else return launch_streamk<GravF64<2, 128, MODE>, MODEL, MIXED, MODE>(c, a);
  }
}

template <int MODEL, bool MIXED>
int dispatch_mode(md_ctx *c, int mode, PairArgs a) {
  switch (mode) {
  case STAGE_KICK_DRIFT: return dispatch_forward<MODEL, MIXED, STAGE_KICK_DRIFT>(c, a);
  case STAGE_KICK_ONLY: return dispatch_forward<MODEL, MIXED, STAGE_KICK_ONLY>(c, a);
  default: return dispatch_forward<MODEL, MIXED, STAGE_FORCE_ONLY>(c, a);
  }
}

template <bool ADJ>
int refresh(md_ctx *c, const double *lp) {
  int rc = ensure_mirrors(c, ADJ);
  if (rc) return rc;
  const int64_t Np = padded(c->N);
  const int threads = 256;
  int64_t blocks = std::min<int64_t>((Np + threads - 1) / threads, (int64_t)c->nsm * 16);
  void *m0 = c->mirror[c->mirror_cur], *m1 = c->mirror[1 - c->mirror_cur];
  const bool mixed = c->prec == MD_MIXED;
  if (c->model == MD_RING) {
    if (mixed && !ADJ && ring_tc(c))
      mirror_kernel<MD_RING, true, false, 1><<<blocks, threads, 0, c->stream>>>(c->q, lp, c->N, Np, m0, m1);
    else if (mixed) mirror_kernel<MD_RING, true, ADJ, 0><<<blocks, threads, 0, c->stream>>>(c->q, lp, c->N, Np, m0, m1);
    else mirror_kernel<MD_RING, false, ADJ, 0><<<blocks, threads, 0, c->stream>>>(c->q, lp, c->N, Np, m0, m1);
  } else if (c->model == MD_GRAV3D) {
    if (mixed) mirror_kernel<MD_GRAV3D, true, ADJ, 0><<<blocks, threads, 0, c->stream>>>(c->q, lp, c->N, Np, m0, m1);
    else mirror_kernel<MD_GRAV3D, false, ADJ, 0><<<blocks, threads, 0, c->stream>>>(c->q, lp, c->N, Np, m0, m1);
  } else if (c->model == MD_SHEET1D) {
    if (mixed)
      mirror_kernel<MD_SHEET1D, true, ADJ, 0><<<blocks, threads, 0, c->stream>>>(c->q, lp, c->N, Np, m0, m1, c->eps);
    else
      mirror_kernel<MD_SHEET1D, false, ADJ, 0><<<blocks, threads, 0, c->stream>>>(c->q, lp, c->N, Np, m0, m1, c->eps);
  } else {
    if (mixed) mirror_kernel<MD_GRAV2D, true, ADJ, 0><<<blocks, threads, 0, c->stream>>>(c->q, lp, c->N, Np, m0, m1);
    else mirror_kernel<MD_GRAV2D, false, ADJ, 0><<<blocks, threads, 0, c->stream>>>(c->q, lp, c->N, Np, m0, m1);
  }
  MD_LAUNCHED(c);
  return MD_OK;
}

// ------------------------------------------------------------ row shards ---
//
// A row shard (md_shard_*) owns rows [row0, row0 + N) of a system of n_total
// particles and keeps the whole position mirror: its stages evaluate the forces on
// its own rows against every j (the one-sided kernel, every ordered pair, as in the
// paper's two-GPU scheme of Sec. 3.2, Fig. 2) and write the new records of its own
// rows; the records of the other rows arrive by the exchange between stages.
// Policies: the default one-sided shape of each model and precision.

// Records of the shard's rows (global index row0 + i) into m0, and the padding
// records past n_total into both buffers.
template <int MODEL, bool MIXED, int FMT>
__global__ void shard_mirror_kernel(const double *__restrict__ q, int64_t n, int64_t row0, int64_t n_total,
                                    int64_t Npad, void *m0, void *m1) {
  const int64_t G = (int64_t)gridDim.x * blockDim.x;
  const int64_t work = n + (Npad - n_total);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < work; i += G) {
    if (i < n) {
      const double y = MODEL == MD_GRAV2D ? q[n + i] : 0.0;
      write_record_fmt<MODEL, MIXED, false, FMT>(m0, row0 + i, q[i], y, 0.0, 0.0);
    } else {
      const int64_t g = n_total + (i - n);
      write_pad_fmt<MODEL, MIXED, false, FMT>(m0, g);
      write_pad_fmt<MODEL, MIXED, false, FMT>(m1, g);
    }
  }
}

template <class Pol, int MODEL, bool MIXED, int MODE>
int launch_streamk_shard(md_ctx *c, PairArgs a) {
  constexpr int64_t TI = (int64_t)NT * Pol::R;
  static_assert(kPadMultiple % TI == 0, "shard rows start on whole i-tiles");
  auto kern = streamk_kernel<Pol, MODEL, MIXED, MODE, true>;
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, 0);
  if (occ < 1) occ = 1;
  if (c->pt.ctas_per_sm > 0 && c->pt.ctas_per_sm < occ) occ = c->pt.ctas_per_sm;
  a.N = c->n_total;
  a.row0 = c->row0;
  a.nrow = c->N;
  a.n_it = (c->N + TI - 1) / TI;
  a.n_jt = (c->n_total + Pol::TJ - 1) / Pol::TJ;
  a.U = a.n_it * a.n_jt;
  const int64_t G = std::min<int64_t>((int64_t)c->nsm * occ, a.U);  // CTAs
  a.P = (int)vcta_count(G, a.U, c->pt.vcta > 0 ? c->pt.vcta : 4);  // virtual CTAs
  int rc = ensure_pair_buffers(c, (int)TI, a.P, Pol::NACC);
  if (rc) return rc;
  a.sched = pair_sched(c);
  a.mirror_in = c->mirror[c->mirror_cur];
  a.mirror_out = c->mirror[1 - c->mirror_cur];
  a.q = c->q;
  a.p = c->p;
  a.epsd = MODEL == MD_RING ? 0.5 * c->eps : c->eps;
  a.slots = c->sk_slots;
  a.tickets = c->sk_tickets;
  kern<<<(int)G, NT, 0, c->stream>>>(a);
  MD_LAUNCHED(c);
  if (MODE == STAGE_KICK_DRIFT) c->mirror_cur = 1 - c->mirror_cur;
  return MD_OK;
}

template <int MODEL, bool MIXED, int MODE>
int dispatch_shard(md_ctx *c, PairArgs a) {
  if constexpr (MODEL == MD_RING) {
    if constexpr (MIXED) {
      if (c->pt.ring_tc) return launch_streamk_shard<RingTC<4, 256, MODE>, MODEL, MIXED, MODE>(c, a);
      return launch_streamk_shard<RingMixed<8, 256, MODE>, MODEL, MIXED, MODE>(c, a);
    } else {
      return launch_streamk_shard<RingF64<2, 128, MODE>, MODEL, MIXED, MODE>(c, a);
    }
  } else {
    if constexpr (MIXED) return launch_streamk_shard<GravMixed<8, 256, MODE>, MODEL, MIXED, MODE>(c, a);
    else return launch_streamk_shard<GravF64<2, 128, MODE>, MODEL, MIXED, MODE>(c, a);
  }
}

// Record format and bytes per particle of a shard's mirror.
int shard_format(const md_ctx *c) { return (c->model == MD_RING && c->prec == MD_MIXED && c->pt.ring_tc) ? 1 : 0; }
size_t shard_record_bytes(const md_ctx *c) {
  const bool mixed = c->prec == MD_MIXED;
  if (c->model == MD_RING) return mixed ? (shard_format(c) == 1 ? 64 : 16) : 32;
  return mixed ? 8 : 16;
}

}  // namespace

int ensure_pair_buffers(md_ctx *c, int TI, int P, int nacc) {
  size_t need_slots = (size_t)P * 2 * nacc * TI * sizeof(double);
  if (need_slots > c->sk_slots_bytes) {
    dev_free(c->sk_slots);
    c->sk_slots = (double *)dev_alloc(need_slots);
    if (!c->sk_slots) {
      c->sk_slots_bytes = 0;
      return set_err(c, MD_ENOMEM, "stream-K slots: %zu bytes", need_slots);
    }
    c->sk_slots_bytes = need_slots;
  }
  // a ticket per i-tile, then the dynamic stream-K counters (pair_sched)
  size_t n_it = (size_t)((c->N + TI - 1) / TI) + 2;
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

int mirror_refresh(md_ctx *c) {
  int rc = refresh<false>(c, nullptr);
  if (rc) return rc;
  c->mirror_valid = true;
  c->mirror_prec = c->prec;
  c->mirror_fmt = mirror_format(c);
  return MD_OK;
}

int adjoint_mirror_refresh(md_ctx *c, const double *lp) {
  c->mirror_valid = false;  // the buffers now hold adjoint records
  return refresh<true>(c, lp);
}

int pair_stage(md_ctx *c, int mode, double kick, double drift, double *fout) {
  if (!c->mirror_valid || c->mirror_prec != c->prec || c->mirror_fmt != mirror_format(c)) {
    int rc = mirror_refresh(c);
    if (rc) return rc;
  }
  if (sym_applies(c)) return sym_pair_stage(c, mode, kick, drift, fout);
  PairArgs a{};
  a.kick = kick;
  a.drift = drift;
  a.fout = fout;
  const bool mixed = c->prec == MD_MIXED;
  if (c->model == MD_RING)
    return mixed ? dispatch_mode<MD_RING, true>(c, mode, a) : dispatch_mode<MD_RING, false>(c, mode, a);
  if (c->model == MD_GRAV3D)
    return mixed ? dispatch_mode<MD_GRAV3D, true>(c, mode, a) : dispatch_mode<MD_GRAV3D, false>(c, mode, a);
  if (c->model == MD_SHEET1D)
    return mixed ? dispatch_mode<MD_SHEET1D, true>(c, mode, a) : dispatch_mode<MD_SHEET1D, false>(c, mode, a);
  return mixed ? dispatch_mode<MD_GRAV2D, true>(c, mode, a) : dispatch_mode<MD_GRAV2D, false>(c, mode, a);
}

template <int MODE>
int reverse_pair_launch(md_ctx *c, PairArgs a) {
  const bool mixed = c->prec == MD_MIXED;
  switch (c->model) {
  case MD_RING:
    if (mixed) return launch_streamk<RingMixedAdj<4, 256, MODE, 3>, MD_RING, true, MODE>(c, a);  // 160 registers
    return launch_streamk<RingF64Adj<2, 128, MODE>, MD_RING, false, MODE>(c, a);
  case MD_GRAV3D:
    if (mixed) return launch_streamk<Grav3DMixedAdj<2, 256, MODE, 4>, MD_GRAV3D, true, MODE>(c, a);  // 128
    return launch_streamk<Grav3DF64Adj<2, 128, MODE>, MD_GRAV3D, false, MODE>(c, a);
  case MD_SHEET1D:
    if (mixed) return launch_streamk<SheetMixedAdj<4, 256, MODE, 4>, MD_SHEET1D, true, MODE>(c, a);  // 124
    return launch_streamk<SheetF64Adj<2, 128, MODE>, MD_SHEET1D, false, MODE>(c, a);
  default:
    // registers for 5 CTAs per SM (96, no spills; 130 and 3 CTAs otherwise): 2% faster gradients
    if (mixed) return launch_streamk<GravMixedAdj<2, 256, MODE, 5>, MD_GRAV2D, true, MODE>(c, a);
    return launch_streamk<GravF64Adj<2, 128, MODE>, MD_GRAV2D, false, MODE>(c, a);
  }
}

int pair_adjoint_stage(md_ctx *c, double b_adj, double b_undo, double drift, double *lq, double *lp,
                       double *epsacc) {
  PairArgs a{};
  a.kick = b_adj;
  a.undo = b_undo;
  a.drift = drift;
  a.lq = lq;
  a.lp = lp;
  a.epsacc = epsacc;
  return reverse_pair_launch<STAGE_ADJOINT>(c, a);
}

int pair_tangent_stage(md_ctx *c, double kick, double drift, double *dq, double *dp) {
  PairArgs a{};
  a.kick = kick;
  a.drift = drift;
  a.lq = dq;
  a.lp = dp;
  return reverse_pair_launch<STAGE_TANGENT>(c, a);
}

int kick_drift_cached(md_ctx *c, double kick, double drift) {
  if (!c->mirror_valid || c->mirror_prec != c->prec || c->mirror_fmt != mirror_format(c)) {
    int rc = mirror_refresh(c);
    if (rc) return rc;
  }
  const int threads = 256;
  int64_t blocks = std::min<int64_t>((c->N + threads - 1) / threads, (int64_t)c->nsm * 16);
  void *mo = c->mirror[1 - c->mirror_cur];
  const bool mixed = c->prec == MD_MIXED;
  if (c->model == MD_RING) {
    if (mixed && ring_tc(c))
      kick_drift_cached_kernel<MD_RING, true, 1><<<blocks, threads, 0, c->stream>>>(c->q, c->p, c->f, c->N, kick, drift, mo);
    else if (mixed) kick_drift_cached_kernel<MD_RING, true, 0><<<blocks, threads, 0, c->stream>>>(c->q, c->p, c->f, c->N, kick, drift, mo);
    else kick_drift_cached_kernel<MD_RING, false, 0><<<blocks, threads, 0, c->stream>>>(c->q, c->p, c->f, c->N, kick, drift, mo);
  } else if (c->model == MD_GRAV3D) {
    if (mixed) kick_drift_cached_kernel<MD_GRAV3D, true, 0><<<blocks, threads, 0, c->stream>>>(c->q, c->p, c->f, c->N, kick, drift, mo);
    else kick_drift_cached_kernel<MD_GRAV3D, false, 0><<<blocks, threads, 0, c->stream>>>(c->q, c->p, c->f, c->N, kick, drift, mo);
  } else if (c->model == MD_SHEET1D) {
    if (mixed) kick_drift_cached_kernel<MD_SHEET1D, true, 0><<<blocks, threads, 0, c->stream>>>(c->q, c->p, c->f, c->N, kick, drift, mo);
    else kick_drift_cached_kernel<MD_SHEET1D, false, 0><<<blocks, threads, 0, c->stream>>>(c->q, c->p, c->f, c->N, kick, drift, mo);
  } else {
    if (mixed) kick_drift_cached_kernel<MD_GRAV2D, true, 0><<<blocks, threads, 0, c->stream>>>(c->q, c->p, c->f, c->N, kick, drift, mo);
    else kick_drift_cached_kernel<MD_GRAV2D, false, 0><<<blocks, threads, 0, c->stream>>>(c->q, c->p, c->f, c->N, kick, drift, mo);
  }
  MD_LAUNCHED(c);
  c->mirror_cur = 1 - c->mirror_cur;
  return MD_OK;
}

int pair_shard_prime(md_ctx *c) {
  if (c->model != MD_RING && c->model != MD_GRAV2D)
    return set_err(c, MD_EINVAL, "row shards: Ring, 2D and HMF systems only");
  int rc = ensure_mirrors(c, false);
  if (rc) return rc;
  const int64_t Np = padded(c->n_total);
  const int threads = 256;
  const int64_t work = c->N + (Np - c->n_total);
  const int64_t blocks = std::min<int64_t>((work + threads - 1) / threads, (int64_t)c->nsm * 16);
  c->mirror_cur = 0;
  void *m0 = c->mirror[0], *m1 = c->mirror[1];
  const bool mixed = c->prec == MD_MIXED;
  if (c->model == MD_RING) {
    if (mixed && shard_format(c) == 1)
      shard_mirror_kernel<MD_RING, true, 1><<<blocks, threads, 0, c->stream>>>(c->q, c->N, c->row0, c->n_total, Np, m0, m1);
    else if (mixed)
      shard_mirror_kernel<MD_RING, true, 0><<<blocks, threads, 0, c->stream>>>(c->q, c->N, c->row0, c->n_total, Np, m0, m1);
    else
      shard_mirror_kernel<MD_RING, false, 0><<<blocks, threads, 0, c->stream>>>(c->q, c->N, c->row0, c->n_total, Np, m0, m1);
  } else {
    if (mixed)
      shard_mirror_kernel<MD_GRAV2D, true, 0><<<blocks, threads, 0, c->stream>>>(c->q, c->N, c->row0, c->n_total, Np, m0, m1);
    else
      shard_mirror_kernel<MD_GRAV2D, false, 0><<<blocks, threads, 0, c->stream>>>(c->q, c->N, c->row0, c->n_total, Np, m0, m1);
  }
  MD_LAUNCHED(c);
  c->mirror_valid = false;  // holds only this shard's rows until the exchange; md_step's refresh must not trust it
  c->mirror_fmt = shard_format(c);
  return MD_OK;
}

int pair_shard_stage(md_ctx *c, int mode, double kick, double drift, double *fout) {
  if (shard_format(c) != c->mirror_fmt)
    return set_err(c, MD_ESTATE, "row shard: the record format changed (ring_tc); call md_shard_begin again");
  PairArgs a{};
  a.kick = kick;
  a.drift = drift;
  a.fout = fout;
  const bool mixed = c->prec == MD_MIXED;
  const bool fo = mode == STAGE_FORCE_ONLY;
  if (c->model == MD_RING) {
    if (mixed) return fo ? dispatch_shard<MD_RING, true, STAGE_FORCE_ONLY>(c, a) : dispatch_shard<MD_RING, true, STAGE_KICK_DRIFT>(c, a);
    return fo ? dispatch_shard<MD_RING, false, STAGE_FORCE_ONLY>(c, a) : dispatch_shard<MD_RING, false, STAGE_KICK_DRIFT>(c, a);
  }
  if (mixed) return fo ? dispatch_shard<MD_GRAV2D, true, STAGE_FORCE_ONLY>(c, a) : dispatch_shard<MD_GRAV2D, true, STAGE_KICK_DRIFT>(c, a);
  return fo ? dispatch_shard<MD_GRAV2D, false, STAGE_FORCE_ONLY>(c, a) : dispatch_shard<MD_GRAV2D, false, STAGE_KICK_DRIFT>(c, a);
}

int pair_shard_segment(md_ctx *c, void **buf, size_t *off, size_t *bytes) {
  static_assert(kPadMultiple == kShardRowAlign, "shard boundaries fall on whole mirror groups and i-tiles");
  const size_t rb = shard_record_bytes(c);
  // the last rank's segment also holds the padding records past n_total
  const int64_t hi = c->shard_rank == c->shard_nranks - 1 ? padded(c->n_total) : c->row0 + c->N;
  *buf = c->mirror[c->mirror_cur];
  *off = (size_t)c->row0 * rb;
  *bytes = (size_t)(hi - c->row0) * rb;
  return MD_OK;
}

extern "C" int md_force_kernel(const md_ctx *c) {
  if (!c) return -1;
  if (c->model == MD_HMF) return MD_KERNEL_HMF;
  if (c->prec != MD_MIXED) return sym_applies(c) ? MD_KERNEL_PAIRS_FP64_SYM : MD_KERNEL_PAIRS_FP64;
  const bool tc = ring_tc(c) && c->pt.r_mixed != 4;
  if (sym_applies(c)) return tc ? MD_KERNEL_PAIRS_TC_SYM : MD_KERNEL_PAIRS_SYM;
  return tc ? MD_KERNEL_PAIRS_TC : MD_KERNEL_PAIRS;
}
