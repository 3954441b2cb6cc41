// The PDHG pass of emd_kernels.cuh (the same three fused steps, the same sums and the same
// decision) as a march over receiver rows.  A warp owns a strip of 120 time samples (staged
// 128: four halo samples on each side; lanes 1..30 own four consecutive samples each, lanes
// 0 and 31 only feed their neighbours) over a segment of receivers, and walks it one receiver
// row at a time.  The steps of an iteration reach the next row only through i -+ 1, so the
// rows behind the front stay in registers: when row r arrives,
//   - the extrapolated flux w = u^k + theta (u^k - u^{k-1}) of row r gives the part of
//     phi^k of row r that needs nothing below it, and completes phi^k of row r - 1 (whose
//     x-divergence needs w of row r);
//   - u^{k+1} of row r - 1 follows (prox: phi^k of rows r - 1 and r - 2);
//   - p_k = div u^{k+1} + f and q_k = div(u^{k+1} - u^k) of row r - 2 are completed with the
//     x-divergence term of row r - 1, and the linesearch sums of row r - 2 are taken (their
//     gradients need row r - 3).
// Time neighbours j -+ 1 come from the adjacent lanes by shuffles.  There is no shared-memory
// round trip and no barrier between the steps: each warp runs on its own and meets the
// others only at a gather's pass boundary (its cumulative count of finished units, then the
// decision's epoch), as in k_solve_tma, whose decider warp is reused.  Rows arrive through a
// per-warp ring of D rows: every lane copies its own 16 bytes of each of the six input planes
// (cp.async, zero fill outside the gather) D rows ahead, and reads only what it copied, so
// the ring needs no barrier.  (A ring of TMA boxes, one box per plane and ring slot, was
// bound by the copy engine's rate of about 4.6 boxes per microsecond per SM at 0.5-1 KB a box
// and ran 3.7-4.7 times slower than the tile pass; it is not built.)
//
// Sums: FP32 within a lane over at most kFoldRows owned rows, then a warp sum per value
// folded into an FP64 accumulator (lane q holds value q); at the end of every unit the FP64
// values go to the gather's accumulators by FP64 atomics.
#pragma once

#include "emd_pass_tma.cuh"

namespace emd {

constexpr int kMarchW = 128;    // staged time samples of a strip
constexpr int kMarchTJ = 120;   // owned time samples of a strip
constexpr int kFoldRows = 32;   // owned rows summed in FP32 before a fold into FP64
constexpr int kMarchMinSeg = 8; // fewest receivers in a segment (each carries a 4-row halo)

// Per-warp shared memory of the march: a ring of D rows of the six input planes, and three
// rows of scratch for values carried two or three rows back.  Every lane copies, reads and
// writes only its own 16 bytes of each row, so the ring needs no barrier of any kind.
template <int D>
struct MarchRing {
  static constexpr int ROW = 6 * kMarchW;           // floats of one staged row (six planes)
  static constexpr int SCRATCH = 3 * kMarchW;       // phi^k of row r - 2, p_k and q_k of row r - 3
  static constexpr int WARP = D * ROW + SCRATCH;    // floats per warp
};

// The unit a warp marches: geometry, planes and this pass's step sizes.
struct MarchUnit {
  int i0, h, j0, nr, nt, ntp;
  bool need_res;
  float alpha, coef, theta, inv, fmean, rdx, rdt;
  const float *ax, *at, *bx, *bt, *ph_prev, *f;  // u^{k-1} (x, t), u^k (x, t), phi^{k-1}, f
  float *ph_cur, *uxn, *utn;                     // phi^k, u^{k+1} (x, t)
};

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// This lane's 16 bytes of staged row r (receiver i0 - 2 + r) of all six planes into ring row
// `dst` (zero fill outside the gather's rows and pitched columns), as one copy group; a row
// past the unit's end commits an empty group, so that every row owns exactly one group.
template <int D>
__device__ __forceinline__ void march_issue(const MarchUnit &m, int r, float *ring) {
  const int lane = threadIdx.x & 31;
  const int gi = m.i0 - 2 + r, gj0 = m.j0 - 4 + 4 * lane;
  if (r < m.h + 4) {
    float *dst = ring + (r % D) * MarchRing<D>::ROW + 4 * lane;
    const bool ok = gi >= 0 && gi < m.nr && gj0 >= 0 && gj0 < m.ntp;
    const size_t o = ok ? static_cast<size_t>(gi) * m.ntp + gj0 : 0;
    cp_async16(dst, m.ax + o, ok);
    cp_async16(dst + kMarchW, m.at + o, ok);
    cp_async16(dst + 2 * kMarchW, m.bx + o, ok);
    cp_async16(dst + 3 * kMarchW, m.bt + o, ok);
    cp_async16(dst + 4 * kMarchW, m.ph_prev + o, ok);
    cp_async16(dst + 5 * kMarchW, m.f + o, ok);
  }
  cp_async_commit();
}

// Issues the unit's first D rows (one group each).
template <int D>
__device__ __forceinline__ void march_prefetch(const MarchUnit &m, float *ring) {
#pragma unroll
  for (int r = 0; r < D; ++r) march_issue<D>(m, r, ring);
}

// A compile-time bool as a value (selects a lambda's instantiation).
template <bool B>
struct BoolConst {
  static constexpr bool value = B;
};

// Warp sums of the nine FP32 lane sums added to the FP64 fold (lane q holds value q).
__device__ __forceinline__ void march_fold(float (&v)[9], double &mine) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    if (q == 6) continue;  // sum |u| is left to the finalize pass
    const float w = warp_sum(v[q]);
    if (lane == q) mine += static_cast<double>(w);
    v[q] = 0.0f;
  }
}

// One unit of pass k (its first D rows already issued into `ring`).  Adds the unit's sums to
// v / mine.  Every x-divergence is formed as the difference of the two face fluxes first and
// scaled after (as the tile passes do), so smooth flux fields lose no accuracy to it.
template <int D, bool COLS_IN, bool ISO>
__device__ __forceinline__ void march_unit(const MarchUnit &m, float *ring, float (&v)[9],
                                           double &mine) {
  using RG = MarchRing<D>;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nrows = m.h + 4;
  const int nr = m.nr, nt = m.nt, ntp = m.ntp;
  const float rdx = m.rdx, rdt = m.rdt, al = m.alpha, cf = m.coef, th = m.theta, inv = m.inv;
  const float fm = m.fmean, cfx = m.coef * m.rdx;
  const int gj0 = m.j0 - 4 + 4 * lane;  // time index of this lane's first sample
  bool cin[4], ctl[4], ctr[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gj = gj0 + q;
    cin[q] = COLS_IN || (gj >= 0 && gj < nt);
    ctl[q] = COLS_IN || gj > 0;
    ctr[q] = COLS_IN || gj + 1 < nt;
  }
  const bool own = lane >= 1 && lane <= 30 && gj0 < ntp;
  float *scr = ring + D * RG::ROW + 4 * lane;  // this lane's scratch: phi^k (r - 2), p, q (r - 3)
  // values of the rows above the front (see the file header)
  float xc[4], wxc[4];         // row r - 1: phi^{k-1} + c (f - mean + div_t w); w's x flux
  float bxP[4], btP[4], fbP[4];  // row r - 1: u^k, f - mean
  float pT[4], qT[4];          // row r - 2: f - mean + div_t u^{k+1}; div_t(u^{k+1} - u^k)
  float nxc[4], dxc[4];        // row r - 2: u^{k+1} x flux and its step
#pragma unroll
  for (int q = 0; q < 4; ++q)
    xc[q] = wxc[q] = bxP[q] = btP[q] = fbP[q] = pT[q] = qT[q] = nxc[q] = dxc[q] = 0.0f;
  int folded = 0;  // owned rows summed into v since the last fold

  // Row r's work.  FAST: a row whose three rows in flight (r, r - 1, r - 2) all lie inside
  // the gather away from receiver 0, and whose row r - 2 is owned -- every row condition
  // holds, so that instantiation carries no row masks or branches (most rows of a unit).
  auto row_step = [&](int r, auto fast) {
    constexpr bool FAST = decltype(fast)::value;
    const float *row = ring + (r % D) * RG::ROW + 4 * lane;
    const int gi = m.i0 - 2 + r;  // receiver of row r
    // ---- row r: w = u^k + theta (u^k - u^{k-1}); x = phi^{k-1} + c (f - mean + div_t w)
    float ax[4], at[4], bx[4], bt[4], ph[4], ff[4], wx[4], wt[4], fb[4], xn[4];
    ld4(row, ax);
    ld4(row + kMarchW, at);
    ld4(row + 2 * kMarchW, bx);
    ld4(row + 3 * kMarchW, bt);
    ld4(row + 4 * kMarchW, ph);
    ld4(row + 5 * kMarchW, ff);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      wx[q] = fmaf(th, bx[q] - ax[q], bx[q]);
      wt[q] = fmaf(th, bt[q] - at[q], bt[q]);
      fb[q] = ff[q] - fm;
    }
    const float wtN = __shfl_down_sync(FULL, wt[0], 1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float wtr = ctr[q] ? (q < 3 ? wt[q + 1] : wtN) : 0.0f, wtl = ctl[q] ? wt[q] : 0.0f;
      xn[q] = fmaf(cf, fb[q] + (wtr - wtl) * rdt, ph[q]);
    }
    if (FAST || r >= 1) {
      // ---- phi^k of row r - 1: x + c (w_x(r) - w_x(r - 1)) / dx
      const int g1 = gi - 1;
      const bool rin1 = FAST || (g1 >= 0 && g1 < nr), xl1 = FAST || g1 > 0, xr1 = FAST || gi < nr;
      const bool own1 = FAST || (r - 1 >= 2 && r - 1 < m.h + 2);
      float phk[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        phk[q] = (rin1 && cin[q]) ? fmaf(cfx, (xr1 ? wx[q] : 0.0f) - (xl1 ? wxc[q] : 0.0f), xc[q]) : 0.0f;
      if (own && own1) st4(m.ph_cur + g1 * ntp + gj0, phk);
      if (FAST || r >= 2) {
        // ---- u^{k+1} of row r - 1 (prox; the x gradient reaches back to row r - 2)
        float phk2[4];
        ld4(scr, phk2);
        const float phL = __shfl_up_sync(FULL, phk[3], 1);
        float nx[4], nv[4], ddx[4], ddt[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float gx = xl1 ? (phk[q] - phk2[q]) * rdx : 0.0f;
          const float gt = ctl[q] ? (phk[q] - (q == 0 ? phL : phk[q - 1])) * rdt : 0.0f;
          float a_, b_;
          prox_cell(fmaf(al, gx, bxP[q]), fmaf(al, gt, btP[q]), al, inv, ISO, a_, b_);
          const bool in_ = rin1 && cin[q];
          nx[q] = in_ ? a_ : 0.0f;
          nv[q] = in_ ? b_ : 0.0f;
          ddx[q] = nx[q] - bxP[q];
          ddt[q] = nv[q] - btP[q];
        }
        if (own && own1) {
          st4(m.uxn + g1 * ntp + gj0, nx);
          st4(m.utn + g1 * ntp + gj0, nv);
          if (m.need_res) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (!cin[q]) continue;
              v[7] = fmaf(nx[q], nx[q], fmaf(nv[q], nv[q], v[7]));
              v[8] = fmaf(ddx[q], ddx[q], fmaf(ddt[q], ddt[q], v[8]));
            }
          }
        }
        const float nvN = __shfl_down_sync(FULL, nv[0], 1), dtN = __shfl_down_sync(FULL, ddt[0], 1);
        // ---- p_k, q_k of row r - 2 (x-divergence from u^{k+1} of rows r - 1 and r - 2)
        const int g2 = gi - 2;
        const bool rin2 = FAST || (g2 >= 0 && g2 < nr), xl2 = FAST || g2 > 0;
        float pc[4], qc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const bool in2 = (FAST || r >= 3) && rin2 && cin[q];
          pc[q] = in2 ? fmaf(rdx, nx[q] - (xl2 ? nxc[q] : 0.0f), pT[q]) : 0.0f;
          qc[q] = in2 ? fmaf(rdx, ddx[q] - (xl2 ? dxc[q] : 0.0f), qT[q]) : 0.0f;
          const float ntr = ctr[q] ? (q < 3 ? nv[q + 1] : nvN) : 0.0f, ntl = ctl[q] ? nv[q] : 0.0f;
          const float dtr = ctr[q] ? (q < 3 ? ddt[q + 1] : dtN) : 0.0f, dtl = ctl[q] ? ddt[q] : 0.0f;
          pT[q] = fbP[q] + (ntr - ntl) * rdt;  // row r - 1, completed by the next row
          qT[q] = (dtr - dtl) * rdt;
          nxc[q] = nx[q];
          dxc[q] = ddx[q];
        }
        if (FAST || (r >= 4 && r - 2 < m.h + 2)) {
          // ---- the linesearch sums of row r - 2 (gradients back to row r - 3)
          float p1[4], q1[4];
          ld4(scr + kMarchW, p1);
          ld4(scr + 2 * kMarchW, q1);
          const float pL = __shfl_up_sync(FULL, pc[3], 1), qL = __shfl_up_sync(FULL, qc[3], 1);
          if (own) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (!cin[q]) continue;
              const float gpx = xl2 ? (pc[q] - p1[q]) * rdx : 0.0f;
              const float gpt = ctl[q] ? (pc[q] - (q == 0 ? pL : pc[q - 1])) * rdt : 0.0f;
              const float gqx = xl2 ? (qc[q] - q1[q]) * rdx : 0.0f;
              const float gqt = ctl[q] ? (qc[q] - (q == 0 ? qL : qc[q - 1])) * rdt : 0.0f;
              v[0] = fmaf(pc[q], pc[q], v[0]);
              v[1] = fmaf(pc[q], qc[q], v[1]);
              v[2] = fmaf(qc[q], qc[q], v[2]);
              v[3] = fmaf(gpx, gpx, fmaf(gpt, gpt, v[3]));
              v[4] = fmaf(gpx, gqx, fmaf(gpt, gqt, v[4]));
              v[5] = fmaf(gqx, gqx, fmaf(gqt, gqt, v[5]));
            }
          }
          if (++folded == kFoldRows) {
            march_fold(v, mine);
            folded = 0;
          }
        }
        st4(scr + kMarchW, pc);  // p_k, q_k of row r - 2: row r - 3 for the next row
        st4(scr + 2 * kMarchW, qc);
      }
      st4(scr, phk);  // phi^k of row r - 1: row r - 2 for the next row
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      xc[q] = xn[q];
      wxc[q] = wx[q];
      bxP[q] = bx[q];
      btP[q] = bt[q];
      fbP[q] = fb[q];
    }
  };

  // rows whose r, r - 1, r - 2 lie in the gather with r - 2 > 0 and an owned r - 2
  const int fast_lo = max(4, 5 - m.i0), fast_hi = min(m.h + 2, nr - m.i0 + 1);
  // Fast rows go two per trip, so the values carried from one row to the next change
  // registers between the two steps instead of being copied back after every row.
  int r = 0;
#pragma unroll 1
  while (r < nrows) {
    if (r >= fast_lo && r + 1 <= fast_hi) {
      cp_async_wait<D - 1>();  // row r's group has landed (later rows may still be in flight)
      row_step(r, BoolConst<true>{});
      march_issue<D>(m, r + D, ring);  // row r's ring row is free: stage row r + D into it
      cp_async_wait<D - 1>();
      row_step(r + 1, BoolConst<true>{});
      march_issue<D>(m, r + 1 + D, ring);
      r += 2;
    } else {
      cp_async_wait<D - 1>();
      row_step(r, BoolConst<false>{});
      march_issue<D>(m, r + D, ring);
      r += 1;
    }
  }
  march_fold(v, mine);
}

// march_unit in the instantiation that the unit needs (ground cost, column edge class).
template <int D>
__device__ __forceinline__ void march_unit_any(const MarchUnit &m, bool iso, float *ring,
                                               float (&v)[9], double &mine) {
  const bool cols_in = m.j0 >= 5 && m.j0 + 124 < m.nt;
  if (iso) {
    if (cols_in)
      march_unit<D, true, true>(m, ring, v, mine);
    else
      march_unit<D, false, true>(m, ring, v, mine);
  } else {
    if (cols_in)
      march_unit<D, true, false>(m, ring, v, mine);
    else
      march_unit<D, false, false>(m, ring, v, mine);
  }
}

// A gather's pass-k sums of this warp (folded into `mine`) to the gather's accumulators, then
// its count of finished units with release semantics (it publishes the warp's stores and sums).
__device__ __forceinline__ void march_flush(const Ctl &c, int g, int n, int k, double &mine, int wid) {
  const int lane = threadIdx.x & 31;
  double *acc = acc_of(c, g, k & 1);
  if (lane < 9 && lane != 6) atomicAdd(acc + (wid % kSpread) * kAcc + lane, mine);
  mine = 0.0;
  __syncwarp();
  if (lane == 0) red_release_add(&c.states[g].tiles_done, static_cast<unsigned>(n));
}

// The run (index into c.march_run) whose units contain unit u: the last run whose first
// unit is <= u (runs are in march order).
__device__ __forceinline__ int march_find(const Ctl &c, int u) {
  int lo = 0, hi = c.march_nrun - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (c.shots[c.march_run[mid]].unit0 <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Persistent solve by marching warps: passes [k_begin, k_end) of every running gather, in one
// cooperative launch.  A gather's work is cut into units -- one segment of seg_h receivers of
// one 120-sample strip -- ordered segment by segment with the strip index fastest, and the
// running gathers' units are laid end to end (total_units per pass).  Marching warp x of the
// T in the grid takes units x, x + T, x + 2T, ...: at every step the warps march horizontally
// adjacent strips of the same segment side by side, so the DRAM bursts their halo columns
// share are fetched once, and each gather's units of a pass sit at the same position of
// every warp's sequence, so gathers pass through the grid one behind the other without a
// grid-wide wait.  NW marching warps and one decider warp per CTA; a ring of D rows in flight
// per warp.
template <int NW, int D, int MINB>
__global__ void __launch_bounds__((NW + 1) * 32, MINB)
    k_solve_march(Ctl c, int total_units, int k_begin, int k_end) {
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ float4 dyn4[];
  float *sbase = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(dyn4) + 127u) & ~static_cast<uintptr_t>(127u));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int T = gridDim.x * NW;  // marching warps in the grid

  if (warp == NW) {  // ---- decider warp: decisions of the gathers the host assigned to this CTA
    decider_loop(
        c, 0, c.march_run[c.march_nrun - 1], k_begin, k_end,
        [&](const Shot &S) { return S.march_owner == static_cast<int>(blockIdx.x); },
        [](const Shot &S) { return S.nunits; });
    return;
  }

  // ---- marching warp
  float *ring = sbase + warp * MarchRing<D>::WARP;
  const int wid = blockIdx.x * NW + warp;
  if (wid >= total_units) return;
  const int run_first = march_find(c, wid);
  float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  double mine = 0.0;
  for (int k = k_begin; k < k_end; ++k) {
    bool any = false;
    int run = run_first;
    for (int u = wid; u < total_units; u += T) {
      while (run + 1 < c.march_nrun && c.shots[c.march_run[run + 1]].unit0 <= u) ++run;
      const int g = c.march_run[run];
      const Shot &S = c.shots[g];
      State *sp = c.states + g;
      // pass k - 1 of the gather is complete (its rows feed these copies); every lane waits
      bool ok = __all_sync(FULL, wait_counter(&sp->tiles_done,
                                              static_cast<unsigned>(k) * static_cast<unsigned>(S.nunits),
                                              &sp->done));
      if (!ok) {
        if (lane == 0) atomicExch(c.error, 1);
        return;
      }
      if (__shfl_sync(FULL, ld_acquire_int(&sp->done), 0)) continue;  // stopped
      const int lu = u - S.unit0, seg = lu / S.strips;
      const int kp = k == 0 ? 0 : (k - 1) % 3, kc = k % 3;
      MarchUnit m;
      m.i0 = seg * S.seg_h;
      m.h = min(S.seg_h, S.nr - m.i0);
      m.j0 = (lu - seg * S.strips) * kMarchTJ;
      m.nr = S.nr;
      m.nt = S.nt;
      m.ntp = S.ntp;
      m.rdx = S.rdx;
      m.rdt = S.rdt;
      m.ax = S.ux[kp];
      m.at = S.ut[kp];
      m.bx = S.ux[kc];
      m.bt = S.ut[kc];
      m.ph_prev = S.ph[(k + 1) & 1];
      m.f = S.f;
      m.ph_cur = S.ph[k & 1];
      m.uxn = S.ux[(k + 1) % 3];
      m.utn = S.ut[(k + 1) % 3];
      m.need_res = (c.tol > 0.0 && (k + 1) % c.check_every == 0) || k + 1 >= c.max_iter;
      march_prefetch<D>(m, ring);  // the unit's first rows load while decision k - 1 is awaited
      ok = __all_sync(FULL, wait_counter(&sp->epoch, static_cast<unsigned>(k), &sp->done));
      if (!ok) {
        cp_async_wait<0>();
        if (lane == 0) atomicExch(c.error, 1);
        return;
      }
      const int4 h0 = __ldcg(reinterpret_cast<const int4 *>(sp));
      const int4 h1 = __ldcg(reinterpret_cast<const int4 *>(sp) + 1);
      if (__shfl_sync(FULL, h0.y, 0)) {  // decision k - 1 stopped the gather
        cp_async_wait<0>();               // let the staged rows land unused
        continue;
      }
      any = true;
      m.alpha = __int_as_float(h0.z);
      m.coef = __int_as_float(h0.w);
      m.theta = __int_as_float(h1.x);
      m.inv = __int_as_float(h1.y);
      m.fmean = __int_as_float(h1.z);
      march_unit_any<D>(m, c.iso != 0, ring, v, mine);
      march_flush(c, g, 1, k, mine, wid);
    }
    if (!any) {
      cp_async_wait<0>();
      return;  // every gather this warp marches has stopped
    }
  }
  cp_async_wait<0>();
}

}  // namespace emd
