// The PDHG pass of emd_kernels.cuh (same three fused steps, same sums, same decision)
// restructured for sm_103a's copy engine and issue rate:
//
//  * Persistent CTAs (two per SM) walk the tile list.  A producer warp stages each tile's
//    six input planes (u^{k-1}, u^k as x and t, phi^{k-1}, f) by TMA (cp.async.bulk.tensor,
//    one 3D descriptor per gather, zero fill outside the planes) into one of two shared
//    memory stages; eight compute warps consume them.  Full / empty mbarriers per stage
//    hand the stages over, so staging (descriptor and state loads, TMA issue) never
//    holds up the compute warps, which synchronise among themselves on a named barrier.
//  * A warp owns one staged row at a time and a lane owns four consecutive time samples
//    (float4 shared-memory access); the j +- 1 neighbours at lane boundaries come from the
//    adjacent lanes by warp shuffles, the i +- 1 neighbours from the rows above / below.
//  * A CTA accumulates its sums over all its tiles of a gather and flushes them once
//    (FP32 within the warp, FP64 above).  In the per-pass kernel (k_pass_tma) it adds its
//    tile count to the gather's ticket and the CTA that completes the count takes the
//    linesearch decision; in the persistent solve (k_solve_tma) every pass runs inside one
//    launch, each warp adds its totals to the accumulators, and a decider warp of the
//    CTA that owns the gather's first tile waits for the cumulative tile count, decides
//    and publishes the step sizes of the next pass (an epoch counter that the other CTAs
//    wait on).
//  * A tile runs one of three instantiations by edge class: no masks, column steps
//    without masks (tiles at the top or bottom of a gather), or fully masked.
//
// Tile: TI receivers x 120 time samples; staged box (TI + 4) x 128 with the halo of 2
// rows and 4 columns.  Lanes 1..30 own the 120 output columns; lanes 0 and 31 only
// feed their neighbours.
#pragma once

#include "emd_kernels.cuh"

namespace emd {

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Arrive on the barrier and announce `bytes` of TMA traffic for the current phase.
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

// Bound of every wait on another warp or CTA: a wait that outlasts it sets the solve's
// error flag (EMD_ERR_TIMEOUT) and the kernel winds down instead of hanging.
constexpr unsigned long long kSpinLimitNs = 4000000000ull;  // 4 s

// Bounded wait on a barrier phase: false if it did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned n = 0;; ++n) {
    if (mbar_test(bar, parity)) return true;
    if ((n & 63u) == 63u && global_ns() - t0 > kSpinLimitNs) return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void tmap_acquire(const CUtensorMap *map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(map) : "memory");
}

// One box of a 3D tensor (x = time sample, y = receiver, z = plane) into shared memory.
__device__ __forceinline__ void tma_load_3d(float *dst, const CUtensorMap *map, int x, int y,
                                            int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_acquire_int(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Waits until *counter >= target (modulo 2^32: cumulative counters of long solves may
// wrap) or the gather has stopped (*done != 0).  False on timeout.
__device__ __forceinline__ bool wait_counter(const unsigned *counter, unsigned target,
                                             const int *done) {
  const unsigned long long t0 = global_ns();
  for (unsigned n = 0;; ++n) {
    if (static_cast<int>(ld_acquire(counter) - target) >= 0 || ld_acquire_int(done)) return true;
    if ((n & 255u) == 255u && global_ns() - t0 > kSpinLimitNs) return false;
    __nanosleep(64);
  }
}

// Orders this thread's later TMA (async proxy) reads of global memory after the
// ordinary stores of other CTAs that it has acquired.
__device__ __forceinline__ void fence_proxy_async_all() {
  asm volatile("fence.proxy.async;\n" ::: "memory");
}

// The contiguous run of tiles CTA b owns: [lo, hi) with lo = b T / G (T tiles, G CTAs).
// Neighbouring tiles of a gather stay in one CTA (halo rows just staged are still in L2)
// and a CTA meets as few gathers as possible (one flush per gather and pass).
__device__ __forceinline__ int tile_lo(int b, int total, int grid) {
  return static_cast<int>(static_cast<long long>(b) * total / grid);
}

__device__ __forceinline__ void ld4(const float *p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4 *>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}

__device__ __forceinline__ void st4(float *p, const float (&v)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// Tile being staged / consumed in one shared-memory stage, with the per-gather scalars
// the compute warps need (so they make no global loads of their own).
struct StageInfo {
  int gather, k, active, i0, j0, nr, nt, ntp;
  int inside;    // 2: every staged cell away from every grid edge; 1: the staged columns
                 // away from the first / last column (rows may reach an edge); 0: neither
  int need_res;  // this pass's residual sums are read (a stopping test or the last iteration)
  int iso;       // isotropic ground cost (vector shrink in the prox)
  float alpha, coef, theta, inv, fmean, rdx, rdt;
  float *ph_cur, *uxn, *utn;
};

template <int TI>
struct TmaTile {
  static constexpr int W = 128, TJ = 120, R = TI + 4;
  static constexpr int BOX = R * W;      // floats of one staged plane
  static constexpr int STAGE = 6 * BOX;  // floats of one stage
  static constexpr unsigned BYTES = STAGE * 4u;
  static constexpr size_t SMEM = 2u * STAGE * 4u + 128u;  // two stages + alignment slack
};

constexpr int kTmaThreads = kThreads + 32;  // eight compute warps + one producer warp

// Geometry, buffers and stopping-test flag of tile t in pass k (no state read).
template <int TI>
__device__ __forceinline__ void tile_info(const Ctl &c, int t, int k, StageInfo &in) {
  using T = TmaTile<TI>;
  const int g = c.tile_shot[t];
  const Shot &S = c.shots[g];
  const int lt = t - S.tile0;
  in.gather = g;
  in.k = k;
  in.i0 = (lt / S.tiles_j) * TI;
  in.j0 = (lt % S.tiles_j) * T::TJ;
  in.nr = S.nr;
  in.nt = S.nt;
  in.ntp = S.ntp;
  in.rdx = S.rdx;
  in.rdt = S.rdt;
  const bool cols_in = in.j0 >= 5 && in.j0 + 124 < S.nt;
  in.inside = cols_in ? (in.i0 >= 3 && in.i0 + TI + 2 < S.nr ? 2 : 1) : 0;
  in.need_res = (c.tol > 0.0 && (k + 1) % c.check_every == 0) || k + 1 >= c.max_iter;
  in.iso = c.iso;
  in.ph_cur = S.ph[k & 1];
  in.uxn = S.ux[(k + 1) % 3];
  in.utn = S.ut[(k + 1) % 3];
}

// Issues the six TMA box loads of tile `in` (pass in.k) into `dst`, announcing their
// bytes on `full`; an inactive tile completes the barrier phase with no traffic.
template <int TI>
__device__ __forceinline__ void load_tile(const Ctl &c, const StageInfo &in, float *dst,
                                          uint64_t *full) {
  using T = TmaTile<TI>;
  if (!in.active) {
    mbar_arrive_tx(full, 0u);
    return;
  }
  const Shot &S = c.shots[in.gather];
  const int k = in.k;
  const int kp = k == 0 ? 0 : (k - 1) % 3, kc = k % 3;
  const int z[6] = {1 + 2 * kp, 2 + 2 * kp, 1 + 2 * kc, 2 + 2 * kc, 7 + ((k + 1) & 1), 0};
  fence_proxy_async_smem();  // the stage was last written by ordinary stores
  tmap_acquire(&S.tmap);
  mbar_arrive_tx(full, T::BYTES);
#pragma unroll
  for (int a = 0; a < 6; ++a)
    tma_load_3d(dst + a * T::BOX, &S.tmap, in.j0 - 4, in.i0 - 2, z[a], full);
}

// Producer: stage tile t (of any gather) into `dst`, announcing its bytes on `full`,
// with the step sizes and stop flag of the gather's state.  A tile of a gather that has
// already stopped is marked inactive (the barrier phase still completes, with no
// traffic).  kpass >= 0: the pass index of a persistent solve (the state's k may still
// lag it while the previous decision is being taken); kpass < 0: use the state's k.
template <int TI>
__device__ __forceinline__ void stage_tile(const Ctl &c, int t, float *dst, uint64_t *full,
                                           StageInfo &in, int kpass = -1) {
  const State *st = c.states + c.tile_shot[t];
  const int4 h0 = __ldcg(reinterpret_cast<const int4 *>(st));
  const int4 h1 = __ldcg(reinterpret_cast<const int4 *>(st) + 1);
  tile_info<TI>(c, t, kpass >= 0 ? kpass : h0.x, in);
  in.active = !h0.y;
  in.alpha = __int_as_float(h0.z);
  in.coef = __int_as_float(h0.w);
  in.theta = __int_as_float(h1.x);
  in.inv = __int_as_float(h1.y);
  in.fmean = __int_as_float(h1.z);
  load_tile<TI>(c, in, dst, full);
}

// Compute warps: add the CTA's sums over `n` tiles of gather g to the gather's
// accumulators; the CTA that completes the gather's tile count takes the decision.
__device__ __forceinline__ void flush_gather(const Ctl &c, int g, int n, float (&v)[9]) {
  const Shot &S = c.shots[g];
  State *st = c.states + g;
  double *acc = acc_of(c, g);
  block_accumulate<9, true>(v, acc + (blockIdx.x % kSpread) * kAcc);
  __shared__ bool last;
  __threadfence();
  compute_sync<true>();
  if (threadIdx.x == 0)
    last = atomicAdd(&st->ticket, static_cast<unsigned>(n)) + n == static_cast<unsigned>(S.ntiles);
  compute_sync<true>();
  if (last) {
    __threadfence();
    DecidePrep pr;
    if (threadIdx.x < 32) pr = decide_prep(c, st);
    double a_[9];
    gather_totals<9, true>(acc, a_);
    if (threadIdx.x < 32) decide(c, st, pr, a_, g);
    if (threadIdx.x == 0) st->ticket = 0u;
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) v[q] = 0.0f;
}

// The three fused steps of one PDHG iteration on one staged tile (see emd_kernels.cuh):
// stage arrays UAx, UAt (u^{k-1}, then u^{k+1}), UBx, UBt (u^k), PH (phi^{k-1}, then
// phi^k, then q), FF (f, then p); smem row r <-> receiver i0 - 2 + r, column c <->
// time sample j0 - 4 + c.  Adds the tile's sums to v.  All compute threads.
// COLS_IN / ROWS_IN: every staged column / row is away from the grid's edges, so no cell
// needs that boundary mask (the masked instantiations give the same values there); a
// tile at the top or bottom of a gather keeps its column steps mask-free, which took
// 7-9 % off a pass of the larger gathers.  ISO: the isotropic ground cost (vector
// shrink); a template parameter because a per-cell branch on it cost 5 % of the pass.
template <int TI, bool COLS_IN, bool ROWS_IN, bool ISO, int NW = kThreads / 32>
__device__ __forceinline__ void pass_tile(const StageInfo &in, float *stg, int lane, int warp,
                                          float (&v)[9]) {
  using T = TmaTile<TI>;
  constexpr int W = T::W, R = T::R, BOX = T::BOX;
  constexpr unsigned FULL = 0xffffffffu;
  float *UAx = stg, *UAt = stg + BOX, *UBx = stg + 2 * BOX, *UBt = stg + 3 * BOX;
  float *PH = stg + 4 * BOX, *FF = stg + 5 * BOX;
  const int nr = in.nr, nt = in.nt, ntp = in.ntp;
  const float rdx = in.rdx, rdt = in.rdt;
  const float alpha = in.alpha, coef = in.coef, theta = in.theta, inv = in.inv, fmean = in.fmean;
  const int i0 = in.i0;
  const int gj0 = in.j0 - 4 + 4 * lane;  // time index of this lane's first cell
  bool cin[4], ctl[4], ctr[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gj = gj0 + q;
    cin[q] = COLS_IN || (gj >= 0 && gj < nt);
    ctl[q] = COLS_IN || gj > 0;
    ctr[q] = COLS_IN || gj + 1 < nt;
  }
  const bool need_res = in.need_res;
  // lanes 1..30 own the tile's 120 output columns (inside the pitched row)
  const bool own = lane >= 1 && lane <= 30 && gj0 < ntp;
  float *ph_cur = in.ph_cur, *uxn = in.uxn, *utn = in.utn;

  // The row loops below are kept rolled: the code a pass executes once (flush, decision,
  // pass boundary) runs from a cold instruction cache, and the smaller tile code took
  // 3 % off a pass (a loop counter costs less than the misses).
  // ---- phase 1: phi^k = phi^{k-1} + c_k (p_{k-1} + theta_k q_{k-1}) on rows 0..R-2
#pragma unroll 1
  for (int rr = 0; rr < (R - 1 + NW - 1) / NW; ++rr) {
    const int r = warp + NW * rr;
    if (r >= R - 1) break;
    const int gi = i0 - 2 + r;
    const bool rin = ROWS_IN || (gi >= 0 && gi < nr), xl = ROWS_IN || gi > 0;
    const bool xr = ROWS_IN || gi + 1 < nr;
    const int o = r * W + 4 * lane;
    float bx[4], bxn[4], bt[4], ax[4], axn[4], at[4], ph[4], ff[4], res[4];
    ld4(UBx + o, bx);
    ld4(UBx + o + W, bxn);
    ld4(UBt + o, bt);
    ld4(UAx + o, ax);
    ld4(UAx + o + W, axn);
    ld4(UAt + o, at);
    ld4(PH + o, ph);
    ld4(FF + o, ff);
    const float btN = __shfl_down_sync(FULL, bt[0], 1), atN = __shfl_down_sync(FULL, at[0], 1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float bxl = xl ? bx[q] : 0.0f, bxr = xr ? bxn[q] : 0.0f;
      const float axl = xl ? ax[q] : 0.0f, axr = xr ? axn[q] : 0.0f;
      const float btl = ctl[q] ? bt[q] : 0.0f, btr = ctr[q] ? (q < 3 ? bt[q + 1] : btN) : 0.0f;
      const float atl = ctl[q] ? at[q] : 0.0f, atr = ctr[q] ? (q < 3 ? at[q + 1] : atN) : 0.0f;
      const float divB = (bxr - bxl) * rdx + (btr - btl) * rdt;
      const float divA = (axr - axl) * rdx + (atr - atl) * rdt;
      const float p = divB + (ff[q] - fmean);
      const float qv = divB - divA;
      const float phk = ph[q] + coef * (p + theta * qv);
      res[q] = (rin && cin[q]) ? phk : 0.0f;
    }
    st4(PH + o, res);
    if (own && r >= 2 && r < TI + 2 && gi < nr) st4(ph_cur + gi * ntp + gj0, res);
  }
  compute_sync<true, NW>();

  // ---- phase 2: u^{k+1} = shrink(u^k + alpha grad phi^k, alpha) / (1 + eps alpha), rows 1..R-2
#pragma unroll 1
  for (int rr = 0; rr < (R - 2 + NW - 1) / NW; ++rr) {
    const int r = 1 + warp + NW * rr;
    if (r >= R - 1) break;
    const int gi = i0 - 2 + r;
    const bool rin = ROWS_IN || (gi >= 0 && gi < nr), xl = ROWS_IN || gi > 0;
    const int o = r * W + 4 * lane;
    float ph[4], phu[4], bx[4], bt[4], nx[4], nv[4];
    ld4(PH + o, ph);
    ld4(PH + o - W, phu);
    ld4(UBx + o, bx);
    ld4(UBt + o, bt);
    const float phL = __shfl_up_sync(FULL, ph[3], 1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float gx = xl ? (ph[q] - phu[q]) * rdx : 0.0f;
      const float gt = ctl[q] ? (ph[q] - (q == 0 ? phL : ph[q - 1])) * rdt : 0.0f;
      const bool in_ = rin && cin[q];
      float ax_, at_;
      prox_cell(bx[q] + alpha * gx, bt[q] + alpha * gt, alpha, inv, ISO, ax_, at_);
      nx[q] = in_ ? ax_ : 0.0f;
      nv[q] = in_ ? at_ : 0.0f;
    }
    st4(UAx + o, nx);
    st4(UAt + o, nv);
    if (own && r >= 2 && r < TI + 2 && gi < nr) {
      st4(uxn + gi * ntp + gj0, nx);
      st4(utn + gi * ntp + gj0, nv);
    }
  }
  compute_sync<true, NW>();

  // ---- phase 3: p_k = div u^{k+1} + f -> FF, q_k = div(u^{k+1} - u^k) -> PH, rows 1..R-3
#pragma unroll 1
  for (int rr = 0; rr < (R - 3 + NW - 1) / NW; ++rr) {
    const int r = 1 + warp + NW * rr;
    if (r >= R - 2) break;
    const int gi = i0 - 2 + r;
    const bool rin = ROWS_IN || (gi >= 0 && gi < nr), xl = ROWS_IN || gi > 0;
    const bool xr = ROWS_IN || gi + 1 < nr;
    const int o = r * W + 4 * lane;
    float nx[4], nxn[4], nv[4], bx[4], bxn[4], bt[4], ff[4], pp[4], qq[4];
    ld4(UAx + o, nx);
    ld4(UAx + o + W, nxn);
    ld4(UAt + o, nv);
    ld4(UBx + o, bx);
    ld4(UBx + o + W, bxn);
    ld4(UBt + o, bt);
    ld4(FF + o, ff);
    const float nvN = __shfl_down_sync(FULL, nv[0], 1), btN = __shfl_down_sync(FULL, bt[0], 1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float nxl = xl ? nx[q] : 0.0f, nxr = xr ? nxn[q] : 0.0f;
      const float bxl = xl ? bx[q] : 0.0f, bxr = xr ? bxn[q] : 0.0f;
      const float ntl = ctl[q] ? nv[q] : 0.0f, ntr = ctr[q] ? (q < 3 ? nv[q + 1] : nvN) : 0.0f;
      const float btl = ctl[q] ? bt[q] : 0.0f, btr = ctr[q] ? (q < 3 ? bt[q + 1] : btN) : 0.0f;
      const float divN = (nxr - nxl) * rdx + (ntr - ntl) * rdt;
      const float divB = (bxr - bxl) * rdx + (btr - btl) * rdt;
      const bool in_ = rin && cin[q];
      pp[q] = in_ ? divN + (ff[q] - fmean) : 0.0f;
      qq[q] = in_ ? divN - divB : 0.0f;
    }
    st4(FF + o, pp);
    st4(PH + o, qq);
  }
  compute_sync<true, NW>();

  // ---- phase 4: the linesearch / residual / distance sums over the tile's own cells
#pragma unroll 1
  for (int rr = 0; rr < (TI + NW - 1) / NW; ++rr) {
    const int r = 2 + warp + NW * rr;
    if (r >= TI + 2) break;
    const int gi = i0 - 2 + r;
    const bool xl = ROWS_IN || gi > 0;
    const int o = r * W + 4 * lane;
    float pp[4], pu[4], qq[4], qu[4];
    ld4(FF + o, pp);
    ld4(FF + o - W, pu);
    ld4(PH + o, qq);
    ld4(PH + o - W, qu);
    const float pL = __shfl_up_sync(FULL, pp[3], 1), qL = __shfl_up_sync(FULL, qq[3], 1);
    if (own && gi < nr) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (!cin[q]) continue;
        const float gpx = xl ? (pp[q] - pu[q]) * rdx : 0.0f;
        const float gpt = ctl[q] ? (pp[q] - (q == 0 ? pL : pp[q - 1])) * rdt : 0.0f;
        const float gqx = xl ? (qq[q] - qu[q]) * rdx : 0.0f;
        const float gqt = ctl[q] ? (qq[q] - (q == 0 ? qL : qq[q - 1])) * rdt : 0.0f;
        v[0] += pp[q] * pp[q];
        v[1] += pp[q] * qq[q];
        v[2] += qq[q] * qq[q];
        v[3] += gpx * gpx + gpt * gpt;
        v[4] += gpx * gqx + gpt * gqt;
        v[5] += gqx * gqx + gqt * gqt;
      }
      if (need_res) {  // sum |u| is left to the finalize pass, which recomputes it
        float nx[4], nv[4], bx[4], bt[4];
        ld4(UAx + o, nx);
        ld4(UAt + o, nv);
        ld4(UBx + o, bx);
        ld4(UBt + o, bt);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (!cin[q]) continue;
          const float dx_ = nx[q] - bx[q], dt_ = nv[q] - bt[q];
          v[7] += nx[q] * nx[q] + nv[q] * nv[q];
          v[8] += dx_ * dx_ + dt_ * dt_;
        }
      }
    }
  }
}

// pass_tile in the instantiation that tile `in` needs (its ground cost and edge class).
template <int TI, int NW = kThreads / 32>
__device__ __forceinline__ void pass_tile_any(const StageInfo &in, float *stg, int lane, int warp,
                                              float (&v)[9]) {
  if (in.iso) {
    if (in.inside == 2)
      pass_tile<TI, true, true, true, NW>(in, stg, lane, warp, v);
    else if (in.inside == 1)
      pass_tile<TI, true, false, true, NW>(in, stg, lane, warp, v);
    else
      pass_tile<TI, false, false, true, NW>(in, stg, lane, warp, v);
  } else {
    if (in.inside == 2)
      pass_tile<TI, true, true, false, NW>(in, stg, lane, warp, v);
    else if (in.inside == 1)
      pass_tile<TI, true, false, false, NW>(in, stg, lane, warp, v);
    else
      pass_tile<TI, false, false, false, NW>(in, stg, lane, warp, v);
  }
}

// One PDHG pass over every gather's tiles.  Grid: persistent, at most two CTAs per SM;
// CTA b takes the contiguous tiles [tile_lo(b), tile_lo(b + 1)).  Warp 8 produces,
// warps 0..7 compute.
template <int TI, int MINB = 2>
__global__ void __launch_bounds__(kTmaThreads, MINB) k_pass_tma(Ctl c, int total_tiles) {
  using T = TmaTile<TI>;
  extern __shared__ float4 dyn4[];
  float *sbase = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(dyn4) + 127u) & ~static_cast<uintptr_t>(127u));
  __shared__ __align__(8) uint64_t full[2], empty[2];
  __shared__ StageInfo info[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t_lo = tile_lo(blockIdx.x, total_tiles, gridDim.x);
  const int t_hi = tile_lo(blockIdx.x + 1, total_tiles, gridDim.x);

  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], 1);
    mbar_init(&empty[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kThreads / 32) {  // ---- producer warp: one lane stages every tile
    if (lane == 0) {
      int i = 0;
      for (int t = t_lo; t < t_hi; ++t, ++i) {
        const int s = i & 1;
        if (i >= 2 && !mbar_wait(&empty[s], ((i - 2) >> 1) & 1)) {
          atomicExch(c.error, 1);
          break;  // the compute warps time out on `full` in turn
        }
        stage_tile<TI>(c, t, sbase + s * T::STAGE, &full[s], info[s]);
      }
    }
    return;
  }

  // ---- compute warps
  float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int seg = 0;  // tiles of the current gather summed into v
  int i = 0;
  for (int t = t_lo; t < t_hi; ++t, ++i) {
    const int s = i & 1;
    const bool ok = mbar_wait(&full[s], (i >> 1) & 1);
    int bad;
    asm volatile("{\n .reg .pred p, q;\n setp.eq.u32 p, %1, 0;\n"
                 " bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(bad)
                 : "r"(static_cast<unsigned>(ok)), "n"(kThreads)
                 : "memory");
    if (bad) {
      if (threadIdx.x == 0) atomicExch(c.error, 1);
      return;
    }
    const StageInfo in = info[s];
    if (in.active) {
      pass_tile_any<TI>(in, sbase + s * T::STAGE, lane, warp, v);
      ++seg;
      const int tn = t + 1;
      const int gn = tn < t_hi ? c.tile_shot[tn] : -1;
      if (gn != in.gather) {
        flush_gather(c, in.gather, seg, v);
        seg = 0;
      }
    }
    compute_sync<true>();                   // every compute warp is done with stage s
    if (threadIdx.x == 0) mbar_arrive(&empty[s]);  // hand it back to the producer
  }
}

// ---------------------------------------------------------------------------------
// Persistent solve: every pass of the solve in one cooperative launch.
//
// Per gather, `tiles_done` counts finished tiles over all passes and `epoch` counts
// decisions.  A decider warp (the tenth warp of the CTA that owns the gather's first tile)
// waits for tiles_done to reach (k + 1) ntiles, takes decision k and publishes epoch =
// k + 1; it loads the gather's state and prepares the FP64 decision inputs while pass k is
// still being computed, so only the sums are left on the critical path.  The producer
// stages a tile of pass k once the gather's pass k - 1 is complete (tiles_done >= k
// ntiles), which overlaps the first tile's loads with the decision; the compute warps use
// the step sizes only after epoch >= k.  At each pass boundary the compute warps tell the
// producer (mbarrier `go`) whether any gather of this CTA is still running; the producer
// has staged the pass's first tile before it knows, and the compute warps drain it when
// they stop.

constexpr int kSolveThreads = kTmaThreads + 32;  // eight compute, one producer, one decider warp

__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;\n" ::: "memory");
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait until the cumulative counter reaches target (compared modulo 2^32, so long
// solves may wrap it), then an acquire fence.  Spins without sleeping: the one warp that
// calls it has nothing else to do, and a sleep would add its wake-up to the critical path.
// False on timeout.
__device__ __forceinline__ bool wait_count(const unsigned *counter, unsigned target) {
  const unsigned long long t0 = global_ns();
  for (unsigned n = 0;; ++n) {
    if (static_cast<int>(ld_relaxed(counter) - target) >= 0) break;
    if ((n & 255u) == 255u && global_ns() - t0 > kSpinLimitNs) return false;
  }
  fence_acq_rel_gpu();
  return true;
}

// Decider warp: decision k of gather g from its totals, written to the global state from
// registers only (no read of what was just stored: a global load here is a round trip on
// the critical path).  `trials` is the warp's running trial count of the gather.  The
// reported residuals are left to the caller, after the release.
__device__ __forceinline__ Decision decide_publish(const Ctl &c, State *st, const DecidePrep &pr,
                                                   const double (&a_)[9], int g, int &trials) {
  const Decision o = decide_core(c, pr, a_);
  trials += o.trials_now;
  if ((threadIdx.x & 31) != 0) return o;
  st->s_p2 = a_[0];
  st->s_u1 = a_[6];
  st->s_u2 = a_[7];
  st->s_du2 = a_[8];
  st->trials = trials;
  if (o.status == ST_OK) {
    st->alpha = o.alpha;
    st->theta = o.theta;
    st->coef = o.coef;
    st->k = o.k_new;
    st->alpha_f = o.alpha_f;
    st->coef_f = o.coef_f;
    st->theta_f = o.theta_f;
    st->inv_f = o.inv_f;
  } else {
    st->status = o.status;
  }
  write_trace(c, g, pr.k, o, a_[0], pr.fnorm);
  if (o.done) {
    st->done = 1;
    atomicAdd(c.n_done, 1);
  }
  return o;
}

// The CTA that owns tile t when CTA b of `grid` owns [tile_lo(b), tile_lo(b + 1)): the
// largest b with floor(b total / grid) <= t.
__device__ __forceinline__ int tile_owner(int t, int total, int grid) {
  return static_cast<int>((static_cast<long long>(t + 1) * grid - 1) / total);
}

// Compute warps: add the CTA's sums over `n` tiles of gather g to the gather's pass-k
// accumulator set (FP64 reductions in L2), then the tile count with release semantics (it
// also publishes this CTA's tile stores and sums: the barrier gathers them under thread
// 0).  Each warp adds its own FP32 totals (lane q holds value q) to one of the kSpread
// FP64 copies: one conversion and one reduction per warp, and no block-wide FP64 sum
// (whose eight conversions and seven adds, at 64 cycles of the FP64 pipe each, sat on
// the critical path of every pass).
template <int NW>
__device__ __forceinline__ void flush_gather_persistent(const Ctl &c, int g, int n, int k,
                                                        float (&v)[9]) {
  double *acc = acc_of(c, g, k & 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float mine = 0.0f;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const float w = warp_sum(v[q]);
    if (lane == q) mine = w;
  }
  if (lane < 9)
    atomicAdd(acc + ((blockIdx.x * NW + warp) % kSpread) * kAcc + lane, static_cast<double>(mine));
  compute_sync<true, NW>();
  if (threadIdx.x == 0) red_release_add(&c.states[g].tiles_done, static_cast<unsigned>(n));
#pragma unroll
  for (int q = 0; q < 9; ++q) v[q] = 0.0f;
}

// Decider warp: the totals of a gather's kSpread accumulator copies.  Lanes 2n and 2n + 1
// (n < 9) each load half of the copies of value n and sum them pairwise in registers, one
// exchange adds the two halves, and one shuffle per value then gives every lane all nine:
// 8 warp-wide FP64 adds on the critical path instead of 15 (each occupies the FP64 pipe
// for 64 cycles, whatever its active lanes).  Lanes past 17 repeat value 0, so control
// flow stays uniform.
__device__ __forceinline__ void warp_totals(const double *acc, double (&out)[9]) {
  constexpr int H = kSpread / 2;
  static_assert(kSpread % 2 == 0 && (H & (H - 1)) == 0, "pairwise sum over a power of two");
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int n = lane < 18 ? lane >> 1 : 0, h = lane & 1;
  double c[H];
#pragma unroll
  for (int q = 0; q < H; ++q) c[q] = __ldcg(acc + (h * H + q) * kAcc + n);
#pragma unroll
  for (int w = H / 2; w >= 1; w >>= 1)
#pragma unroll
    for (int q = 0; q < w; ++q) c[q] += c[q + w];
  c[0] += __shfl_xor_sync(FULL, c[0], 1);
#pragma unroll
  for (int m = 0; m < 9; ++m) out[m] = __shfl_sync(FULL, c[0], 2 * m);
}

// Decider warp of a persistent solve: decisions k_begin .. k_end - 1 of the gathers g_lo ..
// g_hi for which owns(S) holds.  Decision k of a gather waits until its cumulative count of
// finished work units reaches (k + 1) count(S), sums the pass's accumulators, decides,
// publishes the new state and releases epoch = k + 1.  The state load and the FP64
// preparation overlap the pass; the warp is the only writer of the gather's state.
template <class Owns, class Count>
__device__ __forceinline__ void decider_loop(const Ctl &c, int g_lo, int g_hi, int k_begin,
                                             int k_end, Owns owns, Count count) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  if (c.debug_fault == 2) return;  // test hook: no decision is ever published
  for (int k = k_begin; k < k_end; ++k) {
    bool any = false;
    for (int g = g_lo; g <= g_hi; ++g) {
      const Shot &S = c.shots[g];
      if (!owns(S)) continue;
      State *st = c.states + g;
      if (st->done) continue;
      any = true;
      const DecidePrep pr = decide_prep(c, st);  // overlaps pass k's compute
      int trials = st->trials;
      // every lane waits (a wait run by one lane slows the warp's later shuffles)
      const bool ok = __all_sync(
          FULL, wait_count(&st->tiles_done, static_cast<unsigned>(k + 1) * static_cast<unsigned>(count(S))));
      if (!ok) {
        if (lane == 0) atomicExch(c.error, 1);
        return;
      }
      double a_[9];
      double *acc = acc_of(c, g, k & 1);
      warp_totals(acc, a_);
      const Decision o = decide_publish(c, st, pr, a_, g, trials);
      __syncwarp();  // the new state, before the release
      if (lane == 0) {
        st_release(&st->epoch, static_cast<unsigned>(k + 1));
        if (o.checked) residuals(pr, a_, st->r_feas, st->r_step);
      }
      // pass k + 2 adds into this set again; the release of epoch k + 2 (after decision
      // k + 1) orders these zeros before any of its flushes
#pragma unroll
      for (int q = lane; q < kSpread * kAcc; q += 32) acc[q] = 0.0;
    }
    if (!any) return;
  }
}

// NW compute warps, one producer and one decider warp; NS shared-memory stages (the
// producer keeps up to NS - 1 tiles loading while one is computed).  Runs passes
// [k_begin, k_end) of every gather in the tile list (a batch solved to a tolerance is run
// in chunks, and each chunk's list holds only the gathers still running).
template <int TI, int MINB = 2, int NW = kThreads / 32, int NS = 2>
__global__ void __launch_bounds__((NW + 2) * 32, MINB)
    k_solve_tma(Ctl c, int total_tiles, int k_begin, int k_end) {
  using T = TmaTile<TI>;
  constexpr int NT = NW * 32;  // compute threads
  extern __shared__ float4 dyn4[];
  float *sbase = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(dyn4) + 127u) & ~static_cast<uintptr_t>(127u));
  __shared__ __align__(8) uint64_t full[NS], empty[NS], gob;
  __shared__ StageInfo info[NS];
  __shared__ int go_flag, hot_gather;
  __shared__ float hot[5];  // alpha, coef, theta, 1/(1+eps alpha), fmean of hot_gather
  __shared__ int hot_done;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t_lo = tile_lo(blockIdx.x, total_tiles, gridDim.x);
  const int t_hi = tile_lo(blockIdx.x + 1, total_tiles, gridDim.x);

  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    mbar_init(&gob, 1);
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == NW + 1) {  // ---- decider warp: decisions of the gathers this CTA owns
    decider_loop(
        c, c.tile_shot[t_lo], c.tile_shot[t_hi - 1], k_begin, k_end,
        [&](const Shot &S) {
          return tile_owner(S.tile0, total_tiles, gridDim.x) == static_cast<int>(blockIdx.x);
        },
        [](const Shot &S) { return S.ntiles; });
    return;
  }

  if (warp == NW) {  // ---- producer warp: one lane stages every tile of every pass
    if (lane == 0) {
      int i = 0;
      for (int k = k_begin; k < k_end; ++k) {
        bool first = true;
        for (int t = t_lo; t < t_hi; ++t, ++i) {
          const int s = i % NS;
          if (i >= NS && !mbar_wait(&empty[s], ((i - NS) / NS) & 1)) {
            atomicExch(c.error, 1);
            return;
          }
          const int g = c.tile_shot[t];
          const State *st = c.states + g;
          if (k > 0) {
            const unsigned need = static_cast<unsigned>(k) * static_cast<unsigned>(c.shots[g].ntiles);
            if (!wait_counter(&st->tiles_done, need, &st->done)) {
              atomicExch(c.error, 1);
              return;
            }
            fence_proxy_async_all();  // pass k - 1's stores, by other CTAs, feed these loads
          }
          stage_tile<TI>(c, t, sbase + s * T::STAGE, &full[s], info[s], k);
          if (first) {
            first = false;
            if (!mbar_wait(&gob, (k - k_begin) & 1)) {
              atomicExch(c.error, 1);
              return;
            }
            if (!go_flag) return;
          }
        }
      }
    }
    return;
  }

  // ---- compute warps
  float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int i = 0;
  for (int k = k_begin; k < k_end; ++k) {
    // pass boundary: is any gather of this CTA still running after decision k - 1?  The
    // whole of warp 0 waits (the same loads in every lane): a wait loop run by one lane
    // leaves the warp split, and every later shuffle of it then costs ~10x.
    if (warp == 0) {
      int go = 0;
      bool ok = true;
      int last_g = -1;
      for (int t = t_lo; t < t_hi && ok; ++t) {
        const int g = c.tile_shot[t];
        if (g == last_g) continue;
        last_g = g;
        State *st = c.states + g;
        ok = wait_counter(&st->epoch, static_cast<unsigned>(k), &st->done);
        if (ok && !ld_acquire_int(&st->done)) go = 1;
      }
      ok = __all_sync(0xffffffffu, ok);
      go = __any_sync(0xffffffffu, go);
      if (lane == 0) {
        if (!ok) atomicExch(c.error, 1);
        go_flag = ok ? go : 0;
        hot_gather = -1;
        mbar_arrive(&gob);
      }
    }
    compute_sync<true, NW>();
    if (!go_flag) {  // stop: drain the first tile the producer staged for this pass
      (void)mbar_wait(&full[i % NS], (i / NS) & 1);
      return;
    }
    int seg = 0;  // tiles of the current gather summed into v
    for (int t = t_lo; t < t_hi; ++t, ++i) {
      const int s = i % NS;
      const bool ok = mbar_wait(&full[s], (i / NS) & 1);
      int bad;
      asm volatile("{\n .reg .pred p, q;\n setp.eq.u32 p, %1, 0;\n"
                   " bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
                   : "=r"(bad)
                   : "r"(static_cast<unsigned>(ok)), "n"(NT)
                   : "memory");
      if (bad) {
        if (threadIdx.x == 0) atomicExch(c.error, 1);
        return;
      }
      StageInfo in = info[s];
      if (in.gather != hot_gather) {  // this pass's step sizes of the tile's gather
        compute_sync<true, NW>();
        if (threadIdx.x == 0) {
          const State *st = c.states + in.gather;
          const int4 h0 = __ldcg(reinterpret_cast<const int4 *>(st));
          const int4 h1 = __ldcg(reinterpret_cast<const int4 *>(st) + 1);
          hot_done = h0.y;
          hot[0] = __int_as_float(h0.z);
          hot[1] = __int_as_float(h0.w);
          hot[2] = __int_as_float(h1.x);
          hot[3] = __int_as_float(h1.y);
          hot[4] = __int_as_float(h1.z);
          hot_gather = in.gather;
        }
        compute_sync<true, NW>();
      }
      if (!hot_done) {
        in.alpha = hot[0];
        in.coef = hot[1];
        in.theta = hot[2];
        in.inv = hot[3];
        in.fmean = hot[4];
        pass_tile_any<TI, NW>(in, sbase + s * T::STAGE, lane, warp, v);
        ++seg;
        const int tn = t + 1;
        const int gn = tn < t_hi ? c.tile_shot[tn] : -1;
        if (gn != in.gather) {
          flush_gather_persistent<NW>(c, in.gather, seg, k, v);
          seg = 0;
        }
      }
      compute_sync<true, NW>();                      // every compute warp is done with stage s
      if (threadIdx.x == 0) mbar_arrive(&empty[s]);  // hand it back to the producer
    }
  }
}
}  // namespace emd
