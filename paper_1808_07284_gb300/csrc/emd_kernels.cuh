// Device code of the GB300 dynamic-formulation EMD solver (PDHG with linesearch).
//
// One PDHG iteration of Algorithm 1 is ONE fused stencil pass over the gather.  Pass k:
//   (1) finishes iteration k-1's dual ascent (Sec. 2.2, dual update):
//         phi^k = phi^{k-1} + c_k (p_{k-1} + theta_k q_{k-1}),  c_k = delta alpha_k,
//       where p_{k-1} = div u^k + f and q_{k-1} = div(u^k - u^{k-1}), so that
//       div ubar + f = p + theta q with ubar = u^k + theta (u^k - u^{k-1});
//   (2) takes iteration k's primal prox (Sec. 2.2, primal update):
//         u^{k+1} = shrink(u^k + alpha_k grad phi^k, alpha_k) / (1 + eps alpha_k);
//   (3) accumulates the inner products the linesearch of iteration k needs.  With the
//       Euclidean norm, a trial step a gives dphi(a) = delta a (p_k + s q_k), s = a/alpha_k,
//       so the test  sqrt(delta) a ||grad dphi|| <= zeta ||dphi||  reads
//         delta a^2 (G_pp + 2 s G_pq + s^2 G_qq) <= zeta^2 (P_pp + 2 s P_pq + s^2 P_qq)
//       with six sums that do not depend on a.  One pass therefore settles every
//       backtracking trial of Algorithm 1 exactly; the trial loop runs on scalars.
//       The same pass sums the stopping residual and the distance of u^{k+1}.
// In the per-pass kernels the last CTA of each gather (atomic ticket) reduces the FP64
// accumulators and takes the linesearch decision, writing (alpha_{k+1}, theta_{k+1},
// c_{k+1}) for pass k+1; the persistent solve (emd_pass_tma.cuh) has a decider warp.
//
// Tiles: TI rows (receivers) x TJ = W - 8 columns (time) per CTA, staged in shared
// memory with a 2-row / 4-column halo on every side (the dependency cone of the three
// fused steps), loaded with 16-byte cp.async and zero fill outside the pitched planes.
// Iterates are FP32; per-thread partial sums are FP32 over a handful of cells and
// one warp, everything above a warp is FP64 (FP64 atomics into L2).
#pragma once

#include <cuda.h>  // CUtensorMap (the TMA descriptor type); no driver API call is made here
#include <cuda_runtime.h>

#include <cstdint>

namespace emd {

constexpr int kThreads = 256;
constexpr int kAcc = 12;  // FP64 accumulators per gather

// Per-gather constants of one solve (device copy in the workspace).  A gather's nine
// pitched planes sit at a uniform stride: z = 0 f, 1 + 2m ux[m], 2 + 2m ut[m], 7 + m ph[m];
// `tmap` describes them as one 3D tensor {ntp, nr, 9} for the TMA pass.
struct Shot {
  CUtensorMap tmap;                 // TMA descriptor of the nine planes (TMA pass only)
  const float *p_obs, *p_pred;      // caller inputs [nr][nt]
  float *phi_out, *m_out;           // caller outputs [nr][nt], [2][nr][nt]
  const float *phi_init, *m_init;   // optional warm start (caller, may be null)
  float *f;                         // Pcal - Pobs, pitched [nr][ntp]
  float *ux[3], *ut[3];             // u^m lives in ux/ut[m % 3], pitched
  float *ph[2];                     // phi^m lives in ph[m & 1], pitched
  int nt, nr, ntp, tiles_j;         // ntp: row pitch in floats (multiple of 32)
  int tile0, ntiles;                // first global tile index and tile count of this gather
  int unit0, nunits;                // marching pass: first unit in the march order, units per pass
  int strips, seg_h;                // marching pass: 120-sample strips, receivers per segment
  int march_owner;                  // marching pass: the CTA whose decider warp decides it
  float rdx, rdt;                   // 1/dx (0 when nr == 1), 1/dt
  double area, lambda;              // dx*dt (dt when nr == 1); 4/dx^2 + 4/dt^2
};

// Per-gather solver state, written by the deciding CTA of each pass.  The first 32
// bytes are what every CTA of the next pass needs (one vector load).
struct alignas(16) State {
  int k, done;                      // accepted iterations so far; 1 once stopped
  float alpha_f, coef_f, theta_f;   // FP32 copies of alpha_k, c_k, theta_k
  float inv_f, fmean_f;             // 1 / (1 + eps alpha_k), the removed mean of f
  int status;
  double alpha, theta, coef;        // alpha_k, theta_k, c_k (FP64, the decision's copies)
  double beta_fixed;                // fixed-step dual step (linesearch == 0)
  double fmean, fnorm;              // mean of f removed by balancing, ||f - fmean||
  double s_p2, s_u1, s_u2, s_du2;   // last pass: ||p||^2, sum|u|, sum u^2, ||du||^2
  double r_feas, r_step;            // residual at the last stopping test
  double gap_sums[4];               // final pass: sum|u|, sum u^2, <phi,f>, sum (|grad phi|-1)_+^2
  double mass_mu, mass_nu, imbalance;
  int trials;
  unsigned int ticket;
  unsigned int tiles_done;          // persistent solve: tiles finished, cumulative over passes
  unsigned int epoch;               // persistent solve: decisions taken (= next pass index)
};

constexpr int kSpread = 16;         // copies of each accumulator (spreads the atomics)
constexpr int kAccBufs = 2;         // accumulator sets per gather (the persistent solve alternates)
// Solve-wide parameters, passed by value to every kernel.
struct Ctl {
  double eps, xi, zeta, delta, tol, alpha0;
  int max_iter, check_every, ls_max_trials, linesearch, balance, debug_fault;
  int iso;                          // 1: isotropic ground cost ||u||_{1,2}; 0: ||u||_{1,1}
  const Shot *shots;
  State *states;
  double *acc;                      // [gather][kAccBufs][kSpread][kAcc] FP64 accumulators (zeroed)
  const int *tile_shot;             // global tile -> gather
  const int *march_run;             // marching pass: the running gathers, in march order
  int march_nrun;                   // ... and how many
  int *n_done;                      // gathers finished
  int *error;                       // set to 1 when a bounded device wait gives up
  double *trace;                    // optional [gather][max_iter][4] history (or null)
};

enum { ST_OK = 0, ST_NONFINITE = 3, ST_LINESEARCH = 4 };

// Accumulator set `buf` of gather g: kSpread copies of kAcc values.
__device__ __forceinline__ double *acc_of(const Ctl &c, int g, int buf = 0) {
  return c.acc + (static_cast<size_t>(g) * kAccBufs + buf) * kSpread * kAcc;
}

// ------------------------------------------------------------------------------ helpers

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool ok) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int sz = ok ? 16 : 0;  // src-size 0 fills the 16 bytes with zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(sz)
               : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// shrink(x, y) = (1 - y/|x|) x for |x| >= y, else 0  ==  sign(x) max(|x| - y, 0).
__device__ __forceinline__ float shrinkf(float v, float a) {
  const float av = fabsf(v);
  return av >= a ? copysignf(av - a, v) : 0.0f;
}

// The primal prox of one cell, v = u^k + alpha grad phi^k: shrink per component for the
// paper's ||u||_{1,1} (Sec. 2.2), or the vector shrink max(1 - alpha/||v||, 0) v for the
// isotropic ||u||_{1,2}; both then divided by 1 + eps alpha (inv).
__device__ __forceinline__ void prox_cell(float vx, float vt, float alpha, float inv, bool iso,
                                          float &nx, float &nt) {
  if (iso) {
    const float n = sqrtf(vx * vx + vt * vt);
    const float s = n > alpha ? (1.0f - alpha / n) * inv : 0.0f;
    nx = s * vx;
    nt = s * vt;
  } else {
    nx = shrinkf(vx, alpha) * inv;
    nt = shrinkf(vt, alpha) * inv;
  }
}

// The norm of one cell's flux and the conjugate term (|w| - 1)_+^2 of the dual, per the
// ground cost (the duality gap's h* of Sec. 2.2's Lagrangian).
__device__ __forceinline__ float cell_norm(float ux, float ut, bool iso) {
  return iso ? sqrtf(ux * ux + ut * ut) : fabsf(ux) + fabsf(ut);
}
__device__ __forceinline__ float cell_conj(float gx, float gt, bool iso) {
  if (iso) {
    const float e = fmaxf(sqrtf(gx * gx + gt * gt) - 1.0f, 0.0f);
    return e * e;
  }
  const float ex = fmaxf(fabsf(gx) - 1.0f, 0.0f), et = fmaxf(fabsf(gt) - 1.0f, 0.0f);
  return ex * ex + et * et;
}

// Barrier over the NW * 32 compute threads: the whole CTA, or (NAMED) the compute warps
// only, when a CTA also holds producer / decider warps that do not take part.
template <bool NAMED, int NW = kThreads / 32>
__device__ __forceinline__ void compute_sync() {
  if (NAMED)
    asm volatile("bar.sync 1, %0;\n" ::"n"(NW * 32) : "memory");
  else
    __syncthreads();
}

// Reduce N per-thread FP32 partials of a CTA's NW compute warps: FP32 within the warp,
// FP64 across warps (pairwise: log2 NW dependent adds), then one FP64 atomic add per value
// into acc[0..N).  Every compute thread must call it.
template <int N, bool NAMED = false, int NW = kThreads / 32>
__device__ __forceinline__ void block_accumulate(float (&v)[N], double *acc) {
  static_assert((NW & (NW - 1)) == 0 && N <= NW * 32, "pairwise sum over a power of two");
  // acc points at this CTA's copy: acc[0..N)
  __shared__ float part[NW][N];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int n = 0; n < N; ++n) {
    const float w = warp_sum(v[n]);
    if (lane == 0) part[warp][n] = w;
  }
  compute_sync<NAMED, NW>();
  if (threadIdx.x < N) {
    double p[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) p[w] = static_cast<double>(part[w][threadIdx.x]);
#pragma unroll
    for (int h = NW / 2; h >= 1; h >>= 1)
#pragma unroll
      for (int w = 0; w < h; ++w) p[w] += p[w + h];
    atomicAdd(acc + threadIdx.x, p[0]);
  }
}

// Returns true in the one CTA of a gather that finished last (all threads see it).
// Each CTA's atomics above are made visible before it takes its ticket.
__device__ __forceinline__ bool last_block(unsigned int *ticket, int nblocks) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == static_cast<unsigned>(nblocks - 1));
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// In the deciding CTA: sums the kSpread copies of the first N (<= 16) accumulators of a
// gather in one round (half-warp h of warp w takes value w + 8 h, one lane per copy),
// zeroes them for the next pass, and leaves the totals in out[0..N).  Every thread.
template <int N, bool NAMED = false>
__device__ __forceinline__ void gather_totals(double *acc, double (&out)[N]) {
  static_assert(kSpread == 16 && N <= 16, "one lane of a half-warp per copy");
  __shared__ double tot[N];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = warp + (kThreads / 32) * (lane >> 4);
  double v = 0.0;
  if (n < N) {
    double *a = acc + (lane & 15) * kAcc + n;
    v = __ldcg(a);
    *a = 0.0;
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((lane & 15) == 0 && n < N) tot[n] = v;
  compute_sync<NAMED>();
#pragma unroll
  for (int q = 0; q < N; ++q) out[q] = tot[q];
}

// ------------------------------------------------------------------------------ decision

// Writes the FP32 copies of the step sizes that the next pass reads.
__device__ __forceinline__ void publish(State *st, double eps) {
  st->alpha_f = static_cast<float>(st->alpha);
  st->coef_f = static_cast<float>(st->coef);
  st->theta_f = static_cast<float>(st->theta);
  st->inv_f = 1.0f / (1.0f + static_cast<float>(eps * st->alpha));
}

// What the decision needs besides the pass's sums: loaded and precomputed by the
// deciding warp while the sums are still being gathered.  FP64 is slow on this part (a
// warp instruction occupies the FP64 pipe for 64 cycles whatever its active lanes), so
// everything that does not depend on the sums is prepared here, per lane: lane t holds
// trial t's test coefficients and the step sizes (FP64 and FP32) that trial t would
// accept, and the residual test is prepared in squared form.
struct DecidePrep {
  double alpha, theta, coef, beta_fixed, fnorm;
  double s_lane, s_lane2, base32;  // sqrt(1 + theta_k) xi^lane, its square, xi^32
  double dak2;                      // delta alpha_k^2
  double s2x, cl;                   // 2 s_lane; delta alpha_k^2 s_lane^2 / zeta^2
  double alpha_l, coef_l;           // alpha_k s_lane, delta alpha_k s_lane
  float alpha_lf, coef_lf, theta_lf, inv_lf;  // their FP32 copies, 1 / (1 + eps alpha)
  double thr_feas, tol2;            // r_feas <= tol <=> P_pp <= thr_feas; tol^2
  int k;
  int check;                        // this decision runs the residual test
};

// The per-lane part of DecidePrep from its loaded fields (k, alpha, theta, coef,
// beta_fixed, fnorm).
__device__ __forceinline__ void decide_prep_lanes(const Ctl &c, DecidePrep &d) {
  const int lane = threadIdx.x & 31;
  double xl = 1.0, base = c.xi;  // xl = xi^lane; base ends as xi^32
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    if ((lane >> b) & 1) xl *= base;
    base *= base;
  }
  d.base32 = base;
  d.s_lane = sqrt(1.0 + d.theta) * xl;  // upper end of [alpha_k, alpha_k sqrt(1+theta_k)]
  d.s_lane2 = d.s_lane * d.s_lane;
  d.dak2 = c.delta * d.alpha * d.alpha;
  d.s2x = 2.0 * d.s_lane;
  d.cl = d.dak2 * d.s_lane2 / (c.zeta * c.zeta);
  d.alpha_l = d.alpha * d.s_lane;
  d.coef_l = c.delta * d.alpha_l;
  d.alpha_lf = static_cast<float>(d.alpha_l);
  d.coef_lf = static_cast<float>(d.coef_l);
  d.theta_lf = static_cast<float>(d.s_lane);
  d.inv_lf = 1.0f / (1.0f + static_cast<float>(c.eps * d.alpha_l));
  d.check = c.tol > 0.0 && (d.k + 1) % c.check_every == 0;
  d.tol2 = c.tol * c.tol;
  d.thr_feas = d.fnorm > 0.0 ? d.tol2 * d.fnorm * d.fnorm : d.tol2;
}

// St: State (global) or any copy of it with the same field names (shared memory).
template <typename St>
__device__ __forceinline__ DecidePrep decide_prep(const Ctl &c, const St *st) {
  DecidePrep d;
  d.k = st->k;
  d.alpha = st->alpha;
  d.theta = st->theta;
  d.coef = st->coef;
  d.beta_fixed = st->beta_fixed;
  d.fnorm = st->fnorm;
  decide_prep_lanes(c, d);
  return d;
}

// Outcome of one decision (identical in every lane of the deciding warp).
struct Decision {
  int status, trials_now, k_new;
  bool done, checked;
  double alpha, theta, coef;
  float alpha_f, coef_f, theta_f, inv_f;  // FP32 copies for the next pass
};

// True unless x is an infinity or a NaN (integer test of the exponent: no FP64 op).
__device__ __forceinline__ bool finite_bits(double x) {
  return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// Linesearch decision of Algorithm 1 from the sums of pass k, taken by one warp.
// a: 0 P_pp, 1 P_pq, 2 P_qq, 3 G_pp, 4 G_pq, 5 G_qq, 6 sum|u|, 7 sum u^2, 8 sum du^2.
// Trial t (0-based) uses a = alpha_k s_t with s_t = sqrt(1 + theta_k) xi^t, so the trials
// do not depend on each other: lane t tests trial t (32 at a time) and a ballot picks the
// first that passes -- the same choice as Algorithm 1's sequential backtracking.  The
// test delta a^2 ||grad(p + s q)||^2 <= zeta^2 ||p + s q||^2 is evaluated as
// cl (G_pp + 2s G_pq + s^2 G_qq) <= P_pp + 2s P_pq + s^2 P_qq with cl = delta a^2 / zeta^2.
// Then the stopping test (max_iter; the residual every check_every iterations when
// tol > 0, compared in squared form: max(r_feas, r_step) <= tol).
__device__ Decision decide_core(const Ctl &c, const DecidePrep &d, const double (&a_)[9]) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const double Ppp = a_[0], Ppq = a_[1], Pqq = a_[2], Gpp = a_[3], Gpq = a_[4], Gqq = a_[5];
  bool finite = true;  // constant indices keep a_ in registers
#pragma unroll
  for (int n = 0; n < 9; ++n) finite = finite && finite_bits(a_[n]);
  Decision o;
  o.status = ST_OK;
  o.trials_now = 1;
  o.done = false;
  o.checked = false;
  o.alpha = d.alpha;
  o.theta = d.theta;
  o.coef = d.coef;
  o.alpha_f = o.coef_f = o.theta_f = o.inv_f = 0.0f;
  if (!finite) {
    o.status = ST_NONFINITE;
    o.done = true;
  } else if (c.linesearch && d.fnorm == 0.0 && Ppp == 0.0 && Pqq == 0.0) {
    // Identical gathers (the balanced f identically zero) with p and q identically zero: the
    // dual move is zero for every step size and every trial would pass, on every iteration.
    // The step keeps the lower end alpha_k of [alpha_k, alpha_k sqrt(1 + theta_k)] (theta =
    // 1); growing by the upper end, it would overflow the FP32 dual step within about 200
    // iterations and inf * 0 would turn phi into NaN (reading Q20).
    o.theta = 1.0;
    o.coef = c.delta * o.alpha;
    o.alpha_f = static_cast<float>(o.alpha);
    o.coef_f = static_cast<float>(o.coef);
    o.theta_f = 1.0f;
    o.inv_f = 1.0f / (1.0f + static_cast<float>(c.eps * o.alpha));
  } else if (c.linesearch) {
    const bool pass0 = lane < c.ls_max_trials && c.debug_fault != 1 &&
                       d.cl * fma(d.s_lane2, Gqq, fma(d.s2x, Gpq, Gpp)) <=
                           fma(d.s_lane2, Pqq, fma(d.s2x, Ppq, Ppp));
    const unsigned m0 = __ballot_sync(FULL, pass0);
    if (m0) {  // the common case: one of the first 32 trials; its values were prepared
      const int w = __ffs(m0) - 1;
      o.trials_now = w + 1;
      o.theta = __shfl_sync(FULL, d.s_lane, w);
      o.alpha = __shfl_sync(FULL, d.alpha_l, w);
      o.coef = __shfl_sync(FULL, d.coef_l, w);
      o.alpha_f = __shfl_sync(FULL, d.alpha_lf, w);
      o.coef_f = __shfl_sync(FULL, d.coef_lf, w);
      o.theta_f = __shfl_sync(FULL, d.theta_lf, w);
      o.inv_f = __shfl_sync(FULL, d.inv_lf, w);
    } else {  // trials 32 and beyond, 32 at a time
      const double b2 = d.base32 * d.base32;
      double s2x = d.s2x * d.base32, s2 = d.s_lane2 * b2, cl = d.cl * b2;
      int found = -1;
      double s_found = 0.0;
      for (int t0 = 32; t0 < c.ls_max_trials && found < 0; t0 += 32) {
        const bool pass = t0 + lane < c.ls_max_trials && c.debug_fault != 1 &&
                          cl * fma(s2, Gqq, fma(s2x, Gpq, Gpp)) <= fma(s2, Pqq, fma(s2x, Ppq, Ppp));
        const unsigned m = __ballot_sync(FULL, pass);
        if (m) {
          const int w = __ffs(m) - 1;
          found = t0 + w;
          s_found = 0.5 * __shfl_sync(FULL, s2x, w);
        }
        s2x *= d.base32;
        s2 *= b2;
        cl *= b2;
      }
      if (found >= 0) {
        o.trials_now = found + 1;
        o.theta = s_found;
        o.alpha = d.alpha * s_found;
        o.coef = c.delta * o.alpha;
        o.alpha_f = static_cast<float>(o.alpha);
        o.coef_f = static_cast<float>(o.coef);
        o.theta_f = static_cast<float>(o.theta);
        o.inv_f = 1.0f / (1.0f + static_cast<float>(c.eps * o.alpha));
      } else {
        o.trials_now = c.ls_max_trials;
        o.status = ST_LINESEARCH;
        o.done = true;
      }
    }
  } else {
    o.coef = d.beta_fixed;
    o.theta = 1.0;
    o.alpha_f = static_cast<float>(o.alpha);
    o.coef_f = static_cast<float>(o.coef);
    o.theta_f = 1.0f;
    o.inv_f = 1.0f / (1.0f + static_cast<float>(c.eps * o.alpha));
  }
  o.k_new = o.status == ST_OK ? d.k + 1 : d.k;
  if (!o.done && o.k_new >= c.max_iter) o.done = true;
  if (!o.done && d.check) {
    o.checked = true;
    if (Ppp <= d.thr_feas && a_[8] <= d.tol2 * fmax(a_[7], 1e-60)) o.done = true;
  }
  return o;
}

// The reported residuals of a checked decision (Q6): r_feas = ||div u + f|| / ||f||,
// r_step = ||du|| / ||u||.  Not on the decision's critical path.
__device__ __forceinline__ void residuals(const DecidePrep &d, const double (&a_)[9],
                                          double &r_feas, double &r_step) {
  r_feas = d.fnorm > 0.0 ? sqrt(a_[0]) / d.fnorm : sqrt(a_[0]);
  r_step = sqrt(a_[8]) / fmax(sqrt(a_[7]), 1e-30);
}

// One entry of the optional per-iteration history (lane 0 of the deciding warp).
__device__ __forceinline__ void write_trace(const Ctl &c, int gather, int k0, const Decision &o,
                                            double Ppp, double fnorm) {
  if (c.trace && k0 < c.max_iter) {
    double *e = c.trace + (static_cast<size_t>(gather) * c.max_iter + k0) * 4;
    e[0] = o.alpha;
    e[1] = o.theta;
    e[2] = static_cast<double>(o.trials_now);
    e[3] = fnorm > 0.0 ? sqrt(Ppp) / fnorm : sqrt(Ppp);
  }
}

// The decision of a gather whose state lives in global memory; only lane 0 writes it.
__device__ void decide(const Ctl &c, State *st, const DecidePrep &d, const double (&a_)[9],
                       int gather) {
  const Decision o = decide_core(c, d, a_);
  if ((threadIdx.x & 31) != 0) return;
  st->s_p2 = a_[0];
  st->s_u1 = a_[6];
  st->s_u2 = a_[7];
  st->s_du2 = a_[8];
  st->trials += o.trials_now;
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
  write_trace(c, gather, d.k, o, a_[0], d.fnorm);
  if (o.checked) residuals(d, a_, st->r_feas, st->r_step);
  if (o.done) {
    st->done = 1;
    atomicAdd(c.n_done, 1);
  }
}

// ------------------------------------------------------------------------------ prepare

// Builds f = Pcal - Pobs in the pitched plane, zeroes or warm-starts the iterates, sums f,
// f^2, |Pcal| + |Pobs| and the exact differences Pcal - Pobs in FP64 (Sec. 2.1 mass balance:
// mu + nu = |Pcal| + |Pobs| and mu - nu = Pcal - Pobs cell by cell, so sum mu and sum nu are
// half the sum and half the difference of the last two) and initialises each gather's state.
// Grid: (PX, n); CTA x walks rows x, x + PX, ... of gather b0 + blockIdx.y.
__global__ void __launch_bounds__(kThreads) k_prepare(Ctl c, int b0) {
  const int b = b0 + static_cast<int>(blockIdx.y);
  const Shot S = c.shots[b];
  State *st = c.states + b;
  double sf = 0.0, sf2 = 0.0, sab = 0.0, sdx = 0.0;
  for (int i = blockIdx.x; i < S.nr; i += gridDim.x) {
    for (int j = threadIdx.x; j < S.ntp; j += kThreads) {
      const bool in = j < S.nt;
      const size_t g = static_cast<size_t>(i) * S.nt + j;
      const int o = i * S.ntp + j;
      const float po = in ? S.p_obs[g] : 0.0f;
      const float pp = in ? S.p_pred[g] : 0.0f;
      const float f = pp - po;
      S.f[o] = f;
      const double fd = static_cast<double>(f), dp = static_cast<double>(pp), dq = static_cast<double>(po);
      sf += fd;
      sf2 = fma(fd, fd, sf2);
      sdx += dp - dq;
      sab += fabs(dp) + fabs(dq);
      float ux = 0.0f, ut = 0.0f, ph = 0.0f;
      if (in && S.m_init) {
        // the outer faces (x plane row 0, t plane column 0) carry no flux
        ux = i > 0 ? S.m_init[g] : 0.0f;
        ut = j > 0 ? S.m_init[static_cast<size_t>(S.nr) * S.nt + g] : 0.0f;
      }
      if (in && S.phi_init) ph = S.phi_init[g];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        S.ux[m][o] = m == 0 ? ux : 0.0f;
        S.ut[m][o] = m == 0 ? ut : 0.0f;
      }
      S.ph[0][o] = 0.0f;
      S.ph[1][o] = ph;  // pass 0 reads phi^{-1} := phi_init from ph[1]
    }
  }
  // block reduction in FP64 (this kernel runs once per solve)
  __shared__ double red[kThreads / 32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double v[4] = {sf, sf2, sab, sdx};
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    v[n] = warp_sum_d(v[n]);
    if (lane == 0) red[warp][n] = v[n];
  }
  __syncthreads();
  double *acc = acc_of(c, b);
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w][threadIdx.x];
    atomicAdd(acc + (blockIdx.x % kSpread) * kAcc + threadIdx.x, t);
  }
  if (!last_block(&st->ticket, gridDim.x)) return;
  double a_[4];
  gather_totals<4>(acc, a_);
  if (threadIdx.x != 0) return;
  const double N = static_cast<double>(S.nr) * S.nt;
  const double fmean = c.balance ? a_[0] / N : 0.0;
  st->fmean = fmean;
  st->fmean_f = static_cast<float>(fmean);
  st->fnorm = sqrt(fmax(a_[1] - 2.0 * fmean * a_[0] + N * fmean * fmean, 0.0));
  st->mass_mu = S.area * 0.5 * (a_[2] + a_[3]);
  st->mass_nu = S.area * 0.5 * (a_[2] - a_[3]);
  st->imbalance = S.area * a_[3];
  double alpha;
  if (c.linesearch) {
    alpha = c.alpha0 > 0.0 ? c.alpha0 : 1.0 / sqrt(c.delta * S.lambda);
  } else {
    alpha = c.alpha0 > 0.0 ? c.alpha0 : 1.0 / sqrt(S.lambda);
  }
  st->alpha = alpha;
  st->beta_fixed = 1.0 / (S.lambda * alpha);
  st->theta = 1.0;
  st->coef = 0.0;  // pass 0: phi^0 = phi^{-1} (the initial potential)
  publish(st, c.eps);
  st->k = 0;
  st->trials = 0;
  st->status = ST_OK;
  st->r_feas = st->r_step = -1.0;
  st->ticket = 0u;
  __threadfence();
  st->done = 0;
}

// ------------------------------------------------------------------------------ the pass

// FINAL = false: PDHG pass k (see the file header).  FINAL = true: after the last
// accepted iteration K, finishes phi^K, writes phi^K and u^K to the caller's outputs and
// sums the duality gap.  Grid: one CTA per tile of every gather (tile_shot maps it).
template <int TI, int W, bool FINAL>
__global__ void __launch_bounds__(kThreads) k_pass(Ctl c) {
  constexpr int TJ = W - 8;          // output columns per tile
  constexpr int R = TI + 4;          // staged rows: i0-2 .. i0+TI+1
  constexpr int NRS = kThreads / W;  // rows per sweep of the CTA
  static_assert(kThreads % W == 0, "W must divide the CTA");
  extern __shared__ float4 smem4[];
  float *sm = reinterpret_cast<float *>(smem4);
  float *UAx = sm;          // u^{k-1} (then u^{k+1})
  float *UAt = sm + 1 * R * W;
  float *UBx = sm + 2 * R * W;  // u^k
  float *UBt = sm + 3 * R * W;
  float *PH = sm + 4 * R * W;   // phi^{k-1} -> phi^k -> q_k
  float *FF = sm + 5 * R * W;   // f -> p_k

  const int gtile = blockIdx.x;
  const int s = c.tile_shot[gtile];
  const Shot &S = c.shots[s];
  State *st = c.states + s;

  // the 32 hot bytes of the state: k, done and the FP32 step sizes
  const int4 h0 = __ldcg(reinterpret_cast<const int4 *>(st));
  const int4 h1 = __ldcg(reinterpret_cast<const int4 *>(st) + 1);
  if (!FINAL && h0.y) return;  // this gather has stopped
  const int k = h0.x;
  const float alpha = __int_as_float(h0.z), coef = __int_as_float(h0.w);
  const float theta = __int_as_float(h1.x), inv = __int_as_float(h1.y);
  const float fmean = __int_as_float(h1.z);

  const int nr = S.nr, nt = S.nt, ntp = S.ntp;
  const float rdx = S.rdx, rdt = S.rdt;
  const int lt = gtile - S.tile0;
  const int i0 = (lt / S.tiles_j) * TI;
  const int j0 = (lt % S.tiles_j) * TJ;

  const int kp = k == 0 ? 0 : (k - 1) % 3, kc = k % 3, kn = (k + 1) % 3;
  const float *ph_prev = S.ph[(k + 1) & 1];
  float *ph_cur = S.ph[k & 1];

  // ---- stage the six input planes (rows i0-2.., columns j0-4..) into shared memory
  {
    const float *src[6] = {S.ux[kp], S.ut[kp], S.ux[kc], S.ut[kc], ph_prev, S.f};
    constexpr int Q = W / 4;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      for (int v = threadIdx.x; v < R * Q; v += kThreads) {
        const int r = v / Q, q = v - r * Q;
        const int gi = i0 - 2 + r, gj = j0 - 4 + 4 * q;
        const bool ok = gi >= 0 && gi < nr && gj >= 0 && gj < ntp;
        const float *g = ok ? src[a] + gi * ntp + gj : src[a];
        cp_async16(sm + a * R * W + r * W + 4 * q, g, ok);
      }
    }
    cp_async_wait_all();
    __syncthreads();
  }

  const int tx = threadIdx.x % W, ty = threadIdx.x / W;
  const int c_ = tx;             // shared-memory column of this thread
  const int gj = j0 - 4 + c_;    // its global time index
  const bool col_in = gj >= 0 && gj < nt;

  // ---- phase 1: phi^k on rows i0-2..i0+TI, columns j0-2..j0+TJ
  if (c_ >= 2 && c_ < TJ + 5) {
    for (int r = ty; r < TI + 3; r += NRS) {
      const int gi = i0 - 2 + r;
      const int o = r * W + c_;
      float phk = 0.0f;
      if (col_in && gi >= 0 && gi < nr) {
        const bool xl = gi > 0, xr = gi + 1 < nr, tl = gj > 0, tr = gj + 1 < nt;
        const float bxl = xl ? UBx[o] : 0.0f, bxr = xr ? UBx[o + W] : 0.0f;
        const float btl = tl ? UBt[o] : 0.0f, btr = tr ? UBt[o + 1] : 0.0f;
        const float axl = xl ? UAx[o] : 0.0f, axr = xr ? UAx[o + W] : 0.0f;
        const float atl = tl ? UAt[o] : 0.0f, atr = tr ? UAt[o + 1] : 0.0f;
        const float divB = (bxr - bxl) * rdx + (btr - btl) * rdt;
        const float divA = (axr - axl) * rdx + (atr - atl) * rdt;
        const float p = divB + (FF[o] - fmean);
        const float q = divB - divA;
        phk = PH[o] + coef * (p + theta * q);
        if (r >= 2 && r < TI + 2 && c_ >= 4 && c_ < TJ + 4) {
          if (FINAL)
            S.phi_out[static_cast<size_t>(gi) * nt + gj] = phk;
          else
            ph_cur[gi * ntp + gj] = phk;
        }
      }
      PH[o] = phk;
    }
  }
  __syncthreads();

  if (FINAL) {
    // ---- duality gap terms and the caller's copies of phi^K and u^K, over the tile
    float v[4] = {0.f, 0.f, 0.f, 0.f};  // sum|u|, sum u^2, <phi, f>, sum (|grad phi|-1)_+^2
    if (col_in && c_ >= 4 && c_ < TJ + 4) {
      for (int r = 2 + ty; r < TI + 2; r += NRS) {
        const int gi = i0 - 2 + r;
        if (gi >= nr) break;
        const int o = r * W + c_;
        const float gx = gi > 0 ? (PH[o] - PH[o - W]) * rdx : 0.0f;
        const float gt = gj > 0 ? (PH[o] - PH[o - 1]) * rdt : 0.0f;
        const float ux = UBx[o], ut = UBt[o];
        const size_t g = static_cast<size_t>(gi) * nt + gj;
        S.m_out[g] = ux;
        S.m_out[static_cast<size_t>(nr) * nt + g] = ut;
        v[0] += cell_norm(ux, ut, c.iso);
        v[1] += ux * ux + ut * ut;
        v[2] += PH[o] * (FF[o] - fmean);
        v[3] += cell_conj(gx, gt, c.iso);
      }
    }
    double *acc = acc_of(c, s);
    block_accumulate<4>(v, acc + (lt % kSpread) * kAcc);
    if (!last_block(&st->ticket, S.ntiles)) return;
    double a_[4];
    gather_totals<4>(acc, a_);
    if (threadIdx.x == 0) {
      for (int n = 0; n < 4; ++n) st->gap_sums[n] = a_[n];
      st->ticket = 0u;
    }
    return;
  }

  // ---- phase 2: u^{k+1} = prox on rows i0-1..i0+TI, columns j0-1..j0+TJ
  if (c_ >= 3 && c_ < TJ + 5) {
    for (int r = 1 + ty; r < TI + 3; r += NRS) {
      const int gi = i0 - 2 + r;
      const int o = r * W + c_;
      float nx = 0.0f, nt_ = 0.0f;
      if (col_in && gi >= 0 && gi < nr) {
        const float gx = gi > 0 ? (PH[o] - PH[o - W]) * rdx : 0.0f;
        const float gt = gj > 0 ? (PH[o] - PH[o - 1]) * rdt : 0.0f;
        prox_cell(UBx[o] + alpha * gx, UBt[o] + alpha * gt, alpha, inv, c.iso, nx, nt_);
        if (r >= 2 && r < TI + 2 && c_ >= 4 && c_ < TJ + 4) {
          S.ux[kn][gi * ntp + gj] = nx;
          S.ut[kn][gi * ntp + gj] = nt_;
        }
      }
      UAx[o] = nx;
      UAt[o] = nt_;
    }
  }
  __syncthreads();

  // ---- phase 3: p_k = div u^{k+1} + f, q_k = div(u^{k+1} - u^k) on rows i0-1..i0+TI-1,
  //      columns j0-1..j0+TJ-1 (p overwrites f, q overwrites phi^k)
  if (c_ >= 3 && c_ < TJ + 4) {
    for (int r = 1 + ty; r < TI + 2; r += NRS) {
      const int gi = i0 - 2 + r;
      const int o = r * W + c_;
      float p = 0.0f, q = 0.0f;
      if (col_in && gi >= 0 && gi < nr) {
        const bool xl = gi > 0, xr = gi + 1 < nr, tl = gj > 0, tr = gj + 1 < nt;
        const float nxl = xl ? UAx[o] : 0.0f, nxr = xr ? UAx[o + W] : 0.0f;
        const float ntl = tl ? UAt[o] : 0.0f, ntr = tr ? UAt[o + 1] : 0.0f;
        const float bxl = xl ? UBx[o] : 0.0f, bxr = xr ? UBx[o + W] : 0.0f;
        const float btl = tl ? UBt[o] : 0.0f, btr = tr ? UBt[o + 1] : 0.0f;
        const float divN = (nxr - nxl) * rdx + (ntr - ntl) * rdt;
        const float divB = (bxr - bxl) * rdx + (btr - btl) * rdt;
        p = divN + (FF[o] - fmean);
        q = divN - divB;
      }
      FF[o] = p;
      PH[o] = q;
    }
  }
  __syncthreads();

  // ---- phase 4: the linesearch / residual / distance sums over the tile
  float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (col_in && c_ >= 4 && c_ < TJ + 4) {
    for (int r = 2 + ty; r < TI + 2; r += NRS) {
      const int gi = i0 - 2 + r;
      if (gi >= nr) break;
      const int o = r * W + c_;
      const float p = FF[o], q = PH[o];
      const float gpx = gi > 0 ? (p - FF[o - W]) * rdx : 0.0f;
      const float gpt = gj > 0 ? (p - FF[o - 1]) * rdt : 0.0f;
      const float gqx = gi > 0 ? (q - PH[o - W]) * rdx : 0.0f;
      const float gqt = gj > 0 ? (q - PH[o - 1]) * rdt : 0.0f;
      v[0] += p * p;
      v[1] += p * q;
      v[2] += q * q;
      v[3] += gpx * gpx + gpt * gpt;
      v[4] += gpx * gqx + gpt * gqt;
      v[5] += gqx * gqx + gqt * gqt;
      const float nx = UAx[o], nt_ = UAt[o];
      const float dx_ = nx - UBx[o], dt_ = nt_ - UBt[o];
      v[6] += cell_norm(nx, nt_, c.iso);
      v[7] += nx * nx + nt_ * nt_;
      v[8] += dx_ * dx_ + dt_ * dt_;
    }
  }
  double *acc = acc_of(c, s);
  block_accumulate<9>(v, acc + (lt % kSpread) * kAcc);
  if (!last_block(&st->ticket, S.ntiles)) return;
  DecidePrep pr;
  if (threadIdx.x < 32) pr = decide_prep(c, st);
  double a_[9];
  gather_totals<9>(acc, a_);
  if (threadIdx.x < 32) decide(c, st, pr, a_, s);
  if (threadIdx.x == 0) st->ticket = 0u;
}

// ------------------------------------------------------------------------------ adjoint

// Sum of phi in FP64 (per-thread FP32 over a grid-stride, FP64 above a warp).
__global__ void __launch_bounds__(kThreads) k_adj_sum(const float *phi, size_t n, double *acc) {
  float v[1] = {0.0f};
  for (size_t i = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * kThreads)
    v[0] += phi[i];
  block_accumulate<1>(v, acc);
}

// grad_pred = g * area * (phi - mean), grad_obs = -grad_pred (Sec. 2.3 adjoint source).
__global__ void __launch_bounds__(kThreads) k_adj_scale(const float *phi, size_t n, double area,
                                                        int balance, const double *acc,
                                                        const float *grad_out, float *gp,
                                                        float *go) {
  const float mean = balance ? static_cast<float>(acc[0] / static_cast<double>(n)) : 0.0f;
  const float g = static_cast<float>((grad_out ? static_cast<double>(*grad_out) : 1.0) * area);
  for (size_t i = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * kThreads) {
    const float v = g * (phi[i] - mean);
    gp[i] = v;
    if (go) go[i] = -v;
  }
}

// One gather of a batched adjoint (device copy in the caller's workspace).
struct AdjJob {
  const float *phi;
  float *gp, *go;          // d dist / d Pcal, and its negative (nullable)
  const float *grad_out;   // device scalar or null (= 1)
  long long n;             // cells
  double area;             // dx dt (dt when nr == 1)
};

// Sums of phi of every gather of a batch: grid (X, B), acc[b] += sum of gather b (FP32 per
// thread over a grid stride, FP64 above the warp).
__global__ void __launch_bounds__(kThreads) k_adj_sum_batched(const AdjJob *jobs, double *acc) {
  const AdjJob J = jobs[blockIdx.y];
  float v[1] = {0.0f};
  const long long stride = static_cast<long long>(gridDim.x) * kThreads;
  for (long long i = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x; i < J.n; i += stride)
    v[0] += J.phi[i];
  block_accumulate<1>(v, acc + blockIdx.y);
}

// grad_pred = g area (phi - mean), grad_obs = -grad_pred for gather blockIdx.y (Sec. 2.3),
// four cells per thread where every pointer of the gather is 16-byte aligned.
__global__ void __launch_bounds__(kThreads) k_adj_scale_batched(const AdjJob *jobs, const double *acc,
                                                                int balance) {
  const AdjJob J = jobs[blockIdx.y];
  const float mean = balance ? static_cast<float>(acc[blockIdx.y] / static_cast<double>(J.n)) : 0.0f;
  const float g = static_cast<float>((J.grad_out ? static_cast<double>(*J.grad_out) : 1.0) * J.area);
  const long long stride = static_cast<long long>(gridDim.x) * kThreads;
  const long long t0 = blockIdx.x * static_cast<long long>(kThreads) + threadIdx.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(J.phi) | reinterpret_cast<uintptr_t>(J.gp) |
                     reinterpret_cast<uintptr_t>(J.go)) & 15u) == 0;
  long long done = 0;
  if (vec) {
    const long long n4 = J.n / 4;
    const float4 *p4 = reinterpret_cast<const float4 *>(J.phi);
    float4 *gp4 = reinterpret_cast<float4 *>(J.gp), *go4 = reinterpret_cast<float4 *>(J.go);
    for (long long i = t0; i < n4; i += stride) {
      const float4 x = p4[i];
      const float4 y = make_float4(g * (x.x - mean), g * (x.y - mean), g * (x.z - mean), g * (x.w - mean));
      gp4[i] = y;
      if (go4) go4[i] = make_float4(-y.x, -y.y, -y.z, -y.w);
    }
    done = 4 * n4;
  }
  for (long long i = done + t0; i < J.n; i += stride) {
    const float y = g * (J.phi[i] - mean);
    J.gp[i] = y;
    if (J.go) J.go[i] = -y;
  }
}

// ------------------------------------------------------------------------------ decompose

// mu = Pcal+ + Pobs-, nu = Pobs+ + Pcal- (Sec. 2.1) and their FP64 sums.
__global__ void __launch_bounds__(kThreads) k_decompose(const float *po, const float *pp, size_t n,
                                                        float *mu, float *nu, double *acc) {
  double smu = 0.0, snu = 0.0;
  for (size_t i = blockIdx.x * static_cast<size_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * kThreads) {
    const float o = po[i], p = pp[i];
    const float m = fmaxf(p, 0.0f) + fmaxf(-o, 0.0f);
    const float v = fmaxf(o, 0.0f) + fmaxf(-p, 0.0f);
    if (mu) mu[i] = m;
    if (nu) nu[i] = v;
    smu += static_cast<double>(fmaxf(p, 0.0f)) + static_cast<double>(fmaxf(-o, 0.0f));
    snu += static_cast<double>(fmaxf(o, 0.0f)) + static_cast<double>(fmaxf(-p, 0.0f));
  }
  __shared__ double red[kThreads / 32][2];
  smu = warp_sum_d(smu);
  snu = warp_sum_d(snu);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = smu;
    red[threadIdx.x >> 5][1] = snu;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
    atomicAdd(acc + threadIdx.x, s);
  }
}

}  // namespace emd
