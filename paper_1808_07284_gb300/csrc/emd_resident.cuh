// Shared-memory-resident solve for small gathers: one CTA holds a whole gather in shared
// memory for the entire solve (up to kResidentMaxCells cells), so a PDHG iteration costs
// four block-wide phases, a block reduction and the linesearch decision -- no global
// memory traffic, atomics or cross-CTA waits.  In a batch every gather gets its own CTA
// and the gathers run independently (the paper solves one EMD per shot).
//
// Shared planes, packed [nr][nt]: UB (u^k, x and t), UN (u^{k+1}, x and t; the two swap
// after every accepted iteration), PH (phi), FF (f), PP (p = div u^{k+1} + f) and
// QQ (q = div(u^{k+1} - u^k)).  Phase 1 of the next pass needs exactly p and q of this
// one (phi^{k+1} = phi^k + c_{k+1} (p_k + theta_{k+1} q_k)), so they are kept, not
// recomputed.  Sixteen warps do the cell work; a seventeenth prepares the next decision
// (state, sqrt(1 + theta), the powers of xi) while they run and takes it afterwards.
#pragma once

#include "emd_kernels.cuh"

namespace emd {

constexpr int kResWarps = 16;                     // cell-work warps
constexpr int kResThreads = (kResWarps + 1) * 32;  // + the decision warp
constexpr int kResPlanes = 8;
constexpr int kResidentMaxCells = 7168;            // 8 planes x 4 B x 7168 = 224 KB

inline size_t resident_smem_bytes(long long cells) {
  return static_cast<size_t>(cells) * kResPlanes * sizeof(float);
}

// Row and column of cell c of an nr x nt gather (float reciprocal, then corrected).
__device__ __forceinline__ void cell_ij(int c, int nt, float inv_nt, int &i, int &j) {
  i = __float2int_rz((static_cast<float>(c) + 0.5f) * inv_nt);
  if (i * nt > c) --i;
  if ((i + 1) * nt <= c) ++i;
  j = c - i * nt;
}

__global__ void __launch_bounds__(kResThreads, 1) k_solve_resident(Ctl c) {
  constexpr int NT = kResWarps * 32;
  const int g = blockIdx.x;
  const Shot &S = c.shots[g];
  State *st = c.states + g;
  extern __shared__ float4 dyn4[];
  float *sm = reinterpret_cast<float *>(dyn4);
  const int nr = S.nr, nt = S.nt, N = nr * nt, ntp = S.ntp;
  const float rdx = S.rdx, rdt = S.rdt, inv_nt = 1.0f / static_cast<float>(nt);
  float *Bx = sm, *Bt = sm + N, *Nx = sm + 2 * N, *Nv = sm + 3 * N;
  float *PH = sm + 4 * N, *FF = sm + 5 * N, *PP = sm + 6 * N, *QQ = sm + 7 * N;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool worker = warp < kResWarps;

  __shared__ float sc[5];         // alpha, coef, theta, 1/(1+eps alpha), fmean (FP32)
  __shared__ double tot[9];       // this pass's sums
  __shared__ float part[kResWarps][9];
  __shared__ DecidePrep dp;       // the decision's FP64 state (k, alpha, theta, ...)
  __shared__ int sdone, sstatus, strials;
  __shared__ double last_sums[3];  // ||p||^2, sum u^2, ||du||^2 of the last pass

  // ---- load the gather: f, u^0, phi^{-1} (the warm start) from the prepared planes
  for (int q = tid; q < N; q += blockDim.x) {
    int i, j;
    cell_ij(q, nt, inv_nt, i, j);
    const int o = i * ntp + j;
    FF[q] = S.f[o];
    Bx[q] = S.ux[0][o];
    Bt[q] = S.ut[0][o];
    PH[q] = S.ph[1][o];
    PP[q] = 0.0f;
    QQ[q] = 0.0f;
  }
  if (tid == 0) {
    sc[0] = st->alpha_f;
    sc[1] = st->coef_f;
    sc[2] = st->theta_f;
    sc[3] = st->inv_f;
    sc[4] = st->fmean_f;
    dp.k = 0;
    dp.alpha = st->alpha;
    dp.theta = st->theta;
    dp.coef = st->coef;
    dp.beta_fixed = st->beta_fixed;
    dp.fnorm = st->fnorm;
    sdone = 0;
    sstatus = ST_OK;
    strials = 0;
  }
  __syncthreads();

  while (true) {
    const int k = dp.k;
    const float alpha = sc[0], coef = sc[1], theta = sc[2], inv = sc[3], fmean = sc[4];
    const bool need_res = (c.tol > 0.0 && (k + 1) % c.check_every == 0) || k + 1 >= c.max_iter;
    DecidePrep pr;
    if (worker) {
      // ---- phase 1: phi^k = phi^{k-1} + c_k (p_{k-1} + theta_k q_{k-1})
      for (int q = tid; q < N; q += NT) PH[q] += coef * (PP[q] + theta * QQ[q]);
    } else {
      // the decision warp: this pass's decision inputs, while the cells are worked on
      pr = dp;
      decide_prep_lanes(c, pr);
    }
    __syncthreads();
    if (worker) {
      // ---- phase 2: u^{k+1} = shrink(u^k + alpha grad phi^k, alpha) / (1 + eps alpha)
      for (int q = tid; q < N; q += NT) {
        int i, j;
        cell_ij(q, nt, inv_nt, i, j);
        const float ph = PH[q];
        const float gx = i > 0 ? (ph - PH[q - nt]) * rdx : 0.0f;
        const float gt = j > 0 ? (ph - PH[q - 1]) * rdt : 0.0f;
        prox_cell(Bx[q] + alpha * gx, Bt[q] + alpha * gt, alpha, inv, c.iso, Nx[q], Nv[q]);
      }
    }
    __syncthreads();
    if (worker) {
      // ---- phase 3: p = div u^{k+1} + f, q = div(u^{k+1} - u^k)
      for (int q = tid; q < N; q += NT) {
        int i, j;
        cell_ij(q, nt, inv_nt, i, j);
        const bool xl = i > 0, xr = i + 1 < nr, tl = j > 0, tr = j + 1 < nt;
        const float nxl = xl ? Nx[q] : 0.0f, nxr = xr ? Nx[q + nt] : 0.0f;
        const float ntl = tl ? Nv[q] : 0.0f, ntr = tr ? Nv[q + 1] : 0.0f;
        const float bxl = xl ? Bx[q] : 0.0f, bxr = xr ? Bx[q + nt] : 0.0f;
        const float btl = tl ? Bt[q] : 0.0f, btr = tr ? Bt[q + 1] : 0.0f;
        const float divN = (nxr - nxl) * rdx + (ntr - ntl) * rdt;
        const float divB = (bxr - bxl) * rdx + (btr - btl) * rdt;
        PP[q] = divN + (FF[q] - fmean);
        QQ[q] = divN - divB;
      }
    }
    __syncthreads();
    float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (worker) {
      // ---- phase 4: the sums
      for (int q = tid; q < N; q += NT) {
        int i, j;
        cell_ij(q, nt, inv_nt, i, j);
        const float p = PP[q], qv = QQ[q];
        const float gpx = i > 0 ? (p - PP[q - nt]) * rdx : 0.0f;
        const float gpt = j > 0 ? (p - PP[q - 1]) * rdt : 0.0f;
        const float gqx = i > 0 ? (qv - QQ[q - nt]) * rdx : 0.0f;
        const float gqt = j > 0 ? (qv - QQ[q - 1]) * rdt : 0.0f;
        v[0] += p * p;
        v[1] += p * qv;
        v[2] += qv * qv;
        v[3] += gpx * gpx + gpt * gpt;
        v[4] += gpx * gqx + gpt * gqt;
        v[5] += gqx * gqx + gqt * gqt;
        if (need_res) {
          const float nx = Nx[q], nv = Nv[q], dx_ = nx - Bx[q], dt_ = nv - Bt[q];
          v[7] += nx * nx + nv * nv;
          v[8] += dx_ * dx_ + dt_ * dt_;
        }
      }
#pragma unroll
      for (int n = 0; n < 9; ++n) {
        const float w = warp_sum(v[n]);
        if (lane == 0) part[warp][n] = w;
      }
    }
    __syncthreads();
    if (tid < 9) {
      double t = 0.0;
      for (int w = 0; w < kResWarps; ++w) t += static_cast<double>(part[w][tid]);
      tot[tid] = t;
    }
    __syncthreads();
    if (!worker) {
      double a_[9];
#pragma unroll
      for (int n = 0; n < 9; ++n) a_[n] = tot[n];
      const Decision o = decide_core(c, pr, a_);
      if (lane == 0) {
        write_trace(c, g, pr.k, o, a_[0], pr.fnorm);
        strials += o.trials_now;
        last_sums[0] = a_[0];
        last_sums[1] = a_[7];
        last_sums[2] = a_[8];
        if (o.status == ST_OK) {
          dp.k = o.k_new;
          dp.alpha = o.alpha;
          dp.theta = o.theta;
          dp.coef = o.coef;
          sc[0] = o.alpha_f;
          sc[1] = o.coef_f;
          sc[2] = o.theta_f;
          sc[3] = o.inv_f;
        } else {
          sstatus = o.status;
        }
        if (o.checked) residuals(pr, a_, st->r_feas, st->r_step);
        sdone = o.done;
      }
    }
    __syncthreads();
    if (sstatus == ST_OK) {  // accepted: u^{k+1} becomes the current iterate
      float *t0 = Bx, *t1 = Bt;
      Bx = Nx;
      Bt = Nv;
      Nx = t0;
      Nv = t1;
    }
    if (sdone) break;
  }

  // ---- hand the last iterates to the finalize pass, in the buffers it reads at k = K:
  // u^{K-1} in u[(K - 1) % 3], u^K in u[K % 3], phi^{K-1} in ph[(K + 1) & 1]
  const int K = dp.k;
  const int kp = K == 0 ? 0 : (K - 1) % 3, kc = K % 3;
  for (int q = tid; q < N; q += blockDim.x) {
    int i, j;
    cell_ij(q, nt, inv_nt, i, j);
    const int o = i * ntp + j;
    if (K > 0) {
      S.ux[kp][o] = Nx[q];
      S.ut[kp][o] = Nv[q];
    }
    S.ux[kc][o] = Bx[q];
    S.ut[kc][o] = Bt[q];
    S.ph[(K + 1) & 1][o] = PH[q];
  }
  if (tid == 0) {
    st->k = K;
    st->trials = strials;
    st->status = sstatus;
    st->alpha = dp.alpha;
    st->theta = dp.theta;
    st->coef = dp.coef;
    publish(st, c.eps);
    st->s_p2 = last_sums[0];
    st->s_u2 = last_sums[1];
    st->s_du2 = last_sums[2];
    st->done = 1;
    atomicAdd(c.n_done, 1);
  }
}

}  // namespace emd
