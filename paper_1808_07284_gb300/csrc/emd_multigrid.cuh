// Two-grid warm start (Sec. 2.2, closing paragraph; Sec. 3.3): the time axis of both
// gathers is coarsened by an integer factor r, the EMD is solved on the coarse grid, and
// its solution is carried back to the fine grid by sinc (Whittaker-Shannon) interpolation
// to start the fine solve.
//
// Restriction: coarse sample J of a row is the mean of fine samples rJ .. rJ + r - 1,
// the record padded with zeros to a multiple of r, so the coarse gather carries the fine
// gather's mass.
//
// Interpolation: out[i][j] = sum_J in[i][J] sinc(x_j - J), x_j the fine position in coarse
// sample units -- (j - (r - 1)/2) / r for cell-centred data (phi, x flux), j / r for the
// time flux, whose samples sit on the faces between time cells.  Writing x_j = n_j / (2r)
// with the integer n_j = 2j - (r - 1) or 2j, and using sin(pi (x - J)) = (-1)^J sin(pi x),
// every kernel entry is (-1)^J c_j / (n_j - 2rJ) with c_j = 2r sin(pi x_j) / pi, and 1
// where n_j = 2rJ (there sin(pi x_j) = 0, so the other entries of the column vanish and
// the coarse value comes back exactly).  The sum runs over every coarse sample of the
// record: a dense [nr x nc] by [nc x nt] contraction, done here as a shared-memory-tiled
// FP32 product whose kernel tile is generated on the fly (it never touches memory).
#pragma once

#include <cuda_runtime.h>

namespace emd {

// One restriction or interpolation: a [nr][n_in] float array in, [nr][n_out] out.
struct TimeJob {
  const float *in;
  float *out;
  int nr, n_in, n_out, r;
  int staggered;  // interpolation: 1 = time faces (x_j = j / r), 0 = cell centres
  int zero_row0;  // interpolation: row 0 is an outer face (x flux of receiver 0): write 0
  int zero_col0;  // interpolation: column 0 is an outer face (time flux of sample 0): write 0
};

constexpr int kRestrictThreads = 256;

// Block means along time; blockIdx.y is the job (from the device table `jobs`, or `one`
// when the table is NULL).  Adjacent threads take adjacent coarse samples, so a warp
// reads 32 r consecutive floats of one row.
__global__ void __launch_bounds__(kRestrictThreads)
    k_restrict_time(const TimeJob *jobs, TimeJob one) {
  const TimeJob J = jobs ? jobs[blockIdx.y] : one;
  const long long n = static_cast<long long>(J.nr) * J.n_out;
  const float inv_r = 1.0f / static_cast<float>(J.r);
  for (long long c = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; c < n;
       c += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(c / J.n_out);
    const int q = static_cast<int>(c - static_cast<long long>(i) * J.n_out);
    const float *row = J.in + static_cast<size_t>(i) * J.n_in;
    const int j0 = q * J.r, j1 = min(j0 + J.r, J.n_in);
    float s = 0.0f;
    for (int j = j0; j < j1; ++j) s += row[j];
    J.out[c] = s * inv_r;
  }
}

constexpr int kIpBM = 64;    // rows (receivers) of an output tile
constexpr int kIpBN = 128;   // fine time samples of an output tile
constexpr int kIpBK = 32;    // coarse samples per staged chunk
constexpr int kIpThreads = 256;
constexpr float kPi = 3.14159265358979323846f;

// Sinc interpolation; grid (fine-sample tiles, row tiles, jobs), jobs as for the
// restriction.  Warp w owns rows 8w .. 8w + 7 of the tile and lane l the columns l,
// l + 32, l + 64, l + 96: 32 accumulators per thread.  Per chunk the coarse values are staged transposed ([J][row],
// padded so the transposing stores do not collide on a bank) and the kernel tile is
// computed in place: each thread owns one column and 16 of the chunk's coarse samples.
__global__ void __launch_bounds__(kIpThreads) k_prolong_time(const TimeJob *jobs, TimeJob one) {
  const TimeJob Jb = jobs ? jobs[blockIdx.z] : one;
  const int i0 = blockIdx.y * kIpBM, j0 = blockIdx.x * kIpBN;
  if (i0 >= Jb.nr || j0 >= Jb.n_out) return;  // this job is smaller than the grid
  __shared__ float As[kIpBK][kIpBM + 1];
  __shared__ float Ss[kIpBK][kIpBN];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int two_r = 2 * Jb.r;

  // the kernel column this thread generates: x_j = ncol / (2r)
  const int scol = tid & (kIpBN - 1), khalf = tid / kIpBN;
  const int jcol = j0 + scol;
  const int ncol = Jb.staggered ? 2 * jcol : 2 * jcol - (Jb.r - 1);
  int res = ncol % (2 * two_r);  // sin(pi x) has period 2 in x, i.e. 4r in ncol
  if (res < 0) res += 2 * two_r;
  const float c_col =
      sinpif(static_cast<float>(res) / static_cast<float>(two_r)) * static_cast<float>(two_r) / kPi;

  float acc[8][4];
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[t][q] = 0.0f;

  for (int k0 = 0; k0 < Jb.n_in; k0 += kIpBK) {
    for (int e = tid; e < kIpBK * kIpBM; e += kIpThreads) {
      const int row = e / kIpBK, k = e % kIpBK;  // a warp reads 32 consecutive coarse samples
      const int gi = i0 + row, gk = k0 + k;
      As[k][row] = (gi < Jb.nr && gk < Jb.n_in) ? Jb.in[static_cast<size_t>(gi) * Jb.n_in + gk] : 0.0f;
    }
#pragma unroll 4
    for (int kk = 0; kk < kIpBK / 2; ++kk) {
      const int k = khalf * (kIpBK / 2) + kk, J = k0 + k;
      float v = 0.0f;
      if (J < Jb.n_in) {
        const int d = ncol - two_r * J;
        v = d == 0 ? 1.0f : ((J & 1) ? -c_col : c_col) / static_cast<float>(d);
      }
      Ss[k][scol] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kIpBK; ++k) {
      float a[8], s[4];
#pragma unroll
      for (int t = 0; t < 8; ++t) a[t] = As[k][warp * 8 + t];
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q] = Ss[k][lane + 32 * q];
#pragma unroll
      for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[t][q] = fmaf(a[t], s[q], acc[t][q]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int gi = i0 + warp * 8 + t;
    if (gi >= Jb.nr) break;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gj = j0 + lane + 32 * q;
      if (gj >= Jb.n_out) continue;
      const bool outer = (Jb.zero_row0 && gi == 0) || (Jb.zero_col0 && gj == 0);
      Jb.out[static_cast<size_t>(gi) * Jb.n_out + gj] = outer ? 0.0f : acc[t][q];
    }
  }
}

}  // namespace emd
