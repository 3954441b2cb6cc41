// Host side of the C ABI declared in include/emd_gb300.h: argument checks, workspace
// layout, the launch sequence of a solve (prepare -> one fused pass per PDHG iteration
// -> finalize) and result read-back.  All device work is in emd_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdint>
#include <cstring>
#include <vector>

#include "emd_gb300.h"
#include "emd_kernels.cuh"
#include "emd_lsd.cuh"
#include "emd_march.cuh"
#include "emd_multigrid.cuh"
#include "emd_pass_tma.cuh"
#include "emd_resident.cuh"

namespace {

using emd::Ctl;
using emd::kThreads;
using emd::Shot;
using emd::State;

#define EMD_CK(x)                                  \
  do {                                             \
    cudaError_t e_ = (x);                          \
    if (e_ != cudaSuccess) {                       \
      (void)cudaGetLastError();                    \
      return EMD_ERR_CUDA;                         \
    }                                              \
  } while (0)

// Stencil tile shapes (TI rows x (W - 8) time samples per tile); id = index + 1.
// `iter_tma` marks the persistent TMA-staged pass (its finalize pass is the plain one
// with the same tiling).  `solve_march` marks the marching persistent solve (emd_march.cuh:
// NW marching warps per CTA, a ring of D staged rows per warp); its finalize pass, and its
// per-pass fallback where no cooperative launch is possible, are the plain pass with
// TI x (W - 8) tiles.
struct Shape {
  int ti, w;
  void (*iter)(Ctl);
  void (*fin)(Ctl);
  void (*iter_tma)(Ctl, int);
  void (*solve_tma)(Ctl, int, int, int);  // passes [k_begin, k_end) in one cooperative launch
  int minb;                           // persistent pass: CTAs per SM it is compiled for
  int nw, ns;                         // persistent solve: compute warps, shared-memory stages
                                      // (marching solve: rows in flight per warp)
  void (*solve_march)(Ctl, int, int, int);  // passes [k_begin, k_end), marching warps
};

#define EMD_SHAPE(TI, W)                                                                      \
  Shape {                                                                                     \
    TI, W, emd::k_pass<TI, W, false>, emd::k_pass<TI, W, true>, nullptr, nullptr, 0, 0, 0,    \
        nullptr                                                                               \
  }
#define EMD_TMA_SHAPE(TI, MINB, NW, NS)                                                     \
  Shape {                                                                                   \
    TI, 128, nullptr, emd::k_pass<TI, 128, true>, emd::k_pass_tma<TI, MINB>,                \
        emd::k_solve_tma<TI, MINB, NW, NS>, MINB, NW, NS, nullptr                           \
  }
#define EMD_MARCH_SHAPE(NW, D, MINB)                                                        \
  Shape {                                                                                   \
    16, 128, emd::k_pass<16, 128, false>, emd::k_pass<16, 128, true>, nullptr, nullptr, MINB, \
        NW, D, emd::k_solve_march<NW, D, MINB>                                              \
  }
// (A 13 x 120 shape with one CTA per SM, sixteen compute warps and four stages -- three
// tiles in flight -- passed the parity tests but was 20-45 % slower on gathers larger
// than L2 than two CTAs of eight warps with two stages each; it is not compiled.)
const Shape kShapes[] = {EMD_SHAPE(16, 128),          EMD_SHAPE(8, 128),
                         EMD_SHAPE(32, 128),          EMD_SHAPE(8, 256),
                         EMD_SHAPE(16, 256),          EMD_SHAPE(1, 256),
                         EMD_TMA_SHAPE(13, 2, 8, 2),  EMD_TMA_SHAPE(8, 3, 8, 2),
                         EMD_TMA_SHAPE(21, 1, 8, 2),  EMD_MARCH_SHAPE(11, 6, 1),
                         EMD_MARCH_SHAPE(11, 4, 1)};
// (Marching solves need about 165 registers a thread; a scheduler's 16,384 registers then
// hold three warps, so a CTA of eleven marching warps and the decider fills an SM.  Fifteen
// marching warps at 128 registers spill inside the row loop and ran 1.65 times slower.)
#undef EMD_SHAPE
#undef EMD_TMA_SHAPE
#undef EMD_MARCH_SHAPE
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);
constexpr int kTmaShape = 6;         // 13 x 120, two CTAs per SM: the untuned default
constexpr int kTmaFirst = 6;         // shapes kTmaFirst .. kNumShapes - 1 run persistent solves

// Dynamic shared memory of the plain pass / finalize pass of a shape, of its per-pass
// TMA kernel (two stages of six (TI + 4) x 128 planes, plus alignment slack) and of its
// persistent solve (ns such stages).
size_t smem_bytes(const Shape &s) { return sizeof(float) * 6u * (s.ti + 4) * s.w; }
size_t iter_smem_bytes(const Shape &s) {
  return s.iter_tma ? 2u * 6u * (s.ti + 4) * 128u * sizeof(float) + 128u : smem_bytes(s);
}
size_t solve_smem_bytes(const Shape &s) {
  if (s.solve_march)  // per warp: the ring of ns rows of six planes and three scratch rows
    return static_cast<size_t>(s.nw) * (6u * s.ns + 3u) * emd::kMarchW * sizeof(float) + 128u;
  return static_cast<size_t>(s.ns) * 6u * (s.ti + 4) * 128u * sizeof(float) + 128u;
}
bool uses_tma(const Shape &s) { return s.iter_tma != nullptr; }

// cuTensorMapEncodeTiled, reached through the runtime (no link against libcuda).
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_fn() {
  static EncodeTiled fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      (void)cudaGetLastError();
      return static_cast<EncodeTiled>(nullptr);
    }
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// Multiprocessors of the current device (the persistent pass runs two CTAs on each).
int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    (void)cudaGetLastError();
    return 148;
  }
  return n;
}

size_t align256(size_t x) { return (x + 255u) & ~static_cast<size_t>(255u); }
int ntp_of(int nt) { return (nt + 31) / 32 * 32; }
int tiles_of(const Shape &s, int nt, int nr) {
  return ((nr + s.ti - 1) / s.ti) * ((nt + (s.w - 8) - 1) / (s.w - 8));
}

bool size_ok(int nt, int nr) {
  if (nt < 2 || nr < 1 || nt > (1 << 24) || nr > (1 << 20)) return false;
  return static_cast<long long>(nr) * ntp_of(nt) < (1ll << 30);
}

// Workspace: [states | shots | accumulators | tile_shot | n_done + scratch] then, per gather, the
// pitched planes f, u0 (x,t), u1 (x,t), u2 (x,t), phi0, phi1 (36 bytes per cell).
struct Layout {
  size_t states, shots, acc, tiles, units, misc, header, total;
  std::vector<size_t> gather;  // offset of each gather's planes
  std::vector<size_t> plane;   // bytes of one plane (256-aligned)
  int max_tiles;
};

Layout layout(int B, const int *nt, const int *nr) {
  Layout L{};
  L.max_tiles = 0;
  for (int b = 0; b < B; ++b) {
    int mt = 0;
    for (const Shape &s : kShapes) mt = std::max(mt, tiles_of(s, nt[b], nr[b]));
    L.max_tiles += mt;
  }
  L.states = 0;
  L.shots = align256(sizeof(State) * B);
  L.acc = L.shots + align256(sizeof(Shot) * B);
  L.tiles = L.acc + align256(sizeof(double) * emd::kAccBufs * emd::kSpread * emd::kAcc * B);
  L.units = L.tiles + align256(sizeof(int) * static_cast<size_t>(L.max_tiles));
  L.misc = L.units + align256(sizeof(int) * static_cast<size_t>(B));  // the march's gather list
  L.header = L.misc + 256;
  size_t off = L.header;
  for (int b = 0; b < B; ++b) {
    const size_t pl = align256(sizeof(float) * static_cast<size_t>(nr[b]) * ntp_of(nt[b]));
    L.gather.push_back(off);
    L.plane.push_back(pl);
    off += 9 * pl;
  }
  L.total = off;
  return L;
}

// Units of the marching solve for T marching warps, dealt round-robin (unit u to warp
// u mod T).  Every running gather is cut into segments of about H receivers (nseg = ceil(nr /
// H) equal segments) times its 120-sample strips; the warp marching the most units then
// needs ceil(U / T) (h + 4 + c0) row times (4 halo rows, c0 ~ 2 rows to start a unit), and H
// is the candidate that minimises it.  Fills the gathers' unit fields and deciding CTAs (the
// CTA of the warp that marches a gather's first unit); returns the units of one pass, or -1
// when they do not fit an int.
long long march_layout(std::vector<Shot> &shots, const std::vector<int> &run, long long T, int nw) {
  constexpr long long kStartRows = 2;
  int nr_max = 1;
  for (int b : run) {
    Shot &S = shots[b];
    S.strips = (S.nt + emd::kMarchTJ - 1) / emd::kMarchTJ;
    nr_max = std::max(nr_max, S.nr);
  }
  auto units_for = [&](long long H, long long &hmax) {
    long long U = 0;
    hmax = 0;
    for (int b : run) {
      const Shot &S = shots[b];
      const long long nseg = (S.nr + H - 1) / H;
      hmax = std::max(hmax, (S.nr + nseg - 1) / nseg);
      U += S.strips * nseg;
    }
    return U;
  };
  long long best_H = nr_max, best_cost = -1;
  const int cands = std::min(512, std::max(1, (nr_max + emd::kMarchMinSeg - 1) / emd::kMarchMinSeg));
  for (int c = 1; c <= cands; ++c) {
    const long long nseg = std::max<long long>(
        1, static_cast<long long>(std::llround(std::pow(static_cast<double>(nr_max) / emd::kMarchMinSeg,
                                                        (c - 1.0) / std::max(1, cands - 1)))));
    const long long H = std::max<long long>(emd::kMarchMinSeg, (nr_max + nseg - 1) / nseg);
    long long hmax = 0;
    const long long U = units_for(H, hmax);
    if (U > 0x7fffffffll) continue;
    const long long cost = (U + T - 1) / T * (hmax + 4 + kStartRows);
    if (best_cost < 0 || cost < best_cost || (cost == best_cost && H > best_H)) {
      best_cost = cost;
      best_H = H;
    }
  }
  long long U = 0;
  for (int b : run) {
    Shot &S = shots[b];
    const long long nseg = (S.nr + best_H - 1) / best_H;
    S.seg_h = static_cast<int>((S.nr + nseg - 1) / nseg);
    const long long ns = (S.nr + S.seg_h - 1) / S.seg_h;
    S.unit0 = static_cast<int>(U);
    S.nunits = static_cast<int>(S.strips * ns);
    S.march_owner = static_cast<int>((U % T) / nw);
    U += S.nunits;
    if (U > 0x7fffffffll) return -1;
  }
  return U;
}

bool params_ok(const emd_params &p) {
  auto fin = [](double v) { return std::isfinite(v); };
  if (!fin(p.eps) || !fin(p.xi) || !fin(p.zeta) || !fin(p.delta) || !fin(p.alpha0) || !fin(p.tol))
    return false;
  if (!(p.xi > 0 && p.xi < 1) || !(p.zeta > 0 && p.zeta < 1) || !(p.delta > 0) || p.eps < 0)
    return false;
  if (p.max_iter < 1 || p.check_every < 1 || p.ls_max_trials < 1 || p.tol < 0) return false;
  if (p.linesearch != 0 && p.linesearch != 1) return false;
  if (p.ls_norm != 2) return false;  // the GPU path implements the Euclidean test only
  if (p.balance != EMD_BAL_NONE && p.balance != EMD_BAL_MEAN) return false;
  if (p.tile < 0 || p.tile > kNumShapes) return false;
  if (p.launch_mode < 0 || p.launch_mode > 2) return false;
  if (p.debug_fault < 0 || p.debug_fault > 2) return false;
  if (p.norm != EMD_NORM_ANISO && p.norm != EMD_NORM_ISO) return false;
  return true;
}

int pick_shape(const emd_params &p, int B, const int *nt, const int *nr) {
  if (p.tile > 0) return p.tile - 1;
  int nr_max = 0;
  for (int b = 0; b < B; ++b) nr_max = std::max(nr_max, nr[b]);
  (void)nt;
  if (nr_max == 1) return 5;          // 1 x 248: one receiver
  if (nr_max <= 8) return 1;          // 8 x 120
  if (encode_fn()) return kTmaShape;  // 13 x 120, persistent, TMA-staged
  return 0;                           // 16 x 120
}

bool aligned256(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

// With tol > 0 the host checks the finished-gather count after every kPoll passes.
constexpr int kPoll = 64;
// A batched persistent solve with tol > 0 is re-dealt over the CTAs every kRebalance
// stopping tests (check_every passes each).
constexpr int kRebalance = 16;

// Enqueues fused passes on a stream: replays of one CUDA graph of kChunk passes,
// captured once per solve, plus plain launches for the remainder (launch_mode 1: plain
// launches only).
class PassLauncher {
 public:
  static constexpr int kChunk = 32;
  PassLauncher(const Shape &sh, const Ctl &ctl, int tiles, int mode)
      : sh_(sh), ctl_(ctl), tiles_(tiles), mode_(mode) {
    smem_ = iter_smem_bytes(sh);
    grid_ = sh.iter_tma ? std::min(tiles, sh.minb * sm_count()) : tiles;
  }
  ~PassLauncher() {
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
  }
  int launched = 0;  // kernel launches so far (graph nodes included)
  emd_status launch(int n, cudaStream_t stream) {
    launched += n;
    int done = 0;
    if (mode_ != 1 && n >= kChunk) {
      if (!exec_ && capture() != EMD_OK) return EMD_ERR_CUDA;
      for (; done + kChunk <= n; done += kChunk) EMD_CK(cudaGraphLaunch(exec_, stream));
    }
    for (; done < n; ++done) one(stream);
    EMD_CK(cudaGetLastError());
    return EMD_OK;
  }

 private:
  void one(cudaStream_t s) {
    if (sh_.iter_tma)
      sh_.iter_tma<<<grid_, emd::kTmaThreads, smem_, s>>>(ctl_, tiles_);
    else
      sh_.iter<<<grid_, kThreads, smem_, s>>>(ctl_);
  }
  emd_status capture() {
    cudaStream_t cs;
    EMD_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      for (int i = 0; i < kChunk; ++i) one(cs);
      ok = cudaStreamEndCapture(cs, &graph_) == cudaSuccess;
    }
    if (ok) ok = cudaGraphInstantiate(&exec_, graph_, 0) == cudaSuccess;
    cudaStreamDestroy(cs);
    if (!ok) {
      (void)cudaGetLastError();
      return EMD_ERR_CUDA;
    }
    return EMD_OK;
  }
  const Shape &sh_;
  Ctl ctl_;
  int tiles_, grid_ = 0, mode_;
  size_t smem_ = 0;
  cudaGraph_t graph_ = nullptr;
  cudaGraphExec_t exec_ = nullptr;
};

// Fills S.tmap: the gather's nine planes as one 3D float tensor {ntp, nr, 9} with
// strides (ntp * 4, plane bytes) and a box of (TI + 4) rows x 128 samples.
bool encode_tmap(Shot &S, void *base, size_t plane_bytes, int rows) {
  EncodeTiled enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(S.ntp), static_cast<cuuint64_t>(S.nr), 9u};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(S.ntp) * 4u, plane_bytes};
  const cuuint32_t box[3] = {128u, static_cast<cuuint32_t>(rows), 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return enc(&S.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// What a solve takes besides the public arguments: per-gather warm starts (the two-grid
// solve hands each gather its interpolated coarse solution; NULL arrays fall back to
// params' single warm start) and whether to run the finalize pass.  Without it nothing
// but the workspace is written -- the autotuner's trial solves must not touch phi and m,
// which may hold the warm start they read.
struct SolveExtra {
  const float *const *phi_init = nullptr;
  const float *const *m_init = nullptr;
  bool finalize = true;
  bool no_tune = false;   // tile 0 takes the untuned default shape (no timed trial solves)
  bool no_graph = false;  // per-pass fallback by plain launches (capturing a graph allocates)
  // ready[b]: recorded (on another stream) once gather b's inputs are in place.  Each
  // gather is then prepared by a launch of its own after waiting on its event, so the
  // preparation of the first gathers overlaps the copies of the later ones.
  const cudaEvent_t *ready = nullptr;
  // Enqueues the copies that `ready` waits on.  The first solve to reach its prepares (the
  // solve itself, or the autotuner's first trial) runs it once and clears it: the copies
  // are queued after that solve's small host tables, which are pageable copies -- queued
  // behind gigabytes of copies they would hold the host thread until those had finished,
  // and the prepares would be enqueued only after the copies instead of beside them.
  std::function<emd_status()> *stage = nullptr;
};

emd_status solve_impl(int B, const float *const *f_obs, const float *const *f_pred, const int *nt,
                      const int *nr, const double *dt, const double *dx, const emd_params *pp,
                      float *const *phi, float *const *m, emd_result *results, void *ws,
                      size_t ws_bytes, cudaStream_t stream, const SolveExtra &x = SolveExtra{});

// Tile-shape autotuner of the TMA pass.  The first default-tile solve of a (device,
// gather sizes) configuration times each TMA shape on the caller's own data -- two short
// fixed-iteration persistent solves per shape, whose difference is the per-pass cost --
// and keeps the fastest for the rest of the process.  The trial solves stop before the
// finalize pass, so they write the workspace only.
std::mutex g_tune_lock;
std::map<std::vector<long long>, int> g_tuned;

int autotune_shape(int B, const float *const *f_obs, const float *const *f_pred, const int *nt,
                   const int *nr, const double *dt, const double *dx, const emd_params &p,
                   float *const *phi, float *const *m, emd_result *results, void *ws,
                   size_t ws_bytes, cudaStream_t stream, const SolveExtra &x) {
  int dev = 0;
  (void)cudaGetDevice(&dev);
  std::vector<long long> key = {dev, B};
  for (int b = 0; b < B; ++b) {
    key.push_back(nt[b]);
    key.push_back(nr[b]);
  }
  std::lock_guard<std::mutex> guard(g_tune_lock);
  auto it = g_tuned.find(key);
  if (it != g_tuned.end()) return it->second;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return kTmaShape;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return kTmaShape;
  }
  auto timed = [&](int shape, int iters) -> float {
    emd_params q = p;
    q.tile = shape + 1;
    q.max_iter = iters;
    q.tol = 0.0;
    q.launch_mode = 0;  // the persistent solve, which default solves run
    q.trace = nullptr;
    q.debug_fault = 0;
    if (cudaEventRecord(e0, stream) != cudaSuccess) return -1.0f;
    SolveExtra trial = x;
    trial.finalize = false;
    if (solve_impl(B, f_obs, f_pred, nt, nr, dt, dx, &q, phi, m, results, ws, ws_bytes, stream,
                   trial) == EMD_ERR_CUDA)
      return -1.0f;
    float ms = -1.0f;
    if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      return -1.0f;
    return ms;
  };
  int best = kTmaShape;
  float best_t = 0.0f;
  for (int shape = kTmaFirst; shape < kNumShapes; ++shape) {
    (void)timed(shape, 4);  // first use: module load, attribute set-up
    const float t1 = timed(shape, 8), t2 = timed(shape, 40);
    if (t1 < 0.0f || t2 < 0.0f) continue;
    const float per_pass = (t2 - t1) / 32.0f;
    if (best_t == 0.0f || per_pass < best_t) {
      best_t = per_pass;
      best = shape;
    }
  }
  (void)cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g_tuned[key] = best;
  return best;
}

emd_status solve_impl(int B, const float *const *f_obs, const float *const *f_pred, const int *nt,
                      const int *nr, const double *dt, const double *dx, const emd_params *pp,
                      float *const *phi, float *const *m, emd_result *results, void *ws,
                      size_t ws_bytes, cudaStream_t stream, const SolveExtra &x) {
  emd_params p;
  emd_default_params(&p);
  if (pp) p = *pp;
  if (B < 1 || !f_obs || !f_pred || !nt || !nr || !dt || !dx || !phi || !m || !results)
    return EMD_ERR_ARG;
  if (!params_ok(p)) return EMD_ERR_ARG;
  if (B > 1 && (p.phi_init || p.m_init)) return EMD_ERR_ARG;
  for (int b = 0; b < B; ++b) {
    if (!size_ok(nt[b], nr[b])) return EMD_ERR_ARG;
    if (!f_obs[b] || !f_pred[b] || !phi[b] || !m[b]) return EMD_ERR_ARG;
    if (!(dt[b] > 0) || !std::isfinite(dt[b]) || !(dx[b] > 0) || !std::isfinite(dx[b]))
      return EMD_ERR_ARG;
  }
  const Layout L = layout(B, nt, nr);
  if (!ws || !aligned256(ws) || ws_bytes < L.total) return EMD_ERR_WORKSPACE;

  int si = pick_shape(p, B, nt, nr);
  if (uses_tma(kShapes[si]) && !encode_fn()) si = 0;  // no TMA descriptors: plain staging
  long long max_cells = 0;
  for (int b = 0; b < B; ++b) max_cells = std::max(max_cells, static_cast<long long>(nt[b]) * nr[b]);
  // Small gathers: one CTA per gather keeps the whole solve in shared memory.
  const bool resident = p.launch_mode == 0 && p.tile == 0 && max_cells <= emd::kResidentMaxCells;
  if (p.tile == 0 && !resident && si == kTmaShape && !x.no_tune)
    si = autotune_shape(B, f_obs, f_pred, nt, nr, dt, dx, p, phi, m, results, ws, ws_bytes, stream,
                        x);
  const Shape &sh = kShapes[si];
  char *base = static_cast<char *>(ws);

  std::vector<Shot> shots(B);
  std::vector<int> tile_shot;
  int nr_max = 0;
  for (int b = 0; b < B; ++b) {
    Shot &S = shots[b];
    std::memset(&S, 0, sizeof(S));
    S.p_obs = f_obs[b];
    S.p_pred = f_pred[b];
    S.phi_out = phi[b];
    S.m_out = m[b];
    S.phi_init = x.phi_init ? x.phi_init[b] : p.phi_init;
    S.m_init = x.m_init ? x.m_init[b] : p.m_init;
    S.nt = nt[b];
    S.nr = nr[b];
    S.ntp = ntp_of(nt[b]);
    const size_t pl = L.plane[b];
    char *g = base + L.gather[b];
    S.f = reinterpret_cast<float *>(g);
    for (int u = 0; u < 3; ++u) {
      S.ux[u] = reinterpret_cast<float *>(g + (1 + 2 * u) * pl);
      S.ut[u] = reinterpret_cast<float *>(g + (2 + 2 * u) * pl);
    }
    S.ph[0] = reinterpret_cast<float *>(g + 7 * pl);
    S.ph[1] = reinterpret_cast<float *>(g + 8 * pl);
    if (uses_tma(sh) && !encode_tmap(S, g, pl, sh.ti + 4)) return EMD_ERR_CUDA;
    S.tiles_j = (nt[b] + (sh.w - 8) - 1) / (sh.w - 8);
    S.tile0 = static_cast<int>(tile_shot.size());
    S.ntiles = tiles_of(sh, nt[b], nr[b]);
    tile_shot.insert(tile_shot.end(), S.ntiles, b);
    const bool one_d = nr[b] == 1;
    S.rdx = one_d ? 0.0f : static_cast<float>(1.0 / dx[b]);
    S.rdt = static_cast<float>(1.0 / dt[b]);
    S.area = one_d ? dt[b] : dx[b] * dt[b];
    S.lambda = 4.0 / (dt[b] * dt[b]) + (one_d ? 0.0 : 4.0 / (dx[b] * dx[b]));
    nr_max = std::max(nr_max, nr[b]);
  }
  const int grid = static_cast<int>(tile_shot.size());
  std::vector<int> march_run;  // marching solve: the gathers in march order (laid out at launch)
  if (sh.solve_march)
    for (int b = 0; b < B; ++b) march_run.push_back(b);

  State *states = reinterpret_cast<State *>(base + L.states);
  Shot *dshots = reinterpret_cast<Shot *>(base + L.shots);
  int *dtiles = reinterpret_cast<int *>(base + L.tiles);
  int *dunits = reinterpret_cast<int *>(base + L.units);
  int *n_done = reinterpret_cast<int *>(base + L.misc);
  int *err_flag = n_done + 1;
  double *acc = reinterpret_cast<double *>(base + L.acc);

  EMD_CK(cudaMemcpyAsync(dshots, shots.data(), sizeof(Shot) * B, cudaMemcpyHostToDevice, stream));
  EMD_CK(cudaMemcpyAsync(dtiles, tile_shot.data(), sizeof(int) * tile_shot.size(),
                         cudaMemcpyHostToDevice, stream));
  if (!march_run.empty())
    EMD_CK(cudaMemcpyAsync(dunits, march_run.data(), sizeof(int) * march_run.size(),
                           cudaMemcpyHostToDevice, stream));
  EMD_CK(cudaMemsetAsync(states, 0, sizeof(State) * B, stream));
  EMD_CK(cudaMemsetAsync(n_done, 0, 2 * sizeof(int), stream));
  EMD_CK(cudaMemsetAsync(acc, 0, sizeof(double) * emd::kAccBufs * emd::kSpread * emd::kAcc * B,
                         stream));

  Ctl ctl{};
  ctl.eps = p.eps;
  ctl.xi = p.xi;
  ctl.zeta = p.zeta;
  ctl.delta = p.delta;
  ctl.tol = p.tol;
  ctl.alpha0 = p.alpha0;
  ctl.max_iter = p.max_iter;
  ctl.check_every = p.check_every;
  ctl.ls_max_trials = p.ls_max_trials;
  ctl.linesearch = p.linesearch;
  ctl.balance = p.balance;
  ctl.debug_fault = p.debug_fault;
  ctl.iso = p.norm == EMD_NORM_ISO;
  ctl.shots = dshots;
  ctl.states = states;
  ctl.acc = acc;
  ctl.tile_shot = dtiles;
  ctl.march_run = dunits;
  ctl.march_nrun = static_cast<int>(march_run.size());
  ctl.n_done = n_done;
  ctl.error = err_flag;
  ctl.trace = p.trace;

  const size_t smem = smem_bytes(sh);
  if (sh.iter_tma)
    EMD_CK(cudaFuncSetAttribute(sh.iter_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(iter_smem_bytes(sh))));
  else
    EMD_CK(cudaFuncSetAttribute(sh.iter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem)));
  EMD_CK(cudaFuncSetAttribute(sh.fin, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(smem)));

  if (x.stage && *x.stage) {
    const std::function<emd_status()> enqueue = std::move(*x.stage);
    *x.stage = nullptr;
    const emd_status s = enqueue();
    if (s != EMD_OK) return s;
  }
  if (x.ready) {
    for (int b = 0; b < B; ++b) {
      EMD_CK(cudaStreamWaitEvent(stream, x.ready[b], 0));
      emd::k_prepare<<<dim3(std::min(nr[b], 128), 1), kThreads, 0, stream>>>(ctl, b);
      EMD_CK(cudaGetLastError());
    }
  } else {
    emd::k_prepare<<<dim3(std::min(nr_max, 128), B), kThreads, 0, stream>>>(ctl, 0);
    EMD_CK(cudaGetLastError());
  }

  int n_launch = x.ready ? B : 1;  // k_prepare
  if (resident) {
    const size_t rsmem = emd::resident_smem_bytes(max_cells);
    EMD_CK(cudaFuncSetAttribute(emd::k_solve_resident, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(rsmem)));
    emd::k_solve_resident<<<B, emd::kResThreads, rsmem, stream>>>(ctl);
    EMD_CK(cudaGetLastError());
    n_launch += 1;
  }
  // One cooperative launch for the whole solve, when the TMA pass is in use and every CTA
  // of the grid can be resident at once (its CTAs wait on one another between passes).
  // A batch solved to a tolerance runs in chunks of kRebalance checks instead: after each
  // chunk the host drops the gathers that have stopped and deals the tiles of the running
  // ones over every CTA again, so CTAs do not idle while the slowest gathers go on (the
  // per-gather counters are cumulative, so a chunk resumes where the last one stopped).
  bool persistent = false;
  if (!resident && p.launch_mode == 0 && (sh.solve_tma || sh.solve_march)) {
    const bool march = sh.solve_march != nullptr;
    void (*fn)(Ctl, int, int, int) = march ? sh.solve_march : sh.solve_tma;
    int dev = 0, coop = 0, per_sm = 0;
    const size_t tsmem = solve_smem_bytes(sh);
    const int tthreads = (sh.nw + (march ? 1 : 2)) * 32;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(tsmem)) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, tthreads, tsmem) == cudaSuccess &&
        per_sm >= 1) {
      const long long chunk =
          p.tol > 0.0 && B > 1 ? static_cast<long long>(kRebalance) * p.check_every : p.max_iter;
      const int cap = std::min(per_sm, sh.minb) * sm_count();  // co-resident CTAs
      // the chunk's work: tiles (tile pass) or strip-rows (march) of the running gathers
      std::vector<Shot> run_shots;
      long long items = static_cast<long long>(grid);  // the march's units are counted at launch
      int dealt = B;  // gathers the current work list was dealt for
      bool redealt = false;
      long long k0 = 0;
      while (k0 < p.max_iter) {
        const int kb = static_cast<int>(k0);
        const int ke = static_cast<int>(std::min<long long>(p.max_iter, k0 + chunk));
        int n_items = static_cast<int>(items), kb_ = kb, ke_ = ke;
        const int cgrid = march ? cap : std::min(n_items, cap);
        if (march && k0 == 0) {  // the units of the first deal and their warps
          run_shots = shots;
          items = march_layout(run_shots, march_run, static_cast<long long>(cgrid) * sh.nw, sh.nw);
          if (items < 0) return EMD_ERR_ARG;  // more units than an int counts
          n_items = static_cast<int>(items);
          EMD_CK(cudaMemcpyAsync(dshots, run_shots.data(), sizeof(Shot) * B, cudaMemcpyHostToDevice, stream));
        }
        Ctl cctl = ctl;
        void *args[] = {&cctl, &n_items, &kb_, &ke_};
        EMD_CK(cudaLaunchCooperativeKernel(reinterpret_cast<void *>(fn), dim3(cgrid), dim3(tthreads),
                                           args, tsmem, stream));
        persistent = true;
        n_launch += 1;
        k0 = ke;
        if (k0 >= p.max_iter) break;
        // which gathers are still running (and did a bounded wait give up)?
        std::vector<State> hs(B);
        int h_flags[2] = {0, 0};
        EMD_CK(cudaMemcpyAsync(hs.data(), states, sizeof(State) * B, cudaMemcpyDeviceToHost, stream));
        EMD_CK(cudaMemcpyAsync(h_flags, n_done, sizeof(h_flags), cudaMemcpyDeviceToHost, stream));
        EMD_CK(cudaStreamSynchronize(stream));
        if (h_flags[1] || h_flags[0] >= B) break;
        std::vector<int> running;
        for (int b = 0; b < B; ++b)
          if (!hs[b].done) running.push_back(b);
        if (static_cast<int>(running.size()) == dealt) continue;  // none stopped since the last deal
        // some gathers stopped: deal the running ones' work over every CTA again
        run_shots = shots;
        if (march) {
          // a new layout changes the gathers' units per pass: their cumulative counts of
          // finished units restart from k0 times the new count (no kernel is running now)
          items = march_layout(run_shots, running, static_cast<long long>(cap) * sh.nw, sh.nw);
          if (items < 0) return EMD_ERR_ARG;
          for (int b : running) hs[b].tiles_done = static_cast<unsigned>(k0) * static_cast<unsigned>(run_shots[b].nunits);
          ctl.march_nrun = static_cast<int>(running.size());
          EMD_CK(cudaMemcpyAsync(dunits, running.data(), sizeof(int) * running.size(),
                                 cudaMemcpyHostToDevice, stream));
          EMD_CK(cudaMemcpyAsync(states, hs.data(), sizeof(State) * B, cudaMemcpyHostToDevice, stream));
        } else {
          std::vector<int> next;
          for (int b : running) {
            run_shots[b].tile0 = static_cast<int>(next.size());
            next.insert(next.end(), shots[b].ntiles, b);
          }
          items = static_cast<long long>(next.size());
          EMD_CK(cudaMemcpyAsync(dtiles, next.data(), sizeof(int) * next.size(), cudaMemcpyHostToDevice,
                                 stream));
        }
        EMD_CK(cudaMemcpyAsync(dshots, run_shots.data(), sizeof(Shot) * B, cudaMemcpyHostToDevice, stream));
        dealt = static_cast<int>(running.size());
        redealt = true;
      }
      if (redealt) {  // the finalize pass walks every gather's tiles
        EMD_CK(cudaMemcpyAsync(dshots, shots.data(), sizeof(Shot) * B, cudaMemcpyHostToDevice, stream));
        EMD_CK(cudaMemcpyAsync(dtiles, tile_shot.data(), sizeof(int) * tile_shot.size(),
                               cudaMemcpyHostToDevice, stream));
      }
    }
    (void)cudaGetLastError();
  }
  PassLauncher passes(sh, ctl, grid, p.launch_mode == 1 || x.no_graph ? 1 : 2);
  if (persistent || resident) {
    // every pass already enqueued
  } else if (p.tol <= 0.0) {
    const emd_status s = passes.launch(p.max_iter, stream);
    if (s != EMD_OK) return s;
  } else {
    // Run in blocks of `poll` passes and stop once every gather reports done.
    const int poll = kPoll;
    int launched = 0;
    while (launched < p.max_iter) {
      const int n = std::min(poll, p.max_iter - launched);
      const emd_status s = passes.launch(n, stream);
      if (s != EMD_OK) return s;
      launched += n;
      int h_done = 0;
      EMD_CK(cudaMemcpyAsync(&h_done, n_done, sizeof(int), cudaMemcpyDeviceToHost, stream));
      EMD_CK(cudaStreamSynchronize(stream));
      if (h_done >= B) break;
    }
  }

  if (!x.finalize) return EMD_OK;  // an autotuner trial: the caller times the stream
  sh.fin<<<grid, kThreads, smem, stream>>>(ctl);
  EMD_CK(cudaGetLastError());
  n_launch += passes.launched + 1;

  std::vector<State> hs(B);
  int h_flags[2] = {0, 0};
  EMD_CK(cudaMemcpyAsync(hs.data(), states, sizeof(State) * B, cudaMemcpyDeviceToHost, stream));
  EMD_CK(cudaMemcpyAsync(h_flags, n_done, sizeof(h_flags), cudaMemcpyDeviceToHost, stream));
  EMD_CK(cudaStreamSynchronize(stream));
  if (h_flags[1]) {  // a bounded device wait gave up
    for (int b = 0; b < B; ++b) results[b].status = EMD_ERR_TIMEOUT;
    return EMD_ERR_TIMEOUT;
  }

  emd_status first = EMD_OK;
  for (int b = 0; b < B; ++b) {
    const State &st = hs[b];
    emd_result &r = results[b];
    const Shot &S = shots[b];
    const double *g = st.gap_sums;  // final u and phi: sum|u|, sum u^2, <phi,f>, h* terms
    r.dist = S.area * (g[0] + 0.5 * p.eps * g[1]);
    r.dist_l1 = S.area * g[0];
    r.mass_mu = st.mass_mu;
    r.mass_nu = st.mass_nu;
    r.imbalance = st.imbalance;
    // residual of the last iteration from its sums (the last pass measured u^K against u^{K-1})
    r.r_feas = st.fnorm > 0.0 ? std::sqrt(st.s_p2) / st.fnorm : std::sqrt(st.s_p2);
    r.r_step = std::sqrt(st.s_du2) / std::max(std::sqrt(st.s_u2), 1e-30);
    r.residual = std::max(r.r_feas, r.r_step);
    r.duality_gap = p.eps > 0.0 ? S.area * (g[0] + 0.5 * p.eps * g[1] - g[2] + g[3] / (2.0 * p.eps))
                                : std::nan("");
    r.alpha = st.alpha;
    r.theta = st.theta;
    r.iters = st.k;
    r.ls_trials = st.trials;
    r.status = st.status;
    r.launches = n_launch;
    r.tile = resident ? 0 : si + 1;
    if (first == EMD_OK && st.status != EMD_OK) first = static_cast<emd_status>(st.status);
  }
  return first;
}

// ---------------------------------------------------------------- two-grid solve

int coarse_nt(int nt, int r) { return (nt + r - 1) / r; }

bool mg_ok(const emd_mg_params &g) {
  return g.factor >= 1 && g.factor <= (1 << 16) && g.coarse_max_iter >= 1 &&
         std::isfinite(g.coarse_tol) && g.coarse_tol >= 0.0 &&
         (g.interpolate_phi == 0 || g.interpolate_phi == 1);
}

// Workspace of the two-grid solve: the coarse solve's workspace, then per gather the
// coarse gathers (obs, pred), the coarse solution (phi, m) and the job table.  The fine
// solve reuses the buffer from offset 0 once the interpolation has read the coarse
// solution (stream order), so the total is the larger of the two stages.
struct MgLayout {
  bool ok = false;
  size_t coarse_ws = 0, jobs = 0, total = 0;
  std::vector<int> ntc;
  std::vector<size_t> obs, pred, phi, m;
};

constexpr int kMaxMgGathers = 65535 / 3;  // interpolation jobs ride on gridDim.z

MgLayout mg_layout(int B, const int *nt, const int *nr, int r) {
  MgLayout M;
  if (B < 1 || B > kMaxMgGathers || r < 1) return M;
  for (int b = 0; b < B; ++b) {
    if (!size_ok(nt[b], nr[b])) return M;
    M.ntc.push_back(coarse_nt(nt[b], r));
    if (!size_ok(M.ntc[b], nr[b])) return M;  // fewer than two coarse samples
  }
  const Layout Lc = layout(B, M.ntc.data(), nr);
  M.coarse_ws = Lc.total;
  size_t off = align256(Lc.total);
  for (int b = 0; b < B; ++b) {
    const size_t n = sizeof(float) * static_cast<size_t>(nr[b]) * M.ntc[b];
    M.obs.push_back(off);
    off += align256(n);
    M.pred.push_back(off);
    off += align256(n);
    M.phi.push_back(off);
    off += align256(n);
    M.m.push_back(off);
    off += align256(2 * n);
  }
  M.jobs = off;
  off += align256(sizeof(emd::TimeJob) * 3u * B);
  M.total = std::max(off, layout(B, nt, nr).total);
  M.ok = true;
  return M;
}

emd_status mg_impl(int B, const float *const *f_obs, const float *const *f_pred, const int *nt,
                   const int *nr, const double *dt, const double *dx, const emd_params *pp,
                   const emd_mg_params *gp, float *const *phi, float *const *m,
                   emd_result *results, emd_result *coarse, void *ws, size_t ws_bytes,
                   cudaStream_t stream) {
  emd_params p;
  emd_default_params(&p);
  if (pp) p = *pp;
  emd_mg_params g;
  emd_default_mg_params(&g);
  if (gp) g = *gp;
  if (B < 1 || !f_obs || !f_pred || !nt || !nr || !dt || !dx || !phi || !m || !results)
    return EMD_ERR_ARG;
  if (!params_ok(p) || !mg_ok(g) || p.phi_init || p.m_init) return EMD_ERR_ARG;
  for (int b = 0; b < B; ++b) {
    if (!f_obs[b] || !f_pred[b] || !phi[b] || !m[b]) return EMD_ERR_ARG;
    if (!(dt[b] > 0) || !std::isfinite(dt[b]) || !(dx[b] > 0) || !std::isfinite(dx[b]))
      return EMD_ERR_ARG;
  }
  const MgLayout M = mg_layout(B, nt, nr, g.factor);
  if (!M.ok) return EMD_ERR_ARG;
  if (!ws || !aligned256(ws) || ws_bytes < M.total) return EMD_ERR_WORKSPACE;
  char *base = static_cast<char *>(ws);
  const int r = g.factor;

  // 1. restriction of both gathers (one launch for every gather)
  std::vector<const float *> obs_c(B), pred_c(B);
  std::vector<float *> phi_c(B), m_c(B);
  std::vector<double> dt_c(B);
  std::vector<emd::TimeJob> jobs;
  long long cells_c = 0;
  for (int b = 0; b < B; ++b) {
    float *o = reinterpret_cast<float *>(base + M.obs[b]);
    float *q = reinterpret_cast<float *>(base + M.pred[b]);
    obs_c[b] = o;
    pred_c[b] = q;
    phi_c[b] = reinterpret_cast<float *>(base + M.phi[b]);
    m_c[b] = reinterpret_cast<float *>(base + M.m[b]);
    dt_c[b] = dt[b] * r;
    jobs.push_back({f_obs[b], o, nr[b], nt[b], M.ntc[b], r, 0, 0, 0});
    jobs.push_back({f_pred[b], q, nr[b], nt[b], M.ntc[b], r, 0, 0, 0});
    cells_c = std::max(cells_c, static_cast<long long>(nr[b]) * M.ntc[b]);
  }
  emd::TimeJob *djobs = reinterpret_cast<emd::TimeJob *>(base + M.jobs);
  EMD_CK(cudaMemcpyAsync(djobs, jobs.data(), sizeof(emd::TimeJob) * jobs.size(),
                         cudaMemcpyHostToDevice, stream));
  const int rgrid = static_cast<int>(
      std::min<long long>((cells_c + emd::kRestrictThreads - 1) / emd::kRestrictThreads, 4096));
  emd::k_restrict_time<<<dim3(rgrid, static_cast<unsigned>(jobs.size())), emd::kRestrictThreads,
                         0, stream>>>(djobs, emd::TimeJob{});
  EMD_CK(cudaGetLastError());

  // 2. the coarse solve (Algorithm 1 on the coarse grids, spacing r dt)
  emd_params q = p;
  q.max_iter = g.coarse_max_iter;
  q.tol = g.coarse_tol;
  q.trace = nullptr;
  std::vector<emd_result> cres(B);
  const emd_status cs = solve_impl(B, obs_c.data(), pred_c.data(), M.ntc.data(), nr, dt_c.data(),
                                   dx, &q, phi_c.data(), m_c.data(), cres.data(), ws, M.coarse_ws,
                                   stream);
  if (coarse)
    for (int b = 0; b < B; ++b) coarse[b] = cres[b];
  if (cs != EMD_OK) {
    for (int b = 0; b < B; ++b) {
      std::memset(&results[b], 0, sizeof(emd_result));
      results[b].status = cres[b].status != EMD_OK ? cres[b].status : cs;
      results[b].launches = cres[b].launches + 1;
    }
    return cs;
  }

  // 3. sinc interpolation of the coarse solution into phi and m (one launch)
  jobs.clear();
  int nt_max = 0, nr_max = 0;
  for (int b = 0; b < B; ++b) {
    const size_t nc = static_cast<size_t>(nr[b]) * M.ntc[b];
    const size_t nf = static_cast<size_t>(nr[b]) * nt[b];
    if (g.interpolate_phi) jobs.push_back({phi_c[b], phi[b], nr[b], M.ntc[b], nt[b], r, 0, 0, 0});
    jobs.push_back({m_c[b], m[b], nr[b], M.ntc[b], nt[b], r, 0, 1, 0});
    jobs.push_back({m_c[b] + nc, m[b] + nf, nr[b], M.ntc[b], nt[b], r, 1, 0, 1});
    nt_max = std::max(nt_max, nt[b]);
    nr_max = std::max(nr_max, nr[b]);
  }
  EMD_CK(cudaMemcpyAsync(djobs, jobs.data(), sizeof(emd::TimeJob) * jobs.size(),
                         cudaMemcpyHostToDevice, stream));
  const dim3 pgrid((nt_max + emd::kIpBN - 1) / emd::kIpBN, (nr_max + emd::kIpBM - 1) / emd::kIpBM,
                   static_cast<unsigned>(jobs.size()));
  emd::k_prolong_time<<<pgrid, emd::kIpThreads, 0, stream>>>(djobs, emd::TimeJob{});
  EMD_CK(cudaGetLastError());

  // 4. the fine solve, warm-started from phi and m in place (its prepare pass copies them
  //    into the workspace before anything writes phi or m again)
  std::vector<const float *> phi_init(phi, phi + B), m_init(m, m + B);
  SolveExtra x;
  x.phi_init = g.interpolate_phi ? phi_init.data() : nullptr;
  x.m_init = m_init.data();
  const emd_status fs = solve_impl(B, f_obs, f_pred, nt, nr, dt, dx, &p, phi, m, results, ws,
                                   ws_bytes, stream, x);
  for (int b = 0; b < B; ++b) results[b].launches += cres[b].launches + 2;
  return fs;
}

}  // namespace

namespace emd_internal {

// emd_dyn_solve for the no-allocation entry point (emd_noalloc.cu): no autotuner trials
// and no CUDA graph.  Not exported.
__attribute__((visibility("hidden"))) emd_status solve_without_allocation(
    const float *f_obs, const float *f_pred, int nt, int nr, double dt, double dx,
    const emd_params *params, float *phi, float *m, emd_result *result, void *workspace,
    size_t ws_bytes, cudaStream_t stream) {
  SolveExtra x;
  x.no_tune = true;
  x.no_graph = true;
  return solve_impl(1, &f_obs, &f_pred, &nt, &nr, &dt, &dx, params, &phi, &m, result, workspace,
                    ws_bytes, stream, x);
}

}  // namespace emd_internal

extern "C" {

void emd_default_params(emd_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->eps = 1e-4;
  p->xi = 0.5;
  p->zeta = 0.99;
  p->delta = 1e5;
  p->alpha0 = 0.0;
  p->tol = 0.0;
  p->max_iter = 2000;
  p->check_every = 10;
  p->ls_max_trials = 40;
  p->linesearch = 1;
  p->ls_norm = 2;
  p->balance = EMD_BAL_MEAN;
  p->phi_init = nullptr;
  p->m_init = nullptr;
  p->tile = 0;
  p->launch_mode = 0;
  p->debug_fault = 0;
  p->trace = nullptr;
  p->norm = EMD_NORM_ANISO;
}

int emd_tile_count(void) { return kNumShapes; }

size_t emd_workspace_size(int nt, int nr) {
  if (!size_ok(nt, nr)) return 0;
  return layout(1, &nt, &nr).total;
}

size_t emd_batched_workspace_size(int B, const int *nt, const int *nr) {
  if (B < 1 || !nt || !nr) return 0;
  for (int b = 0; b < B; ++b)
    if (!size_ok(nt[b], nr[b])) return 0;
  return layout(B, nt, nr).total;
}

emd_status emd_dyn_solve(const float *f_obs, const float *f_pred, int nt, int nr, double dt,
                         double dx, const emd_params *params, float *phi, float *m,
                         emd_result *result, void *workspace, size_t ws_bytes,
                         emd_stream_t stream) {
  return solve_impl(1, &f_obs, &f_pred, &nt, &nr, &dt, &dx, params, &phi, &m, result, workspace,
                    ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

emd_status emd_dyn_solve_batched(int B, const float *const *f_obs, const float *const *f_pred,
                                 const int *nt, const int *nr, const double *dt,
                                 const double *dx, const emd_params *params,
                                 float *const *phi, float *const *m, emd_result *results,
                                 void *workspace, size_t ws_bytes, emd_stream_t stream) {
  return solve_impl(B, f_obs, f_pred, nt, nr, dt, dx, params, phi, m, results, workspace,
                    ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

emd_status emd_decompose(const float *f_obs, const float *f_pred, int nt, int nr, double dt,
                         double dx, float *mu, float *nu, double *masses, void *workspace,
                         size_t ws_bytes, emd_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!f_obs || !f_pred || !size_ok(nt, nr)) return EMD_ERR_ARG;
  if (!(dt > 0) || !std::isfinite(dt) || !(dx > 0) || !std::isfinite(dx)) return EMD_ERR_ARG;
  const Layout L = layout(1, &nt, &nr);
  if (!workspace || !aligned256(workspace) || ws_bytes < L.total) return EMD_ERR_WORKSPACE;
  double *acc = reinterpret_cast<double *>(static_cast<char *>(workspace) + L.misc + 64);
  const size_t n = static_cast<size_t>(nt) * nr;
  EMD_CK(cudaMemsetAsync(acc, 0, 2 * sizeof(double), stream));
  const int blocks = static_cast<int>(std::min<size_t>((n + kThreads - 1) / kThreads, 2048));
  emd::k_decompose<<<blocks, kThreads, 0, stream>>>(f_obs, f_pred, n, mu, nu, acc);
  EMD_CK(cudaGetLastError());
  if (masses) {
    double h[2];
    EMD_CK(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, stream));
    EMD_CK(cudaStreamSynchronize(stream));
    const double area = nr == 1 ? dt : dx * dt;
    masses[0] = area * h[0];
    masses[1] = area * h[1];
  }
  return EMD_OK;
}

emd_status emd_adjoint(const float *phi, int nt, int nr, double dt, double dx, int balance,
                       const float *grad_out, float *grad_pred, float *grad_obs,
                       void *workspace, size_t ws_bytes, emd_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!phi || !grad_pred || !size_ok(nt, nr)) return EMD_ERR_ARG;
  if (balance != EMD_BAL_NONE && balance != EMD_BAL_MEAN) return EMD_ERR_ARG;
  if (!(dt > 0) || !std::isfinite(dt) || !(dx > 0) || !std::isfinite(dx)) return EMD_ERR_ARG;
  const Layout L = layout(1, &nt, &nr);
  if (!workspace || !aligned256(workspace) || ws_bytes < L.total) return EMD_ERR_WORKSPACE;
  double *acc = reinterpret_cast<double *>(static_cast<char *>(workspace) + L.misc + 128);
  const size_t n = static_cast<size_t>(nt) * nr;
  const int blocks = static_cast<int>(std::min<size_t>((n + kThreads - 1) / kThreads, 2048));
  const double area = nr == 1 ? dt : dx * dt;
  if (balance == EMD_BAL_MEAN) {
    EMD_CK(cudaMemsetAsync(acc, 0, sizeof(double), stream));
    emd::k_adj_sum<<<blocks, kThreads, 0, stream>>>(phi, n, acc);
    EMD_CK(cudaGetLastError());
  }
  emd::k_adj_scale<<<blocks, kThreads, 0, stream>>>(phi, n, area, balance, acc, grad_out,
                                                     grad_pred, grad_obs);
  EMD_CK(cudaGetLastError());
  return EMD_OK;
}

size_t emd_batched_adjoint_workspace_size(int B) {
  if (B < 1) return 0;
  return align256(sizeof(emd::AdjJob) * static_cast<size_t>(B)) + align256(sizeof(double) * B);
}

emd_status emd_adjoint_batched(int B, const float *const *phi, const int *nt, const int *nr,
                               const double *dt, const double *dx, int balance,
                               const float *grad_out, float *const *grad_pred,
                               float *const *grad_obs, void *workspace, size_t ws_bytes,
                               emd_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (B < 1 || !phi || !nt || !nr || !dt || !dx || !grad_pred) return EMD_ERR_ARG;
  if (balance != EMD_BAL_NONE && balance != EMD_BAL_MEAN) return EMD_ERR_ARG;
  if (B > 65535) return EMD_ERR_ARG;  // gathers ride on gridDim.y
  std::vector<emd::AdjJob> jobs(B);
  long long n_max = 0;
  for (int b = 0; b < B; ++b) {
    if (!phi[b] || !grad_pred[b] || !size_ok(nt[b], nr[b])) return EMD_ERR_ARG;
    if (!(dt[b] > 0) || !std::isfinite(dt[b]) || !(dx[b] > 0) || !std::isfinite(dx[b]))
      return EMD_ERR_ARG;
    emd::AdjJob &J = jobs[b];
    J.phi = phi[b];
    J.gp = grad_pred[b];
    J.go = grad_obs ? grad_obs[b] : nullptr;
    J.grad_out = grad_out ? grad_out + b : nullptr;
    J.n = static_cast<long long>(nt[b]) * nr[b];
    J.area = nr[b] == 1 ? dt[b] : dx[b] * dt[b];
    n_max = std::max(n_max, J.n);
  }
  const size_t need = emd_batched_adjoint_workspace_size(B);
  if (!workspace || !aligned256(workspace) || ws_bytes < need) return EMD_ERR_WORKSPACE;
  char *base = static_cast<char *>(workspace);
  emd::AdjJob *djobs = reinterpret_cast<emd::AdjJob *>(base);
  double *acc = reinterpret_cast<double *>(base + align256(sizeof(emd::AdjJob) * static_cast<size_t>(B)));
  EMD_CK(cudaMemcpyAsync(djobs, jobs.data(), sizeof(emd::AdjJob) * B, cudaMemcpyHostToDevice, stream));
  // about two waves of 256-thread blocks over the largest gather, at most 4 cells per thread
  const int bx = static_cast<int>(std::max<long long>(
      1, std::min<long long>((n_max + 4ll * kThreads - 1) / (4ll * kThreads),
                             std::max(1, 2 * 8 * sm_count() / B))));
  if (balance == EMD_BAL_MEAN) {
    EMD_CK(cudaMemsetAsync(acc, 0, sizeof(double) * B, stream));
    emd::k_adj_sum_batched<<<dim3(bx, B), kThreads, 0, stream>>>(djobs, acc);
    EMD_CK(cudaGetLastError());
  }
  emd::k_adj_scale_batched<<<dim3(bx, B), kThreads, 0, stream>>>(djobs, acc, balance);
  EMD_CK(cudaGetLastError());
  return EMD_OK;
}

size_t emd_misfit_batched_host_workspace_size(int B, const int *nt, const int *nr) {
  const size_t solve = emd_batched_workspace_size(B, nt, nr);
  if (solve == 0) return 0;
  size_t t = align256(solve) + align256(emd_batched_adjoint_workspace_size(B));
  for (int b = 0; b < B; ++b) {
    const size_t plane = sizeof(float) * static_cast<size_t>(nt[b]) * nr[b];
    t += 3 * align256(plane) + align256(2 * plane);  // obs (then the adjoint source), pred, phi; m
  }
  return t;
}

emd_status emd_misfit_batched_host(int B, const float *const *f_obs, const float *const *f_pred,
                                   const int *nt, const int *nr, const double *dt,
                                   const double *dx, const emd_params *params,
                                   float *const *grad_pred, emd_result *results, void *workspace,
                                   size_t ws_bytes, emd_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  emd_params p;
  emd_default_params(&p);
  if (params) p = *params;
  if (B < 1 || B > 65535 || !f_obs || !f_pred || !nt || !nr || !dt || !dx || !results)
    return EMD_ERR_ARG;
  if (!params_ok(p) || p.phi_init || p.m_init) return EMD_ERR_ARG;
  for (int b = 0; b < B; ++b) {
    if (!f_obs[b] || !f_pred[b] || !size_ok(nt[b], nr[b])) return EMD_ERR_ARG;
    if (!(dt[b] > 0) || !std::isfinite(dt[b]) || !(dx[b] > 0) || !std::isfinite(dx[b]))
      return EMD_ERR_ARG;
  }
  const size_t need = emd_misfit_batched_host_workspace_size(B, nt, nr);
  if (!workspace || !aligned256(workspace) || ws_bytes < need) return EMD_ERR_WORKSPACE;

  // workspace: the solve's, the adjoint's, then per gather obs | pred | phi | m
  const size_t solve_ws = emd_batched_workspace_size(B, nt, nr);
  const size_t adj_ws = emd_batched_adjoint_workspace_size(B);
  char *base = static_cast<char *>(workspace);
  char *q = base + align256(solve_ws) + align256(adj_ws);
  std::vector<const float *> d_obs(B), d_pred(B);
  std::vector<float *> d_gp(B), d_phi(B), d_m(B);
  std::vector<size_t> bytes(B);
  for (int b = 0; b < B; ++b) {
    bytes[b] = sizeof(float) * static_cast<size_t>(nt[b]) * nr[b];
    d_gp[b] = reinterpret_cast<float *>(q);  // the adjoint source reuses the obs staging
    d_obs[b] = d_gp[b];
    q += align256(bytes[b]);
    d_pred[b] = reinterpret_cast<const float *>(q);
    q += align256(bytes[b]);
    d_phi[b] = reinterpret_cast<float *>(q);
    q += align256(bytes[b]);
    d_m[b] = reinterpret_cast<float *>(q);
    q += align256(2 * bytes[b]);
  }

  // The copies run on a stream of this call, ordered after the caller's earlier work on
  // `stream`; each gather's event lets its preparation start as soon as it has landed.
  struct Owned {
    cudaStream_t cs = nullptr;
    std::vector<cudaEvent_t> ev;
    ~Owned() {
      if (cs) {
        (void)cudaStreamSynchronize(cs);  // no copy may still write the workspace on return
        (void)cudaStreamDestroy(cs);
      }
      for (cudaEvent_t e : ev) (void)cudaEventDestroy(e);
    }
  } own;
  EMD_CK(cudaStreamCreateWithFlags(&own.cs, cudaStreamNonBlocking));
  own.ev.reserve(B + 1);
  for (int i = 0; i <= B; ++i) {
    cudaEvent_t e;
    EMD_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    own.ev.push_back(e);
  }
  EMD_CK(cudaEventRecord(own.ev[B], stream));
  EMD_CK(cudaStreamWaitEvent(own.cs, own.ev[B], 0));
  std::function<emd_status()> stage = [&]() -> emd_status {
    for (int b = 0; b < B; ++b) {
      EMD_CK(cudaMemcpyAsync(d_gp[b], f_obs[b], bytes[b], cudaMemcpyHostToDevice, own.cs));
      EMD_CK(cudaMemcpyAsync(const_cast<float *>(d_pred[b]), f_pred[b], bytes[b],
                             cudaMemcpyHostToDevice, own.cs));
      EMD_CK(cudaEventRecord(own.ev[b], own.cs));
    }
    return EMD_OK;
  };

  SolveExtra x;
  x.ready = own.ev.data();
  x.stage = &stage;
  const emd_status st = solve_impl(B, d_obs.data(), d_pred.data(), nt, nr, dt, dx, &p, d_phi.data(),
                                   d_m.data(), results, base, solve_ws, stream, x);
  if (st == EMD_ERR_ARG || st == EMD_ERR_CUDA || st == EMD_ERR_TIMEOUT || st == EMD_ERR_WORKSPACE)
    return st;
  if (grad_pred) {
    const emd_status sa = emd_adjoint_batched(B, d_phi.data(), nt, nr, dt, dx, p.balance, nullptr,
                                              d_gp.data(), nullptr, base + align256(solve_ws),
                                              adj_ws, stream_);
    if (sa != EMD_OK) return sa;
    for (int b = 0; b < B; ++b)
      if (grad_pred[b])
        EMD_CK(cudaMemcpyAsync(grad_pred[b], d_gp[b], bytes[b], cudaMemcpyDeviceToHost, stream));
    EMD_CK(cudaStreamSynchronize(stream));
  }
  return st;
}

void emd_default_mg_params(emd_mg_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->factor = 10;
  p->coarse_max_iter = 150;
  p->coarse_tol = 0.0;
  p->interpolate_phi = 1;
}

size_t emd_mg_workspace_size(int nt, int nr, int factor) {
  const MgLayout M = mg_layout(1, &nt, &nr, factor);
  return M.ok ? M.total : 0;
}

size_t emd_batched_mg_workspace_size(int B, const int *nt, const int *nr, int factor) {
  if (B < 1 || !nt || !nr) return 0;
  const MgLayout M = mg_layout(B, nt, nr, factor);
  return M.ok ? M.total : 0;
}

emd_status emd_restrict_time(const float *in, int nt, int nr, int factor, float *out,
                             emd_stream_t stream) {
  if (!in || !out || factor < 1 || factor > (1 << 16) || !size_ok(nt, nr)) return EMD_ERR_ARG;
  const int nc = coarse_nt(nt, factor);
  const long long cells = static_cast<long long>(nr) * nc;
  const int grid = static_cast<int>(
      std::min<long long>((cells + emd::kRestrictThreads - 1) / emd::kRestrictThreads, 4096));
  emd::k_restrict_time<<<dim3(grid, 1), emd::kRestrictThreads, 0,
                         reinterpret_cast<cudaStream_t>(stream)>>>(
      nullptr, emd::TimeJob{in, out, nr, nt, nc, factor, 0, 0, 0});
  EMD_CK(cudaGetLastError());
  return EMD_OK;
}

emd_status emd_prolong_time(const float *in, int nc, int nr, int factor, int nt, int staggered,
                            int zero_row0, int zero_col0, float *out, emd_stream_t stream) {
  if (!in || !out || factor < 1 || factor > (1 << 16) || nc < 1 || nt < 1) return EMD_ERR_ARG;
  if (!size_ok(std::max(nt, 2), nr) || !size_ok(std::max(nc, 2), nr)) return EMD_ERR_ARG;
  if (static_cast<long long>(factor) * nc > (1ll << 28)) return EMD_ERR_ARG;  // 2 r J fits an int
  if ((staggered | zero_row0 | zero_col0) & ~1) return EMD_ERR_ARG;
  const dim3 grid((nt + emd::kIpBN - 1) / emd::kIpBN, (nr + emd::kIpBM - 1) / emd::kIpBM, 1);
  emd::k_prolong_time<<<grid, emd::kIpThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      nullptr, emd::TimeJob{in, out, nr, nc, nt, factor, staggered, zero_row0, zero_col0});
  EMD_CK(cudaGetLastError());
  return EMD_OK;
}

emd_status emd_dyn_solve_mg(const float *f_obs, const float *f_pred, int nt, int nr, double dt,
                            double dx, const emd_params *params, const emd_mg_params *mg,
                            float *phi, float *m, emd_result *result, emd_result *coarse,
                            void *workspace, size_t ws_bytes, emd_stream_t stream) {
  return mg_impl(1, &f_obs, &f_pred, &nt, &nr, &dt, &dx, params, mg, &phi, &m, result, coarse,
                 workspace, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

emd_status emd_dyn_solve_batched_mg(int B, const float *const *f_obs,
                                    const float *const *f_pred, const int *nt, const int *nr,
                                    const double *dt, const double *dx,
                                    const emd_params *params, const emd_mg_params *mg,
                                    float *const *phi, float *const *m, emd_result *results,
                                    emd_result *coarse, void *workspace, size_t ws_bytes,
                                    emd_stream_t stream) {
  return mg_impl(B, f_obs, f_pred, nt, nr, dt, dx, params, mg, phi, m, results, coarse,
                 workspace, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

emd_status emd_lsd(const float *f_obs, const float *f_pred, int nt, int nr, double dt, double dx,
                   double *value, float *grad_pred, float *grad_obs, void *workspace,
                   size_t ws_bytes, emd_stream_t stream_) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!f_obs || !f_pred || !size_ok(nt, nr)) return EMD_ERR_ARG;
  if (!(dt > 0) || !std::isfinite(dt) || !(dx > 0) || !std::isfinite(dx)) return EMD_ERR_ARG;
  if (!workspace || !aligned256(workspace) || ws_bytes < 256) return EMD_ERR_WORKSPACE;
  double *acc = static_cast<double *>(workspace);
  const size_t n = static_cast<size_t>(nt) * nr;
  const double area = nr == 1 ? dt : dx * dt;
  EMD_CK(cudaMemsetAsync(acc, 0, sizeof(double), stream));
  const int blocks = static_cast<int>(std::min<size_t>((n + kThreads - 1) / kThreads, 2048));
  emd::k_lsd<<<blocks, kThreads, 0, stream>>>(f_obs, f_pred, n, static_cast<float>(area), grad_pred,
                                              grad_obs, acc);
  EMD_CK(cudaGetLastError());
  if (value) {
    double h = 0.0;
    EMD_CK(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, stream));
    EMD_CK(cudaStreamSynchronize(stream));
    *value = 0.5 * area * h;
  }
  return EMD_OK;
}

const char *emd_status_string(emd_status s) {
  switch (s) {
    case EMD_OK: return "ok";
    case EMD_ERR_ARG: return "invalid argument";
    case EMD_ERR_CUDA: return "CUDA error";
    case EMD_ERR_NONFINITE: return "non-finite iterate";
    case EMD_ERR_LINESEARCH: return "linesearch did not terminate";
    case EMD_ERR_TIMEOUT: return "device wait timed out";
    case EMD_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
  }
  return "unknown status";
}

}  // extern "C"
