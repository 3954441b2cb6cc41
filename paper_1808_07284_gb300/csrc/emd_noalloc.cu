// emd_dyn_solve_noalloc: one EMD solve with no device allocation by anyone.
//
// Some callers cannot call cudaMalloc: code whose host framework owns every device
// allocation (a custom allocator, a fixed memory budget), a real-time loop that must never
// block on the allocator, or a plug-in handed only its input and output buffers.  This
// entry point serves them.  Its scratch space is a file-scope device array compiled into
// the library, so every GPU that loads the library holds kScratchBytes of it until the
// process exits.  The solve itself takes no step that allocates behind the caller's back:
// no autotuner trial solves and no CUDA graph (see solve_without_allocation).
//
// The array's name in host code is only a host-side stand-in: passing it to a kernel
// would fault (or, where the GPU can reach host memory, silently use the wrong memory).
// The device address comes from cudaGetSymbolAddress, called once per device, with that
// device current, on the first call made on it.
#include <cuda_runtime.h>

#include <mutex>

#include "emd_gb300.h"

namespace emd_internal {
emd_status solve_without_allocation(const float *f_obs, const float *f_pred, int nt, int nr,
                                    double dt, double dx, const emd_params *params, float *phi,
                                    float *m, emd_result *result, void *workspace,
                                    size_t ws_bytes, cudaStream_t stream);
}

namespace {

constexpr size_t kScratchBytes = static_cast<size_t>(16) << 20;  // 16 MiB per GPU
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_lock;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (set up on the first call there).
emd_status scratch_address(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return EMD_ERR_CUDA;
  }
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return EMD_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return EMD_OK;
}

}  // namespace

extern "C" emd_status emd_dyn_solve_noalloc(const float *f_obs, const float *f_pred, int nt,
                                            int nr, double dt, double dx,
                                            const emd_params *params, float *phi, float *m,
                                            emd_result *result, emd_stream_t stream) {
  const size_t need = emd_workspace_size(nt, nr);
  if (need == 0) return EMD_ERR_ARG;
  if (need > kScratchBytes) return EMD_ERR_WORKSPACE;  // gather too large for the built-in scratch
  emd_params p;
  emd_default_params(&p);
  if (params) p = *params;
  if (p.launch_mode == 2) p.launch_mode = 1;  // graph replays would instantiate a graph
  void *ws = nullptr;
  const emd_status s = scratch_address(&ws);
  if (s != EMD_OK) return s;
  // The solve clears everything that must start at zero (state, accumulators, counters)
  // and rewrites every plane it reads, so the previous call's contents do not matter.
  return emd_internal::solve_without_allocation(f_obs, f_pred, nt, nr, dt, dx, &p, phi, m, result,
                                                ws, kScratchBytes,
                                                reinterpret_cast<cudaStream_t>(stream));
}
