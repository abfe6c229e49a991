// vio_detect_grid_noalloc: grid-cell detection for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside a
// pre-sized memory pool or under a device-memory budget that forbids new
// allocations, plugins hosted by a runtime that owns every allocation, and
// real-time loops where an allocation (which can synchronise the device) is
// not allowed. vio_detect_grid needs a vio_ctx, and creating one allocates
// the per-cell candidate scratch. This variant instead uses a scratch array
// that is part of the library image itself: a file-scope __device__ array of
// fixed size, which every GPU that loads the library holds until the process
// exits. The caller still passes the inputs and outputs.
//
// Host code cannot use the array's name as a device address (in host code
// that symbol is only a stand-in), so the first call on each device looks the
// address up with cudaGetSymbolAddress while that device is current, checks
// the result, and caches it; later calls on that device reuse it. Make that
// first call before any stream capture.
//
// Every call shares the one array: two calls that overlap on the GPU (on
// different streams, or from different threads without ordering) race on it
// and must not be issued. Each call writes every scratch entry it later
// reads, so nothing needs clearing between calls.
#include <mutex>

#include "common.cuh"
#include "detect_dev.cuh"

namespace {

// VIO_NOALLOC_MAX_CELL_SLOTS packed candidate keys plus one count per cell.
static __device__ __align__(256) unsigned long long g_noalloc_cand[VIO_NOALLOC_MAX_CELL_SLOTS];
static __device__ __align__(256) int32_t g_noalloc_count[VIO_NOALLOC_MAX_CELL_SLOTS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long* g_cand_ptr[kMaxDevices] = {};
int32_t* g_count_ptr[kMaxDevices] = {};

// Device addresses of the scratch arrays for the current device (looked up
// once per device).
bool scratch_for_current_device(unsigned long long** cand, int32_t** count) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_cand_ptr[dev]) {
    void* a = nullptr;
    void* b = nullptr;
    if (cudaGetSymbolAddress(&a, g_noalloc_cand) != cudaSuccess || !a) return false;
    if (cudaGetSymbolAddress(&b, g_noalloc_count) != cudaSuccess || !b) return false;
    g_cand_ptr[dev] = (unsigned long long*)a;
    g_count_ptr[dev] = (int32_t*)b;
  }
  *cand = g_cand_ptr[dev];
  *count = g_count_ptr[dev];
  return true;
}

}  // namespace

extern "C" vio_status vio_detect_grid_noalloc(const vio_params* p, const vio_pyr_layout* layout,
                                              const vio_pyr_batch* batch,
                                              const uint8_t* d_occupancy, const uint8_t* d_mask,
                                              int64_t mask_stride, float* d_kp, int16_t* d_score,
                                              int32_t* d_count, int32_t capacity,
                                              void* stream) {
  if (!vio::detect_params_ok(p) || p->n_levels < 1 || p->n_levels > VIO_MAX_LEVELS ||
      !layout || layout->n_levels < 1 || layout->w[0] < 1 ||
      layout->h[0] < 1 || layout->pitch[0] < layout->w[0])
    return VIO_ERR_INVALID_ARG;
  if (!batch || batch->n_images < 1 || !batch->d_level0 || !d_kp || !d_score || !d_count ||
      capacity < 0)
    return VIO_ERR_INVALID_ARG;
  if (batch->n_images > 1 && batch->level0_stride < (int64_t)layout->pitch[0] * layout->h[0])
    return VIO_ERR_INVALID_ARG;
  if (d_mask && batch->n_images > 1 && mask_stride < (int64_t)layout->w[0] * layout->h[0])
    return VIO_ERR_INVALID_ARG;
  if (!vio::det::detect_fits(p->cell_w, p->cell_h, p->k_per_cell))
    return VIO_ERR_UNSUPPORTED;
  const long long cells = (long long)(layout->w[0] / p->cell_w) * (layout->h[0] / p->cell_h);
  // the fixed scratch bounds the work of one call (k >= 1, so the count array,
  // one entry per cell, is within its bound whenever the key slots are)
  if ((long long)batch->n_images * cells * p->k_per_cell > VIO_NOALLOC_MAX_CELL_SLOTS ||
      batch->n_images > 65535)
    return VIO_ERR_UNSUPPORTED;
  unsigned long long* cand = nullptr;
  int32_t* count = nullptr;
  if (!scratch_for_current_device(&cand, &count)) return VIO_ERR_CUDA;
  const cudaError_t e = vio::launch_detect(*p, vio::make_geom(*layout), vio::make_batch(*batch),
                                           d_occupancy, d_mask, mask_stride, cand, count, d_kp,
                                           d_score, d_count, capacity, (cudaStream_t)stream);
  return e == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}
