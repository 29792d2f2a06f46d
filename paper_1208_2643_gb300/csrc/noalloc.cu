// Allocation-free variant of the mass reduction (see mpfc_mass_noalloc in include/mpfc.h).
//
// mpfc_mass sums phi through a handle whose partial sums live in the caller's
// workspace.  This entry point needs neither a handle nor a workspace: its partial
// sums live in a file-scope static device array, so a caller that holds only a device
// array of phi can get the mass without any device allocation by this library or by
// itself.
#include <mutex>

#include "../../include/mpfc.h"
#include "mpfc_internal.h"

namespace {

using mpfc::kMaxPartials;

// Static scratch: kMaxPartials block partial sums, then one slot for the
// last-block-done counter and one for the result.  Every GPU that loads the library
// holds these 8.2 KB until the process exits.
constexpr int kScratchDoubles = kMaxPartials + 2;
constexpr int kThreads = 256;
constexpr long long kCellsPerThread = 16;
constexpr long long kMaxCells = (long long)kMaxPartials * kThreads * kCellsPerThread;   // 2048 x 2048

static __device__ __align__(256) double g_mass_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double block_total(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double x = 0.0;
  if (wid == 0) {
    x = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  }
  __syncthreads();
  return x;   // valid in thread 0
}

// Sums phi over the grid in two deterministic passes: per-block partial sums in
// the scratch, then the last block to finish adds them in block order and writes
// the total into the result slot.
__global__ void k_sum_static(const double* __restrict__ f, long long G, double* scratch) {
  __shared__ double red[32];
  __shared__ bool last;
  double v = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < G; t += (long long)gridDim.x * blockDim.x)
    v += f[t];
  v = block_total(v, red);
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kMaxPartials);
  if (threadIdx.x == 0) {
    scratch[blockIdx.x] = v;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double w = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) w += ((volatile double*)scratch)[b];
  w = block_total(w, red);
  if (threadIdx.x == 0) scratch[kMaxPartials + 1] = w;
}

// Resolves the device address of the static scratch for the current device (once
// per device; the host-side symbol is not a device address).
int scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "cudaGetDevice", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return MPFC_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_mass_scratch);
    if (e != cudaSuccess || !p) {
      mpfc_set_cuda_error(e, "cudaGetSymbolAddress(g_mass_scratch)", __FILE__, __LINE__);
      return MPFC_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return MPFC_OK;
}

}  // namespace

extern "C" int mpfc_mass_noalloc(const double* d_phi, int m, int n, double h, void* cuda_stream, double* out) {
  if (!d_phi || !out || m <= 0 || n <= 0 || !(h > 0)) return MPFC_ERR_INVALID;
  long long G = (long long)m * (long long)n;
  if (G > kMaxCells) return MPFC_ERR_TOO_LARGE;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != MPFC_OK) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the counter must start at zero whatever the previous call left behind
  cudaError_t e = cudaMemsetAsync(scratch + kMaxPartials, 0, sizeof(double), s);
  if (e != cudaSuccess) {
    mpfc_set_cuda_error(e, "cudaMemsetAsync(counter)", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  long long blocks = (G + kThreads - 1) / kThreads;
  if (blocks > kMaxPartials) blocks = kMaxPartials;
  k_sum_static<<<(int)blocks, kThreads, 0, s>>>(d_phi, G, scratch);
  double total = 0.0;
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(&total, scratch + kMaxPartials + 1, sizeof(double), cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    mpfc_set_cuda_error(e, "mass reduction", __FILE__, __LINE__);
    return MPFC_ERR_CUDA;
  }
  *out = h * h * total;
  return MPFC_OK;
}
