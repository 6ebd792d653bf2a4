// ce_mppi_noalloc.cu -- DBSCAN entry point that allocates no memory.
//
// ce_mppi_dbscan_dev asks its caller for a device workspace.  Some callers
// cannot provide one: a controller whose process forbids device allocations
// after start-up (so that allocator latency or failure can never hit the
// control loop), a host that drives the library from a context where calling
// cudaMalloc is not allowed, or code that owns no allocator of its own.
// ce_mppi_dbscan_noalloc_dev runs the same kernel with its scratch in a
// file-scope __device__ array instead, so it makes no allocation call at all.
#include <cmath>
#include <mutex>

#include "ce_mppi_internal.cuh"

namespace {

// Largest point count the fixed scratch serves.
constexpr int kNoAllocMaxPoints = 16384;
// Bytes of scratch the standalone DBSCAN needs for kNoAllocMaxPoints points
// (same carving as its workspace: cell, sorted, core, 3 coordinates, boxes,
// two angle-bucket tables); each call checks the workspace size against it.
constexpr size_t kNoAllocBytes =
    (size_t)kNoAllocMaxPoints * (3 * sizeof(int) + 3 * sizeof(float)) +
    (size_t)cem::kMaxCells * 6 * sizeof(float) + 2 * sizeof(int) * (size_t)cem::kAngBuckets;

// The scratch: one copy per device that loads the library, kept until exit.
// Its name is only a host-side stand-in in host code; kernels get the device
// address looked up below.
static __device__ __align__(256) unsigned char g_dbscan_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

ce_status_t noalloc_fail(ce_status_t s, const char* msg) {
  cem::set_last_error(msg);   // read back through ce_mppi_last_error()
  return s;
}

}  // namespace

extern "C" {

ce_status_t ce_mppi_dbscan_noalloc_dev(const float* z, int n, int ld, int p, float eps,
                                       int min_pts, int* labels, int* n_clusters,
                                       void* stream) {
  if (p != 2 && p != 3) return noalloc_fail(CE_MPPI_ERR_INVALID_ARG, "p must be 2 or 3");
  if (n < 0 || ld < n || min_pts < 1) return noalloc_fail(CE_MPPI_ERR_INVALID_ARG, "bad sizes");
  if (n > kNoAllocMaxPoints)
    return noalloc_fail(CE_MPPI_ERR_INVALID_ARG,
                        "n exceeds the 16384 points of the fixed scratch (use ce_mppi_dbscan_dev)");
  if (!(eps > 0.02f) || !(eps <= 2.0f))
    return noalloc_fail(CE_MPPI_ERR_INVALID_ARG, "eps must be in (0.02, 2]");
  if (!n_clusters || (n > 0 && (!z || !labels)))
    return noalloc_fail(CE_MPPI_ERR_INVALID_ARG, "NULL pointer");
  // DBSCAN grid as for the allocating entry point: cell side 0.99 eps/sqrt(p).
  const double ci = std::sqrt((double)p) / (0.99 * (double)eps);
  const int G = (int)std::floor(2.0 * ci) + 1;
  const int R = (int)std::ceil((double)eps * ci);
  const int nc = p == 3 ? G * G * G : G * G;
  if (nc > cem::kMaxCells)
    return noalloc_fail(CE_MPPI_ERR_INVALID_ARG, "eps too small for the DBSCAN grid");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(CE_MPPI_ERR_CUDA, "cudaGetDevice failed");
  if (cem::dbscan_ws_bytes(n) > kNoAllocBytes)   // (the carving must fit the array)
    return noalloc_fail(CE_MPPI_ERR_INVALID_ARG, "scratch layout larger than the fixed array");
  // the kernels' shared-memory limits on this device (the library's one
  // configuration guard, shared with every other entry point)
  cem::ensure_configured();
  void* scratch = nullptr;
  {
    // Set-up, once per device, with that device current: the device address
    // of the scratch array.
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_dbscan_scratch);
      if (e != cudaSuccess || !ptr)
        return noalloc_fail(CE_MPPI_ERR_CUDA, "cudaGetSymbolAddress of the DBSCAN scratch failed");
      g_scratch_ptr[dev] = ptr;
    }
    scratch = g_scratch_ptr[dev];
  }
  volatile float ev = eps;
  const float eps2 = ev * ev;
  cem::launch_dbscan_standalone(z, n, ld, p, eps2, (float)ci, G, R, min_pts, labels, n_clusters,
                                scratch, static_cast<cudaStream_t>(stream));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(CE_MPPI_ERR_CUDA, cudaGetErrorString(e));
  return CE_MPPI_OK;
}

}  // extern "C"
