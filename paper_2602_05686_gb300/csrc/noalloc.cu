// A variant of the material-aware strength filter (the same kernels as
// sa_strength with SA_MEASURE_MATERIAL) whose scratch memory is a fixed
// file-scope device array, so that a call allocates no memory at all.
//
// Who needs it: callers that cannot allocate device memory at the point of
// the call, e.g. code running under a memory-pool or allocator policy that
// forbids new allocations, a host callback or real-time loop where an
// allocation could block or fail, or an embedding application that owns all
// device memory and hands this library only its inputs and outputs.
//
// The scratch holds the edge weights w (one double per stored entry) and the
// row sums D (one double per row).  Every GPU that loads this library keeps
// the array for the lifetime of the process.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace sa {

constexpr int64_t NOALLOC_SCRATCH_DOUBLES = 2 * 1024 * 1024;  // 16 MiB

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_ptr[MAX_DEVICES] = {nullptr};

// device address of the scratch array on the current device, looked up once
// per device (the host-side name of the array is not a device address)
int scratch_address(double** out) {
  int dev = 0;
  SA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return SA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      set_cuda_error(e, "cudaGetSymbolAddress(noalloc scratch)");
      cudaGetLastError();
      return SA_ERR_CUDA;
    }
    g_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_ptr[dev];
  return SA_OK;
}
}  // namespace

}  // namespace sa

extern "C" int sa_strength_material_noalloc(int dim, int64_t n, int64_t nnz, const int64_t* row_ptr,
                                            const int32_t* col, const double* coords, const double* sigma_inv,
                                            const uint8_t* dirichlet, double theta, uint8_t* keep, void* stream) {
  if (n < 0 || nnz < 0 || !row_ptr || !col || !coords || !sigma_inv || !keep || (dim != 2 && dim != 3))
    return SA_ERR_INVALID_ARG;
  if (nnz + n > sa::NOALLOC_SCRATCH_DOUBLES) {
    sa::set_error_text("sa_strength_material_noalloc: nnz + n exceeds the 2097152-double (16 MiB) static scratch");
    return SA_ERR_CAPACITY;
  }
  double* scratch = nullptr;
  int st = sa::scratch_address(&scratch);
  if (st != SA_OK) return st;
  // w in [0, nnz), D in [nnz, nnz + n); both are fully written before they
  // are read, so nothing has to be cleared between calls
  return sa::launch_strength_material((cudaStream_t)stream, dim, n, row_ptr, col, coords, sigma_inv, dirichlet, theta,
                                      scratch, scratch + nnz, keep, nullptr);
}
