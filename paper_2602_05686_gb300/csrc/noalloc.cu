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
#include "common.cuh"
#include "kernels.cuh"

namespace sa {

constexpr int64_t NOALLOC_SCRATCH_DOUBLES = 2 * 1024 * 1024;  // 16 MiB for w and D
// one extra 256-byte line after the 16 MiB holds the input-check flag
constexpr int64_t NOALLOC_FLAG_DOUBLES = 32;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES + NOALLOC_FLAG_DOUBLES];

namespace {
// device address of the scratch array in the current device's context.  The
// host-side name of the array is not a device address.  Looked up on every
// call (cheap once the module is loaded), so a reset device or a new primary
// context never leaves a stale cached pointer.
int scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) {
    set_cuda_error(e, "cudaGetSymbolAddress(noalloc scratch)");
    cudaGetLastError();
    return SA_ERR_CUDA;
  }
  *out = static_cast<double*>(p);
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
  if (n == 0) return SA_OK;
  cudaStream_t s = (cudaStream_t)stream;
  // The weight kernels index w by row_ptr and gather x / sigma_inv by column,
  // so the CSR is checked before any of them runs: row pointers from 0 to
  // nnz, monotone, columns in [0, n).  The flag lives in the array's last
  // line; the stream is waited on once to read it (no allocation: the host
  // side is a stack int).
  int* flag = reinterpret_cast<int*>(scratch + sa::NOALLOC_SCRATCH_DOUBLES);
  SA_TRY(sa::memset_d(flag, 0, sizeof(int), s));
  SA_TRY(sa::launch_validate_csr(s, n, n, nnz, row_ptr, col, flag));
  int bad = 0;
  SA_CUDA(cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  SA_CUDA(cudaStreamSynchronize(s));
  if (bad) {
    sa::set_error_text("sa_strength_material_noalloc: invalid CSR (row_ptr not 0..nnz and monotone, or a column "
                       "outside [0, n) or not ascending)");
    return SA_ERR_INVALID_ARG;
  }
  // w in [0, nnz), D in [nnz, nnz + n); both are fully written before they
  // are read, so nothing has to be cleared between calls
  return sa::launch_strength_material(s, dim, n, row_ptr, col, coords, sigma_inv, dirichlet, theta, scratch,
                                      scratch + nnz, keep, nullptr);
}
