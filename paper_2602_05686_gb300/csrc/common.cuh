// Internal helpers shared by the CUDA translation units of the library:
// status handling, the device allocator, launch geometry and warp utilities.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "sa.h"

namespace sa {

// ---------------------------------------------------------------------------
// status handling
// ---------------------------------------------------------------------------
void set_cuda_error(cudaError_t e, const char* what);
void set_error_text(const char* text);

#define SA_CUDA(call)                                   \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) {                            \
      ::sa::set_cuda_error(_e, #call);                  \
      return SA_ERR_CUDA;                               \
    }                                                   \
  } while (0)

#define SA_TRY(call)              \
  do {                            \
    int _s = (call);              \
    if (_s != SA_OK) return _s;   \
  } while (0)

// after every kernel launch: error check + launch count
void count_launch();
void count_launches(long long k);  // k may be negative (kernels captured into a graph, not run)
long long launch_counter();
#define SA_LAUNCHED()        \
  do {                       \
    ::sa::count_launch();    \
    SA_CUDA(cudaGetLastError()); \
  } while (0)

// ---------------------------------------------------------------------------
// device memory: stream-ordered, optionally through a caller allocator
// ---------------------------------------------------------------------------
struct Alloc {
  cudaStream_t stream = nullptr;
  void* (*fn_alloc)(size_t, void*) = nullptr;
  void (*fn_free)(void*, void*) = nullptr;
  void* ctx = nullptr;
  int64_t live_bytes = 0;
  int64_t peak_bytes = 0;

  int get(void** p, size_t bytes);
  void put(void* p, size_t bytes);
};

// typed buffer owned by an Alloc
template <typename T>
struct Buf {
  T* p = nullptr;
  int64_t n = 0;
  Alloc* a = nullptr;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  Buf(Buf&& o) noexcept { p = o.p; n = o.n; a = o.a; o.p = nullptr; o.n = 0; }
  Buf& operator=(Buf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; a = o.a; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~Buf() { release(); }
  int alloc(Alloc* al, int64_t count) {
    release();
    a = al;
    n = count;
    void* q = nullptr;
    int st = al->get(&q, sizeof(T) * (size_t)(count > 0 ? count : 1));
    p = static_cast<T*>(q);
    return st;
  }
  void release() {
    if (p && a) a->put(p, sizeof(T) * (size_t)(n > 0 ? n : 1));
    p = nullptr;
    n = 0;
  }
  size_t bytes() const { return sizeof(T) * (size_t)(n > 0 ? n : 1); }
};

// ---------------------------------------------------------------------------
// launch geometry
// ---------------------------------------------------------------------------
int num_sms();
inline unsigned blocks_for(int64_t threads, int block) {
  int64_t b = (threads + block - 1) / block;
  if (b < 1) b = 1;
  if (b > 0x7fffffffLL) b = 0x7fffffffLL;
  return (unsigned)b;
}
// grid of `block`-thread CTAs that gives one warp per row (grid-stride inside)
inline unsigned warp_rows_grid(int64_t rows, int block = 256) {
  int64_t warps = rows;
  int64_t cap = (int64_t)num_sms() * 32 * (2048 / block);  // a few waves
  if (warps > cap * (block / 32)) warps = cap * (block / 32);
  return blocks_for(warps * 32, block);
}

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int64_t global_warp() {
  return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}
__device__ __forceinline__ int64_t warp_stride() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// primitives (prim.cu)
// ---------------------------------------------------------------------------
// in-place inclusive prefix sum of a[0..n) (int64)
int scan_inplace(Alloc& al, int64_t* a, int64_t n);
// fixed-order reductions: partial sums per CTA of a fixed grid, then one CTA
// sums the partials in index order; deterministic for a given n.
constexpr int RED_BLOCKS = 304;   // 2 x 152 SMs
constexpr int RED_THREADS = 512;
int copy_d2h(void* dst, const void* src, size_t bytes, cudaStream_t s);
int copy_h2d(void* dst, const void* src, size_t bytes, cudaStream_t s);
int memset_d(void* dst, int v, size_t bytes, cudaStream_t s);

}  // namespace sa
