// Primitives: status text, stream-ordered allocation, prefix sums.
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "common.cuh"

namespace sa {

static thread_local char g_last_error[256] = {0};

void set_cuda_error(cudaError_t e, const char* what) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
}

void set_error_text(const char* text) { snprintf(g_last_error, sizeof(g_last_error), "%s", text); }

static unsigned long long g_launches = 0;
void count_launch() { __atomic_fetch_add(&g_launches, 1ull, __ATOMIC_RELAXED); }
// kernels run by graph replays (captured kernels are counted when they run,
// not when they are captured)
void count_launches(long long k) { __atomic_fetch_add(&g_launches, (unsigned long long)k, __ATOMIC_RELAXED); }
long long launch_counter() { return (long long)__atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

// The stream-ordered pool of this process keeps freed memory cached instead
// of returning it to the driver at every synchronisation (a setup allocates
// and frees hundreds of level buffers; a later setup reuses them).  Applies
// to this process's default pool of the current device only.
static void keep_pool_memory() {
  static bool done[64] = {};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  done[dev] = true;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
}

int Alloc::get(void** p, size_t bytes) {
  *p = nullptr;
  if (fn_alloc) {
    *p = fn_alloc(bytes, ctx);
    if (!*p) return SA_ERR_OOM;
    if (reinterpret_cast<uintptr_t>(*p) & 255u) {
      // the block kernels' 32-byte row accesses need aligned buffers
      if (fn_free) fn_free(*p, ctx);
      *p = nullptr;
      set_error_text("allocator callback returned a block not aligned to 256 bytes");
      return SA_ERR_OOM;
    }
  } else {
    keep_pool_memory();
    cudaError_t e = cudaMallocAsync(p, bytes, stream);
    if (e != cudaSuccess) {
      set_cuda_error(e, "cudaMallocAsync");
      cudaGetLastError();
      *p = nullptr;
      return SA_ERR_OOM;
    }
  }
  live_bytes += (int64_t)bytes;
  if (live_bytes > peak_bytes) peak_bytes = live_bytes;
  return SA_OK;
}

void Alloc::put(void* p, size_t bytes) {
  if (!p) return;
  if (fn_free) fn_free(p, ctx);
  else cudaFreeAsync(p, stream);
  live_bytes -= (int64_t)bytes;
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

int copy_d2h(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!bytes) return SA_OK;
  SA_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
  SA_CUDA(cudaStreamSynchronize(s));
  return SA_OK;
}

int copy_h2d(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!bytes) return SA_OK;
  SA_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
  return SA_OK;
}

int memset_d(void* dst, int v, size_t bytes, cudaStream_t s) {
  if (!bytes) return SA_OK;
  SA_CUDA(cudaMemsetAsync(dst, v, bytes, s));
  return SA_OK;
}

// ---------------------------------------------------------------------------
// inclusive scan of int64 in place: tile sums, scan of tile sums, rescan.
// Tile = 1024 threads x 8 consecutive elements.
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024;
constexpr int SCAN_V = 8;
constexpr int64_t SCAN_TILE = SCAN_T * SCAN_V;

__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t* sh, int64_t* total) {
  // v: per-thread value; returns inclusive prefix over the block
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    int64_t s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(FULL, s, o);
      if (lane >= o) s += t;
    }
    sh[lane] = s;
  }
  __syncthreads();
  int64_t r = v + (w > 0 ? sh[w - 1] : 0);
  if (total) *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return r;
}

__global__ void k_tile_sums(const int64_t* __restrict__ a, int64_t n, int64_t* __restrict__ sums) {
  __shared__ int64_t sh[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_V;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_V; ++k)
    if (base + k < n) s += a[base + k];
  int64_t tot;
  block_incl_scan(s, sh, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// single CTA: exclusive scan of the tile sums in place
__global__ void k_scan_sums(int64_t* __restrict__ sums, int64_t nt) {
  __shared__ int64_t sh[32];
  int64_t per = (nt + blockDim.x - 1) / blockDim.x;
  int64_t b0 = (int64_t)threadIdx.x * per;
  int64_t s = 0;
  for (int64_t k = 0; k < per; ++k)
    if (b0 + k < nt) s += sums[b0 + k];
  int64_t incl = block_incl_scan(s, sh, nullptr);
  int64_t run = incl - s;
  for (int64_t k = 0; k < per; ++k)
    if (b0 + k < nt) {
      int64_t t = sums[b0 + k];
      sums[b0 + k] = run;
      run += t;
    }
}

__global__ void k_tile_rescan(int64_t* __restrict__ a, int64_t n, const int64_t* __restrict__ offs) {
  __shared__ int64_t sh[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_V;
  int64_t v[SCAN_V];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_V; ++k) {
    v[k] = (base + k < n) ? a[base + k] : 0;
    s += v[k];
  }
  int64_t incl = block_incl_scan(s, sh, nullptr);
  int64_t run = incl - s + offs[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_V; ++k) {
    run += v[k];
    if (base + k < n) a[base + k] = run;
  }
}

int scan_inplace(Alloc& al, int64_t* a, int64_t n) {
  if (n <= 0) return SA_OK;
  int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  Buf<int64_t> sums;
  SA_TRY(sums.alloc(&al, nt));
  k_tile_sums<<<(unsigned)nt, SCAN_T, 0, al.stream>>>(a, n, sums.p);
  SA_LAUNCHED();
  k_scan_sums<<<1, SCAN_T, 0, al.stream>>>(sums.p, nt);
  SA_LAUNCHED();
  k_tile_rescan<<<(unsigned)nt, SCAN_T, 0, al.stream>>>(a, n, sums.p);
  SA_LAUNCHED();
  return SA_OK;
}

}  // namespace sa

extern "C" const char* sa_last_error(void) { return sa::g_last_error; }

extern "C" int64_t sa_launch_count(void) { return (int64_t)__atomic_load_n(&sa::g_launches, __ATOMIC_RELAXED); }
