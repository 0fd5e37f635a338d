// Several right-hand sides at once (K = 2, 4 or 8 columns, interleaved
// storage: element (i, c) of an n x K block at i*K + c).  Every stored entry
// of every V-cycle matrix and of the outer FP64 operator is read once per
// launch and applied to all K columns; the K values a row needs from a
// gathered x_j are one aligned vector load.  Each column is accumulated in
// the one-vector order (entry order, same lane split, same shuffle tree) and
// goes through the same row update, so a column equals the one-vector kernel
// bitwise.
#include "common.cuh"
#include "profile.cuh"
#include "solve.cuh"
#include "vcycle.cuh"
#include "vkern.cuh"

namespace sa {

// One row of an interleaved block (its K values, K * sizeof(T) contiguous
// bytes, aligned to that size) moves as whole vectors: 32-byte accesses
// (sm_100 and later) where the row fills one or two of them, else the widest
// that fits.  Element-wise accesses at the 32-byte row stride make every warp
// instruction touch eight 128-byte lines for 128 useful bytes and leave the
// stores as partial-sector writes; measured on the 8-column FP32 Chebyshev
// step at 320^3 that cost 1.6x in time.  Buffers start on 256-byte
// boundaries (the allocator contract).
//   ld_row_nc: data read-only for the whole launch (gathered x, b)
//   ld_row:    coherent load (a vector the launch also writes, as d)
template <typename T, int K>
__device__ __forceinline__ void ld_row_nc(const T* __restrict__ p, T (&v)[K]) {
  if constexpr (sizeof(T) == 4 && K == 8) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
  } else if constexpr (sizeof(T) == 8 && K % 4 == 0) {
#pragma unroll
    for (int q = 0; q < K / 4; ++q)
      asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
          : "=d"(v[4 * q]), "=d"(v[4 * q + 1]), "=d"(v[4 * q + 2]), "=d"(v[4 * q + 3])
          : "l"(p + 4 * q));
  } else if constexpr (sizeof(T) == 4 && K == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (sizeof(T) == 4 && K == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x; v[1] = t.y;
  } else if constexpr (sizeof(T) == 8 && K == 2) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x; v[1] = t.y;
  } else {
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = __ldg(p + c);
  }
}

template <typename T, int K>
__device__ __forceinline__ void ld_row(const T* p, T (&v)[K]) {
  if constexpr (sizeof(T) == 4 && K == 8) {
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p)
                 : "memory");
  } else if constexpr (sizeof(T) == 8 && K % 4 == 0) {
#pragma unroll
    for (int q = 0; q < K / 4; ++q)
      asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
                   : "=d"(v[4 * q]), "=d"(v[4 * q + 1]), "=d"(v[4 * q + 2]), "=d"(v[4 * q + 3])
                   : "l"(p + 4 * q)
                   : "memory");
  } else if constexpr (sizeof(T) == 4 && K == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (sizeof(T) == 4 && K == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  } else if constexpr (sizeof(T) == 8 && K == 2) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x; v[1] = t.y;
  } else {
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = p[c];
  }
}

template <typename T, int K>
__device__ __forceinline__ void st_row(T* p, const T (&v)[K]) {
  if constexpr (sizeof(T) == 4 && K == 8) {
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
  } else if constexpr (sizeof(T) == 8 && K % 4 == 0) {
#pragma unroll
    for (int q = 0; q < K / 4; ++q)
      asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p + 4 * q), "d"(v[4 * q]), "d"(v[4 * q + 1]),
                   "d"(v[4 * q + 2]), "d"(v[4 * q + 3])
                   : "memory");
  } else if constexpr (sizeof(T) == 4 && K == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (sizeof(T) == 4 && K == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else if constexpr (sizeof(T) == 8 && K == 2) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  } else {
#pragma unroll
    for (int c = 0; c < K; ++c) p[c] = v[c];
  }
}

// the K values of one gathered row: one 256-bit load for eight FP32
// columns; 128-bit pairs for FP64 (their kernels are FP64-issue bound, and
// a 256-bit load's four results held at once cost the CSR kernels
// registers and occupancy)
template <typename T, int K>
__device__ __forceinline__ void ldvec(const T* __restrict__ p, T (&v)[K]) {
  if constexpr (sizeof(T) == 8 && K % 2 == 0) {
#pragma unroll
    for (int q = 0; q < K / 2; ++q) {
      const double2 t = __ldg(reinterpret_cast<const double2*>(p) + q);
      v[2 * q] = t.x; v[2 * q + 1] = t.y;
    }
  } else {
    ld_row_nc<T, K>(p, v);
  }
}

// Reduction of the K per-lane partial sums over the W lanes of one row.  The
// one-vector kernels add a row's lane sums by the butterfly xor W/2, ..., 1;
// here every exchange also halves the columns a lane carries (a lane keeps
// the lower or upper half and receives its partner's values of that half),
// so each column is added in exactly the butterfly's tree -- bitwise the
// one-vector sum -- with K/2 + K/4 + ... additions per lane instead of
// K log2(W).  On return the lane holds the sums of columns c0 .. c0+V-1 in
// acc[0 .. V); V = K/W when K >= W, else 1 (then lanes whose low bits
// (lane mod W/K) are not zero hold copies).
template <typename T, int K, int W>
__device__ __forceinline__ int lane_reduce(T (&acc)[K], int lane, int& c0) {
  int V = K;
  c0 = 0;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    if (V > 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int j = 0; j < K / 2; ++j) {
        if (j < V / 2) {
          const T send = up ? acc[j] : acc[j + V / 2];
          const T keep = up ? acc[j + V / 2] : acc[j];
          acc[j] = keep + __shfl_xor_sync(FULL, send, o, W);
        }
      }
      if (up) c0 += V / 2;
      V /= 2;
    } else {
      acc[0] += __shfl_xor_sync(FULL, acc[0], o, W);
    }
  }
  return V;
}

// the row product of this thread's row for K interleaved columns; returns the
// number of columns this thread writes (0: none), their sums in acc[0 .. nw)
// being columns c0 .. c0+nw-1 of `row`.  Entries are loaded U at a time
// (values and columns first, then the gathers) and added in entry order, so
// every column's sum is the one-vector kernel's.
// entries per load round: one on SELL rows of one lane (measured: more
// registers cost the level-0 FP32 step more occupancy than the extra loads in
// flight gain), two on CSR lanes and two-lane SELL rows
// FP32 one-lane SELL levels with slices at most STAGE_WCAP entries wide take
// the staged form (SW code SW_STAGED): each warp owns one slice and copies its
// values and columns into shared memory with two bulk copies (cp.async.bulk,
// the TMA engine) completing on a per-warp mbarrier, then gathers with
// STAGE_UG loads in flight.  Measured against the same kernel reading the
// stream directly (27-point SELL-32 at 320^3, eight columns): 2.20 against
// 2.33-2.40 ms.  FP64 never takes it (its kernels are FP64-issue bound).
constexpr int SW_STAGED = -8;
constexpr int STAGE_WPB = 4;     // warps (slices) per block
constexpr int STAGE_WCAP = 32;   // widest slice staged
constexpr int STAGE_UG = 8;      // gathers in flight per thread
template <typename T>
constexpr int staged_code() { return sizeof(T) == 4 ? SW_STAGED : 0; }

// set when a staged kernel's wait for its bulk copies ran out (the kernel
// then writes nothing); read and cleared by block_stage_status
__device__ int g_stage_err = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t cnt) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(cnt) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// bounded wait for the barrier's phase `parity`: false when it ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <typename T, int SW>
struct BUnroll {
  static constexpr int U = SW == 0 ? 1 : 2;
};

template <typename T, int SW, int K>
__device__ __forceinline__ int brow_apply(const MatView<T>& M, const T* __restrict__ X, T (&acc)[K], int64_t& row,
                                          int& c0) {
  constexpr int U = BUnroll<T, SW>::U;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int c = 0; c < K; ++c) acc[c] = (T)0;
  c0 = 0;
  if constexpr (SW == -2) {
    // two lanes per SELL row: even and odd entries
    const int64_t sl = gt >> 6;
    const int r = (int)((gt & 63) >> 1), h = (int)(gt & 1);
    const int64_t i = sl * 32 + r;
    row = i;
    if (i < M.n) {
      const int64_t e = M.p[sl + 1];
      const T* __restrict__ xs = M.c16 ? X + (int64_t)M.base[sl] * K : X;
      int64_t p = M.p[sl] + 32 * h + r;
      for (; p + 64 * (U - 1) < e; p += 64 * U) {
        T a[U], xv[U][K];
        int64_t cc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          a[u] = __ldcs(&M.v[p + 64 * u]);
          cc[u] = M.c16 ? (int64_t)__ldcs(&M.c16[p + 64 * u]) : (int64_t)__ldcs(&M.ci[p + 64 * u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) ldvec<T, K>(xs + cc[u] * K, xv[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int j = 0; j < K; ++j) acc[j] += a[u] * xv[u][j];
      }
      for (; p < e; p += 64) {
        T xv[K];
        const T a = __ldcs(&M.v[p]);
        const int64_t c = M.c16 ? (int64_t)__ldcs(&M.c16[p]) : (int64_t)__ldcs(&M.ci[p]);
        ldvec<T, K>(xs + c * K, xv);
#pragma unroll
        for (int j = 0; j < K; ++j) acc[j] += a * xv[j];
      }
    }
    const int v = lane_reduce<T, K, 2>(acc, h, c0);
    return i < M.n ? v : 0;
  } else if constexpr (SW == SW_STAGED) {
    // one slice per warp, its values and columns staged in shared memory
    extern __shared__ __align__(128) unsigned char stage_smem[];
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    const int64_t sl = (int64_t)blockIdx.x * STAGE_WPB + warp;
    row = sl * 32 + lane;
    if (sl >= ((M.n + 31) >> 5)) return 0;  // warp-uniform
    const int64_t p0 = M.p[sl];
    const int w = (int)((M.p[sl + 1] - p0) >> 5);
    const uint32_t ib = M.c16 ? 2u : 4u;
    T* sv = reinterpret_cast<T*>(stage_smem + 128 + (size_t)warp * STAGE_WCAP * 32 * 8);
    unsigned char* scol = reinterpret_cast<unsigned char*>(sv + STAGE_WCAP * 32);
    const uint32_t ba = smem_u32(reinterpret_cast<uint64_t*>(stage_smem) + warp);
    if (w > 0) {
      if (lane == 0) {
        mbar_init(ba, 1);
        fence_mbar_init();
      }
      __syncwarp();
      if (lane == 0) {
        // p0 is a multiple of 32 entries: both sources 64-byte aligned, both
        // sizes (128 w and 32 w ib bytes) multiples of 16
        mbar_expect_tx(ba, (uint32_t)w * 32u * (4u + ib));
        bulk_g2s(smem_u32(sv), M.v + p0, (uint32_t)w * 128u, ba);
        bulk_g2s(smem_u32(scol), M.c16 ? (const void*)(M.c16 + p0) : (const void*)(M.ci + p0),
                 (uint32_t)w * 32u * ib, ba);
      }
      if (!mbar_wait(ba, 0)) {
        atomicExch(&g_stage_err, 1);
        mbar_wait(ba, 0);  // the copies in flight, again bounded
        return 0;
      }
    }
    if (row >= M.n) return 0;
    const T* __restrict__ xs = M.c16 ? X + (int64_t)M.base[sl] * K : X;
    const uint16_t* s16 = reinterpret_cast<const uint16_t*>(scol);
    const int32_t* s32 = reinterpret_cast<const int32_t*>(scol);
    int k = 0;
    for (; k + STAGE_UG <= w; k += STAGE_UG) {
      T a[STAGE_UG], xv[STAGE_UG][K];
      int64_t cc[STAGE_UG];
#pragma unroll
      for (int u = 0; u < STAGE_UG; ++u) {
        const int q = (k + u) * 32 + lane;
        a[u] = sv[q];
        cc[u] = ib == 2 ? (int64_t)s16[q] : (int64_t)s32[q];
      }
#pragma unroll
      for (int u = 0; u < STAGE_UG; ++u) ldvec<T, K>(xs + cc[u] * K, xv[u]);
#pragma unroll
      for (int u = 0; u < STAGE_UG; ++u)
#pragma unroll
        for (int j = 0; j < K; ++j) acc[j] += a[u] * xv[u][j];
    }
    for (; k < w; ++k) {
      T xv[K];
      const int q = k * 32 + lane;
      const T a = sv[q];
      const int64_t c = ib == 2 ? (int64_t)s16[q] : (int64_t)s32[q];
      ldvec<T, K>(xs + c * K, xv);
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] += a * xv[j];
    }
    return K;
  } else if constexpr (SW == 0) {
    row = gt;
    if (gt >= M.n) return 0;
    const int64_t sl = gt >> 5, r = gt & 31;
    const int64_t b = M.p[sl], e = M.p[sl + 1];
    const T* __restrict__ xs = M.c16 ? X + (int64_t)M.base[sl] * K : X;
    int64_t p = b + r;
    for (; p + 32 * (U - 1) < e; p += 32 * U) {
      T a[U], xv[U][K];
      int64_t cc[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        a[u] = __ldcs(&M.v[p + 32 * u]);
        cc[u] = M.c16 ? (int64_t)__ldcs(&M.c16[p + 32 * u]) : (int64_t)__ldcs(&M.ci[p + 32 * u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) ldvec<T, K>(xs + cc[u] * K, xv[u]);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < K; ++c) acc[c] += a[u] * xv[u][c];
    }
    for (; p < e; p += 32) {
      T xv[K];
      const T a = __ldcs(&M.v[p]);
      const int64_t c = M.c16 ? (int64_t)__ldcs(&M.c16[p]) : (int64_t)__ldcs(&M.ci[p]);
      ldvec<T, K>(xs + c * K, xv);
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] += a * xv[j];
    }
    return K;
  } else {
    if (blockIdx.x < M.nlb) {
      // the long-row bin: one row per warp (warp-uniform), lane-strided
      // sums and the 32-lane tree of the one-vector kernel (one entry per
      // load round for FP64: the K accumulators and gathered values of a
      // second would cost the CSR kernels their occupancy)
      constexpr int U = sizeof(T) == 8 ? 1 : BUnroll<T, SW>::U;
      const int64_t w = gt >> 5;
      if (w >= M.nlong) return 0;
      const int lane = (int)(threadIdx.x & 31);
      const int64_t i = M.lrows[w];
      row = i;
      const int64_t e = M.p[i + 1];
      int64_t q = M.p[i] + lane;
      for (; q + 32 * (U - 1) < e; q += 32 * U) {
        T a[U], xv[U][K];
        int64_t cc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          a[u] = M.v[q + 32 * u];
          cc[u] = M.ci[q + 32 * u];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) ldvec<T, K>(X + cc[u] * K, xv[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int c = 0; c < K; ++c) acc[c] += a[u] * xv[u][c];
      }
      for (; q < e; q += 32) {
        T xv[K];
        const T a = M.v[q];
        ldvec<T, K>(X + (int64_t)M.ci[q] * K, xv);
#pragma unroll
        for (int c = 0; c < K; ++c) acc[c] += a * xv[c];
      }
      const int v = lane_reduce<T, K, 32>(acc, lane, c0);
      constexpr int copies = K >= 32 ? 1 : 32 / K;   // lanes holding the same columns
      return (lane & (copies - 1)) == 0 ? v : 0;
    }
    if constexpr (SW == 1) {
      // rows of one-thread CSR matrices (the prolongators, at most
      // SHORT_ROW_MEAN entries per row on average): one thread per row, the
      // entries in rounds of four loaded together (the last one predicated),
      // each entry's K products added in entry order -- the one-vector
      // kernel's sum -- with the row's K values of a gathered x_j as one
      // 256-bit load (FP32) or 128-bit pairs (FP64).  Measured on a
      // prolongator-shaped operator (4 entries per row, 320^3 -> 120^3),
      // FP32: 0.79 ms against 1.67 ms for four lanes per row with the
      // exchanging butterfly and 3.5 ms for a thread per column; FP64: with
      // one partial sum per column a thread per column pays K-fold loads and
      // the predicated rounds in FP64 issue slots.
      // FP64: thread t takes row perm[t], the rows grouped by length, so that
      // a warp's rounds end together -- its FP64 products issue per warp
      // instruction, and in natural order a warp ran to the longest of its 32
      // rows (about twice its products at 3.8 entries per row; level-0
      // prolongation at 96^3: 125 -> 94 us).  FP32 rows are bound by memory
      // and keep the natural order (the scattered rows cost 26 -> 30 us).
      const int64_t t = (int64_t)(blockIdx.x - M.nlb) * blockDim.x + threadIdx.x;
      row = t;
      if (t >= M.n) return 0;
      int64_t i = t;
      if constexpr (sizeof(T) == 8) {
        if (M.perm) i = M.perm[t];
      }
      row = i;
      const int64_t b = M.p[i], e = M.p[i + 1];
      if (e - b > M.lt) return 0;  // in the long-row bin
      constexpr int R = 4;
      for (int64_t q = b; q < e; q += R) {
        T a[R];
        int32_t cc[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
          const bool in = q + t < e;
          a[t] = in ? M.v[q + t] : (T)0;
          cc[t] = in ? M.ci[q + t] : 0;
        }
#pragma unroll
        for (int t = 0; t < R; ++t) {
          if (q + t < e) {
            T xv[K];
            ldvec<T, K>(X + (int64_t)cc[t] * K, xv);
#pragma unroll
            for (int j = 0; j < K; ++j) acc[j] += a[t] * xv[j];
          }
        }
      }
      c0 = 0;
      return K;
    } else if constexpr (sizeof(T) == 8) {
      // regular rows: K threads per row, thread c taking column c of every
      // entry (the K values of a gathered row of X are contiguous, so the
      // row's threads read them together).  The one-vector kernel's SW lanes
      // are kept as SW partial sums per thread -- entry q goes to partial
      // (q - b) mod SW, in entry order -- and added in its butterfly order,
      // so the column's sum is bitwise the one-vector sum.
      const int64_t g = (int64_t)(blockIdx.x - M.nlb) * blockDim.x + threadIdx.x;
      const int64_t i = g / K;
      const int c = (int)(g % K);
      row = i;
      if (i >= M.n) return 0;
      const int64_t b = M.p[i], e = M.p[i + 1];
      if (e - b > M.lt) return 0;  // in the long-row bin
      // rounds of R = SW * UC consecutive entries (SW on CSR lanes, four on
      // one-thread rows), the last one predicated so that a short row's
      // loads go out together: entry q + t of a round goes to partial t mod SW
      // (q - b is a multiple of SW), each partial adding in entry order.
      // Measured against rounds of 2 SW with a one-entry tail (prolongator
      // rows of 4.5 entries: 1.46x faster; rows of 59 and 75 entries: equal);
      // rounds of two on one-thread rows measured no faster than four.
      constexpr int UC = SW == 1 ? 4 : 1;
      constexpr int R = SW * UC;
      T part[SW];
#pragma unroll
      for (int h = 0; h < SW; ++h) part[h] = (T)0;
      for (int64_t q = b; q < e; q += R) {
        T a[R], xv[R];
        int32_t cc[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
          const bool in = q + t < e;
          a[t] = in ? M.v[q + t] : (T)0;
          cc[t] = in ? M.ci[q + t] : 0;
        }
#pragma unroll
        for (int t = 0; t < R; ++t) xv[t] = q + t < e ? __ldg(&X[(int64_t)cc[t] * K + c]) : (T)0;
#pragma unroll
        for (int u = 0; u < UC; ++u)
#pragma unroll
          for (int h = 0; h < SW; ++h)
            if (q + u * SW + h < e) part[h] += a[u * SW + h] * xv[u * SW + h];
      }
      // the butterfly of the SW lanes: offsets SW/2, ..., 1, lower lane first
#pragma unroll
      for (int o = SW / 2; o > 0; o >>= 1)
#pragma unroll
        for (int h = 0; h < o; ++h) part[h] = part[h] + part[h + o];
      acc[0] = part[0];
      c0 = c;
      return 1;
    } else {
      // FP32 (bandwidth bound, not FP64-issue bound): SW lanes per row as in
      // the one-vector kernel, the K column sums reduced by lane_reduce
      const int64_t g = (int64_t)(blockIdx.x - M.nlb) * blockDim.x + threadIdx.x;
      const int64_t i = g / SW;
      const int sl = (int)(g % SW);
      row = i;
      bool own = false;
      if (i < M.n) {
        const int64_t b = M.p[i], e = M.p[i + 1];
        if (e - b <= M.lt) {
          own = true;
          int64_t q = b + sl;
          for (; q + SW * (U - 1) < e; q += SW * U) {
            T a[U], xv[U][K];
            int64_t cc[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              a[u] = M.v[q + SW * u];
              cc[u] = M.ci[q + SW * u];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) ldvec<T, K>(X + cc[u] * K, xv[u]);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
              for (int cc2 = 0; cc2 < K; ++cc2) acc[cc2] += a[u] * xv[u][cc2];
          }
          for (; q < e; q += SW) {
            T xv[K];
            const T a = M.v[q];
            ldvec<T, K>(X + (int64_t)M.ci[q] * K, xv);
#pragma unroll
            for (int cc2 = 0; cc2 < K; ++cc2) acc[cc2] += a * xv[cc2];
          }
        }
      }
      if constexpr (SW == 1) {
        return own ? K : 0;
      } else {
        const int v = lane_reduce<T, K, SW>(acc, sl, c0);
        constexpr int copies = K >= SW ? 1 : SW / K;
        return own && (sl & (copies - 1)) == 0 ? v : 0;
      }
    }
  }
}

// columns a thread of the regular rows writes (when it writes any): the
// whole row on SELL rows of one lane and FP32 CSR rows of one thread, half
// on two-lane SELL rows, K / lanes on FP32 CSR lanes, one on FP64 CSR (a
// thread per column).  The epilogues move these as one vector where it is
// more than one column; the long-row bin (one column per lane) and FP64 CSR
// keep element stores (the branch would cost those kernels registers).
template <typename T, int SW, int K>
struct BCols {
  static constexpr int V =
      (SW == 0 || SW == SW_STAGED || SW == 1) ? K : SW == -2 ? K / 2 : (sizeof(T) == 8 ? 1 : (K >= SW ? K / SW : 1));
};

// resident blocks per SM asked of the compiler: FP32 rows are latency bound
// and gain from occupancy (6 blocks: 40 registers); the FP64 CSR-lane rows
// (a thread per column) too, but their long-row bin holds eight accumulators
// and an entry's gathered values, which spill below 48 registers (5 blocks;
// measured within 1 % of 6 on the regular rows); FP64 SELL rows and FP64
// one-thread CSR rows (a thread per row) keep them in 64 registers (4 blocks)
template <typename T, int SW>
struct BOcc {
  static constexpr int B = sizeof(T) == 4 ? (SW == SW_STAGED ? 2 : 6) : (SW > 1 ? 5 : 4);
};

template <typename T, int SW, int K>
// d_in and d_out may be one buffer (each thread reads and writes its own row);
// d_in may also be x_in's buffer (after the first step, where x_1 = d_1)
__global__ void __launch_bounds__(256, BOcc<T, SW>::B) k_bvc_cheb(MatView<T> A, const T* __restrict__ b, const T* __restrict__ xin, T* __restrict__ xout,
                           const T* din, T* dout, T c1, T c2, int first) {
  T y[K];
  int64_t i;
  int c0;
  const int nw = brow_apply<T, SW, K>(A, xin, y, i, c0);
  const int64_t o = i * K + c0;
  constexpr int NW = BCols<T, SW, K>::V;
  if constexpr (NW > 1) {
    if (nw == NW) {
      T bb[NW], xx[NW], dd[NW], xo[NW];
      ld_row_nc<T, NW>(b + o, bb);
      ld_row_nc<T, NW>(xin + o, xx);
      if (first) {
#pragma unroll
        for (int j = 0; j < NW; ++j) dd[j] = (T)0;
      } else {
        ld_row<T, NW>(din + o, dd);
      }
#pragma unroll
      for (int j = 0; j < NW; ++j) {
        dd[j] = cheb_dir<T>(bb[j], y[j], dd[j], c1, c2, first);
        xo[j] = xx[j] + dd[j];
      }
      st_row<T, NW>(dout + o, dd);
      st_row<T, NW>(xout + o, xo);
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (j < nw) {
      const T dn = cheb_dir<T>(b[o + j], y[j], first ? (T)0 : din[o + j], c1, c2, first);
      dout[o + j] = dn;
      xout[o + j] = xin[o + j] + dn;
    }
  }
}

template <typename T, int SW, int K>
__global__ void __launch_bounds__(256, BOcc<T, SW>::B) k_bvc_residual(MatView<T> A, const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ r) {
  T y[K];
  int64_t i;
  int c0;
  const int nw = brow_apply<T, SW, K>(A, x, y, i, c0);
  const int64_t o = i * K + c0;
  constexpr int NW = BCols<T, SW, K>::V;
  if constexpr (NW > 1) {
    if (nw == NW) {
      T bb[NW];
      ld_row_nc<T, NW>(b + o, bb);
#pragma unroll
      for (int j = 0; j < NW; ++j) bb[j] = bb[j] - y[j];
      st_row<T, NW>(r + o, bb);
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < K; ++j)
    if (j < nw) r[o + j] = b[o + j] - y[j];
}

template <typename T, int SW, int K>
__global__ void __launch_bounds__(256, BOcc<T, SW>::B) k_bvc_spmv(MatView<T> A, const T* __restrict__ x, T* __restrict__ out) {
  T y[K];
  int64_t i;
  int c0;
  const int nw = brow_apply<T, SW, K>(A, x, y, i, c0);
  const int64_t o = i * K + c0;
  constexpr int NW = BCols<T, SW, K>::V;
  if constexpr (NW > 1) {
    if (nw == NW) {
      T t[NW];
#pragma unroll
      for (int j = 0; j < NW; ++j) t[j] = y[j];
      st_row<T, NW>(out + o, t);
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < K; ++j)
    if (j < nw) out[o + j] = y[j];
}

template <typename T, int SW, int K>
__global__ void __launch_bounds__(256, BOcc<T, SW>::B) k_bvc_spmv_add(MatView<T> A, const T* __restrict__ x, T* __restrict__ out) {
  T y[K];
  int64_t i;
  int c0;
  const int nw = brow_apply<T, SW, K>(A, x, y, i, c0);
  const int64_t o = i * K + c0;
  constexpr int NW = BCols<T, SW, K>::V;
  if constexpr (NW > 1) {
    if (nw == NW) {
      T t[NW];
      ld_row<T, NW>(out + o, t);
#pragma unroll
      for (int j = 0; j < NW; ++j) t[j] += y[j];
      st_row<T, NW>(out + o, t);
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < K; ++j)
    if (j < nw) out[o + j] += y[j];
}

template <typename T, int SW, int K>
__global__ void __launch_bounds__(256, BOcc<T, SW>::B) k_bvc_cheb_out(MatView<T> A, const T* __restrict__ b, const T* __restrict__ xin,
                               const T* __restrict__ d, T c1, T c2, int first, const double* __restrict__ s,
                               double* __restrict__ z) {
  T y[K];
  int64_t i;
  int c0;
  const int nw = brow_apply<T, SW, K>(A, xin, y, i, c0);
  if (nw == 0) return;
  const int64_t o = i * K + c0;
  const double si = s[i];
  constexpr int NW = BCols<T, SW, K>::V;
  if constexpr (NW > 1) {
    if (nw == NW) {
      T bb[NW], xx[NW], dd[NW];
      double zz[NW];
      ld_row_nc<T, NW>(b + o, bb);
      ld_row_nc<T, NW>(xin + o, xx);
      if (first) {
#pragma unroll
        for (int j = 0; j < NW; ++j) dd[j] = (T)0;
      } else {
        ld_row_nc<T, NW>(d + o, dd);
      }
#pragma unroll
      for (int j = 0; j < NW; ++j) zz[j] = si * (double)(xx[j] + cheb_dir<T>(bb[j], y[j], dd[j], c1, c2, first));
      st_row<double, NW>(z + o, zz);
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (j < nw) {
      const T dn = cheb_dir<T>(b[o + j], y[j], first ? (T)0 : d[o + j], c1, c2, first);
      z[o + j] = si * (double)(xin[o + j] + dn);
    }
  }
}

// elementwise forms over the n*K elements
// (the first step's iterate x_1 equals its direction d_1: only d is written)
template <typename T>
__global__ void k_bvc_fine_in(int64_t n, int K, const double* __restrict__ r, const double* __restrict__ s, T c2,
                              T* __restrict__ b, T* __restrict__ d) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n * K) {
    const T bi = (T)(s[e / K] * r[e]);
    b[e] = bi;
    d[e] = c2 * bi;
  }
}

template <typename T>
__global__ void k_bvc_first(int64_t nk, const T* __restrict__ b, T c2, T* __restrict__ d) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nk) d[e] = c2 * b[e];
}

template <typename T>
__global__ void k_bcoarse_in(int64_t n, int K, const T* __restrict__ b, const double* __restrict__ sq,
                             double* __restrict__ t) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n * K) t[e] = sq[e / K] * (double)b[e];
}

template <typename T>
__global__ void k_bcoarse_out(int64_t n, int K, const double* __restrict__ x, const double* __restrict__ sq,
                              T* __restrict__ xo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n * K) xo[e] = (T)(sq[e / K] * x[e]);
}

// launch `Kern<T, sw, K>` over the rows of M
#define BMAT_SW(Kern, KK, M, st, ...)                                                    \
  do {                                                                                   \
    const MatView<T> _mv = view(M);                                                      \
    const unsigned _g = bmat_grid(M, KK);                                                \
    if (staged_form(M))                                                                  \
      Kern<T, staged_code<T>(), KK><<<stage_grid(M), STAGE_WPB * 32, stage_smem_bytes(), st>>>(_mv, __VA_ARGS__); \
    else if ((M).sw == 0 && (M).sell_lanes == 2) Kern<T, -2, KK><<<_g, 256, 0, st>>>(_mv, __VA_ARGS__); \
    else if ((M).sw == 0) Kern<T, 0, KK><<<_g, 256, 0, st>>>(_mv, __VA_ARGS__);          \
    else if ((M).sw == 1) Kern<T, 1, KK><<<_g, 256, 0, st>>>(_mv, __VA_ARGS__);          \
    else Kern<T, CSR_LANES, KK><<<_g, 256, 0, st>>>(_mv, __VA_ARGS__);                   \
  } while (0)

#define LAUNCH_BMAT(Kern, M, st, K, ...)                                                 \
  do {                                                                                   \
    if ((K) == 2) BMAT_SW(Kern, 2, M, st, __VA_ARGS__);                                  \
    else if ((K) == 4) BMAT_SW(Kern, 4, M, st, __VA_ARGS__);                             \
    else BMAT_SW(Kern, 8, M, st, __VA_ARGS__);                                           \
    SA_LAUNCHED();                                                                       \
  } while (0)

template <typename T>
static int block_alloc(Alloc& al, VHier<T>* m) {
  if (m->kready) return SA_OK;
  const int nl = (int)m->lev.size();
  for (int l = 0; l < nl; ++l) {
    VLevel<T>* L = m->lev[l];
    const int64_t nk = L->n * KMAX_BLOCK;
    SA_TRY(L->kb.alloc(&al, nk));
    SA_TRY(L->kx.alloc(&al, nk));
    if (l + 1 < nl) {
      SA_TRY(L->kx2.alloc(&al, nk));
      SA_TRY(L->kr.alloc(&al, nk));
      SA_TRY(L->kd.alloc(&al, nk));
    }
  }
  const int64_t nL = m->lev[nl - 1]->n;
  SA_TRY(m->kct.alloc(&al, nL * KMAX_BLOCK));
  SA_TRY(m->kcs.alloc(&al, nL * KMAX_BLOCK));
  SA_TRY(m->kcy.alloc(&al, nL * KMAX_BLOCK));
  SA_TRY(m->kcx.alloc(&al, nL * KMAX_BLOCK));
  SA_TRY(m->kz.alloc(&al, m->lev[0]->n * KMAX_BLOCK));
  m->kready = 1;
  return SA_OK;
}

// blocks of a K-column launch: SELL and FP32 CSR as the one-vector launch;
// FP64 CSR: the long-row bin's blocks, then K threads per regular row
// the staged form: FP32 one-lane SELL with slices at most STAGE_WCAP wide
template <typename T>
static bool staged_form(const Mat<T>& M) {
  return sizeof(T) == 4 && M.sw == 0 && M.sell_lanes == 1 && M.n > 0 && M.wmax <= STAGE_WCAP;
}
template <typename T>
static unsigned stage_grid(const Mat<T>& M) {
  return blocks_for((M.n + 31) / 32, STAGE_WPB);
}
static size_t stage_smem_bytes() { return 128 + (size_t)STAGE_WPB * STAGE_WCAP * 32 * 8; }

int block_stage_status(cudaStream_t st) {
  int h = 0;
  SA_CUDA(cudaMemcpyFromSymbolAsync(&h, g_stage_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
  SA_CUDA(cudaStreamSynchronize(st));
  if (!h) return SA_OK;
  const int z = 0;
  SA_CUDA(cudaMemcpyToSymbolAsync(g_stage_err, &z, sizeof(int), 0, cudaMemcpyHostToDevice, st));
  set_error_text("a staged SELL kernel's bounded wait for its bulk copies ran out");
  return SA_ERR_CUDA;
}

template <typename T>
static unsigned bmat_grid(const Mat<T>& M, int K) {
  if (M.sw == 0 || M.sw == 1 || sizeof(T) == 4) return mat_grid(M);
  return blocks_for(M.n * (int64_t)K, 256) + (M.nlong > 0 ? long_blocks(M.nlong) : 0u);
}

// one profiled launch (CUDA events around it when profiling is on)
#define BPROF(kind, level, bytes, launch)               \
  do {                                                  \
    int _pi = prof_begin(st, (kind), (level), (bytes)); \
    launch;                                             \
    prof_end(st, _pi);                                  \
  } while (0)

// the cycle of mv() (vcycle.cu) on K columns.  Algorithmic bytes of a
// K-column launch: the matrix once, each vector element K times.
template <typename T>
static int mv_block(VHier<T>* m, cudaStream_t st, int l, int K, const double* r64, T** xo) {
  constexpr bool F64 = sizeof(T) == 8;
  const int K_CHEB = F64 ? PK_B_CHEB64 : PK_B_CHEB32, K_RES = F64 ? PK_B_RESID64 : PK_B_RESID32;
  const int K_RST = F64 ? PK_B_RESTRICT64 : PK_B_RESTRICT32, K_PRL = F64 ? PK_B_PROLONG64 : PK_B_PROLONG32;
  const int K_FST = F64 ? PK_B_FIRST64 : PK_B_FIRST32;
  const double S = sizeof(T);
  VLevel<T>* L = m->lev[l];
  const int nl = (int)m->lev.size();
  const int64_t n = L->n, nk = n * K;
  if (l == nl - 1) {
    int pi = prof_begin(st, PK_B_COARSE, l, 8.0 * n * n + 48.0 * n * K);
    k_bcoarse_in<T><<<g256(nk), 256, 0, st>>>(n, K, L->kb.p, L->sq.p, m->kct.p);
    SA_LAUNCHED();
    SA_TRY(launch_coarse_solve_block(st, m->cf, K, m->kct.p, m->kcs.p, m->kcy.p, m->kcx.p));
    k_bcoarse_out<T><<<g256(nk), 256, 0, st>>>(n, K, m->kcx.p, L->sq.p, L->kx.p);
    prof_end(st, pi);
    SA_LAUNCHED();
    *xo = L->kx.p;
    return SA_OK;
  }
  const int deg = m->deg;
  const double th = 0.5 * (L->lmax + L->lmin), de = 0.5 * (L->lmax - L->lmin);
  const double s1 = th / de;
  const Mat<T>& A = L->A;
  // the first step writes b and d_1 = x_1 into kd; the next step reads both
  // from there and writes d into kx2 and x into kx (then in place / ping-pong)
  if (l == 0) {
    BPROF(K_FST, l, 8.0 * K * n + 8.0 * n + 2.0 * S * K * n,
          (k_bvc_fine_in<T><<<g256(nk), 256, 0, st>>>(n, K, r64, m->s0.p, (T)(1.0 / th), L->kb.p, L->kd.p)));
  } else {
    BPROF(K_FST, l, 2.0 * S * K * n, (k_bvc_first<T><<<g256(nk), 256, 0, st>>>(nk, L->kb.p, (T)(1.0 / th), L->kd.p)));
  }
  SA_LAUNCHED();
  T* x = L->kd.p;  // the iterate
  T* d = L->kd.p;  // the direction
  const double b_chebK = b_mat(A) + 5.0 * S * K * n;
  double rho = 1.0 / s1;
  for (int q = 1; q < deg; ++q) {
    double rn = 1.0 / (2.0 * s1 - rho);
    T* xn = q == 1 ? L->kx.p : (x == L->kx.p ? L->kd.p : L->kx.p);
    T* dn = q == 1 ? L->kx2.p : d;
    BPROF(K_CHEB, l, q == 1 ? b_chebK - S * K * n : b_chebK,
          LAUNCH_BMAT(k_bvc_cheb, A, st, K, L->kb.p, x, xn, d, dn, (T)(rn * rho), (T)(2.0 * rn / de), 0));
    x = xn;
    d = dn;
    rho = rn;
  }
  // post-smoothing buffers: the direction and the other iterate, both not x
  T* post[2];
  {
    int k2 = 0;
    T* cand[3] = {L->kx2.p, L->kd.p, L->kx.p};
    for (int c = 0; c < 3 && k2 < 2; ++c)
      if (cand[c] != x) post[k2++] = cand[c];
  }
  T* xa = x;
  T* xb = post[1];
  T* dp = post[0];
  VLevel<T>* C = m->lev[l + 1];
  BPROF(K_RES, l, b_mat(A) + 3.0 * S * K * n, LAUNCH_BMAT(k_bvc_residual, A, st, K, L->kb.p, xa, L->kr.p));
  BPROF(K_RST, l, b_mat(L->R) + S * K * (n + C->n), LAUNCH_BMAT(k_bvc_spmv, L->R, st, K, L->kr.p, C->kb.p));
  T* xc = nullptr;
  SA_TRY(mv_block(m, st, l + 1, K, nullptr, &xc));
  BPROF(K_PRL, l, b_mat(L->P) + S * K * (C->n + 2.0 * n), LAUNCH_BMAT(k_bvc_spmv_add, L->P, st, K, xc, xa));
  rho = 1.0 / s1;
  for (int q = 0; q < deg; ++q) {
    int first = (q == 0);
    T c1 = (T)0, c2 = (T)(1.0 / th);
    double rn = rho;
    if (!first) {
      rn = 1.0 / (2.0 * s1 - rho);
      c1 = (T)(rn * rho);
      c2 = (T)(2.0 * rn / de);
    }
    if (l == 0 && q == deg - 1) {
      // the last step reads b, x, d and the scaling, and writes the FP64
      // output block in place of x and d
      BPROF(K_CHEB, l, b_mat(A) + 3.0 * S * K * n + 8.0 * K * n + 8.0 * n,
            LAUNCH_BMAT(k_bvc_cheb_out, A, st, K, L->kb.p, xa, dp, c1, c2, first, m->s0.p, m->kz.p));
    } else {
      BPROF(K_CHEB, l, b_chebK, LAUNCH_BMAT(k_bvc_cheb, A, st, K, L->kb.p, xa, xb, dp, dp, c1, c2, first));
      T* t = xa; xa = xb; xb = t;
    }
    if (!first) rho = rn;
  }
  *xo = xa;
  return SA_OK;
}

template <typename T>
int vh_vcycle_block(Alloc& al, VHier<T>* m, cudaStream_t st, int K, const double* R, double** Z) {
  if (K != 2 && K != 4 && K != 8) return SA_ERR_INVALID_ARG;
  SA_TRY(block_alloc(al, m));
  if (m->lev.size() == 1) {
    const int64_t n = m->lev[0]->n;
    SA_TRY(launch_coarse_solve_block(st, m->cf, K, R, m->kcs.p, m->kcy.p, m->kz.p));
    *Z = m->kz.p;
    return SA_OK;
  }
  T* xo = nullptr;
  SA_TRY(mv_block<T>(m, st, 0, K, R, &xo));
  *Z = m->kz.p;
  return SA_OK;
}

template int vh_vcycle_block<double>(Alloc&, VHier<double>*, cudaStream_t, int, const double*, double**);
template int vh_vcycle_block<float>(Alloc&, VHier<float>*, cudaStream_t, int, const double*, double**);

// ---------------------------------------------------------------------------
// outer CG on K columns: Q = A P with the per-column partial p.q sums (the
// one-vector reduction tree per column) and R = B - A X, FP64 SELL
// ---------------------------------------------------------------------------
template <int K>
__global__ void k_bsell_spmv_dot(MatView<double> A, const double* __restrict__ P, double* __restrict__ Q,
                                 double* __restrict__ part) {
  double y[K], c[K];
  int64_t i;
  int c0;
#pragma unroll
  for (int j = 0; j < K; ++j) c[j] = 0.0;
  if (brow_apply<double, 0, K>(A, P, y, i, c0)) {
    const int64_t o = i * K;
    double pp[K];
    ld_row_nc<double, K>(P + o, pp);
    st_row<double, K>(Q + o, y);
#pragma unroll
    for (int j = 0; j < K; ++j) c[j] = y[j] * pp[j];
  }
  __shared__ double sh[K][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // the warp sums of the K columns by the exchanging butterfly (each
  // column's tree is warp_sum's); lane c * (32 / K) ends with column c
  {
    int cc;
    const int v = lane_reduce<double, K, 32>(c, lane, cc);
    constexpr int copies = K >= 32 ? 1 : 32 / K;
    if ((lane & (copies - 1)) == 0)
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j < v) sh[cc + j][w] = c[j];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      double t = lane < (int)(blockDim.x >> 5) ? sh[j][lane] : 0.0;
      t = warp_sum(t);
      if (lane == 0) part[(int64_t)j * gridDim.x + blockIdx.x] = t;
    }
  }
}

template <int K>
__global__ void k_bsell_res64(MatView<double> A, const double* __restrict__ B, const double* __restrict__ X,
                              double* __restrict__ R) {
  double y[K];
  int64_t i;
  int c0;
  if (!brow_apply<double, 0, K>(A, X, y, i, c0)) return;
  const int64_t o = i * K;
  double bb[K];
  ld_row_nc<double, K>(B + o, bb);
#pragma unroll
  for (int j = 0; j < K; ++j) bb[j] = bb[j] - y[j];
  st_row<double, K>(R + o, bb);
}

static MatView<double> sell_view(const Sell<double>& A) {
  MatView<double> m;
  m.n = A.n;
  m.p = A.sp.p;
  m.ci = A.ci.p;
  m.v = A.v.p;
  m.base = A.idx16 ? A.base.p : nullptr;
  m.c16 = A.idx16 ? A.c16.p : nullptr;
  m.lrows = nullptr;
  m.nlong = 0;
  m.lt = INT64_MAX;
  m.nlb = 0;
  m.perm = nullptr;
  return m;
}

int launch_bsell_spmv_dot(cudaStream_t st, const Sell<double>& A, int K, const double* P, double* Q, double* part,
                          int* nparts) {
  *nparts = (int)g256(A.n);
  const MatView<double> mv = sell_view(A);
  // the matrix once; P read and Q written for each of the K columns
  const double bytes = (8.0 + A.idx_bytes()) * A.nnz + 8.0 * (A.nslices + 1) + (A.idx16 ? 4.0 * A.nslices : 0.0) +
                       16.0 * K * A.n;
  if (K != 2 && K != 4 && K != 8) return SA_ERR_INVALID_ARG;
  const int pi = prof_begin(st, PK_B_CG_SPMV, 0, bytes);
  if (K == 2) k_bsell_spmv_dot<2><<<g256(A.n), 256, 0, st>>>(mv, P, Q, part);
  else if (K == 4) k_bsell_spmv_dot<4><<<g256(A.n), 256, 0, st>>>(mv, P, Q, part);
  else k_bsell_spmv_dot<8><<<g256(A.n), 256, 0, st>>>(mv, P, Q, part);
  prof_end(st, pi);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_bsell_residual64(cudaStream_t st, const Sell<double>& A, int K, const double* B, const double* X,
                            double* R) {
  const MatView<double> mv = sell_view(A);
  if (K == 2) k_bsell_res64<2><<<g256(A.n), 256, 0, st>>>(mv, B, X, R);
  else if (K == 4) k_bsell_res64<4><<<g256(A.n), 256, 0, st>>>(mv, B, X, R);
  else if (K == 8) k_bsell_res64<8><<<g256(A.n), 256, 0, st>>>(mv, B, X, R);
  else return SA_ERR_INVALID_ARG;
  SA_LAUNCHED();
  return SA_OK;
}

}  // namespace sa
