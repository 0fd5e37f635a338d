// Graph kernels of the setup: filtered graph G_C, distance-2 maximal
// independent set by fixed-priority rounds, aggregation phases, tentative
// prolongator, deterministic transpose.
#include "common.cuh"
#include "kernels.cuh"

namespace sa {

// ---------------------------------------------------------------------------
// a5. filtered graph G_C (Sec. 2.1): kept off-diagonals; the filtered matrix
// row pointer counts one diagonal per row, so gcrp[i] = rpF[i] - i.
// ---------------------------------------------------------------------------
__global__ void k_graph_rowptr(int64_t n, const int64_t* __restrict__ rpF, int64_t* __restrict__ gcrp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n) gcrp[i] = rpF[i] - i;
}

__global__ void k_graph_compact(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const uint8_t* __restrict__ keep, const int64_t* __restrict__ gcrp,
                                int32_t* __restrict__ gcci) {
  const int lane = lane_id();
  for (int64_t i = global_warp(); i < n; i += warp_stride()) {
    const int64_t b = rp[i], e = rp[i + 1];
    int64_t out = gcrp[i];
    for (int64_t p0 = b; p0 < e; p0 += 32) {
      int64_t p = p0 + lane;
      int32_t j = p < e ? ci[p] : -1;
      bool k = p < e && j != (int32_t)i && keep[p];
      unsigned m = __ballot_sync(FULL, k);
      if (k) gcci[out + __popc(m & ((1u << lane) - 1u))] = j;
      out += __popc(m);
    }
  }
}

int launch_graph_rowptr(cudaStream_t s, int64_t n, const int64_t* rpF, int64_t* gcrp) {
  k_graph_rowptr<<<blocks_for(n + 1, 256), 256, 0, s>>>(n, rpF, gcrp);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_graph_compact(cudaStream_t s, int64_t n, const int64_t* rp, const int32_t* ci, const uint8_t* keep,
                         const int64_t* gcrp, int32_t* gcci) {
  if (n <= 0) return SA_OK;
  k_graph_compact<<<warp_rows_grid(n), 256, 0, s>>>(n, rp, ci, keep, gcrp, gcci);
  SA_LAUNCHED();
  return SA_OK;
}

// ---------------------------------------------------------------------------
// a6. distance-2 maximal independent set.  The result equals the greedy
// set that visits nodes in descending key order (key = fmix32 hash of the
// index salted by the level, in the high word; the index in the low word).
// Tags: 0 = removed (or Dirichlet), ~0 = selected, key + 1 = undecided.
// A round takes two neighbour-max sweeps: m1 = max over the closed
// neighbourhood, m2 = max of m1 over the closed neighbourhood; an undecided
// node with m2 == ~0 has a selected node within distance 2 (removed), one
// with m2 == its own tag is the largest undecided key within distance 2
// (selected).  This is the deterministic parallel greedy MIS applied to G^2.
// ---------------------------------------------------------------------------
constexpr uint64_t TAG_SEL = ~0ull;

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  // MurmurHash3 32-bit finaliser (Appleby, public domain)
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__global__ void k_mis_init(int64_t n, const uint8_t* __restrict__ dir, uint32_t salt, uint32_t seed,
                           uint64_t* __restrict__ tag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (dir && dir[i]) { tag[i] = 0; return; }
  uint32_t h = fmix32((uint32_t)i ^ salt ^ seed);
  uint64_t key = ((uint64_t)h << 32) | (uint64_t)(uint32_t)i;
  tag[i] = key + 1;
}

// neighbour maxima with MIS_SW lanes per G_C row (rows hold 0..26 entries),
// over the rows of `list` (NULL: every row)
constexpr int MIS_SW = 8;

__device__ __forceinline__ bool mis_undecided(uint64_t t) { return t != 0 && t != TAG_SEL; }

__global__ void k_mis_max1(int64_t nl, const int32_t* __restrict__ list, const int64_t* __restrict__ gcrp,
                           const int32_t* __restrict__ gcci, const uint64_t* __restrict__ tag,
                           uint64_t* __restrict__ m1) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t t = gt / MIS_SW;
  const int sl = (int)(gt % MIS_SW);
  uint64_t m = 0;
  int64_t i = -1;
  if (t < nl) {
    i = list ? list[t] : t;
    if (sl == 0) m = tag[i];
    for (int64_t p = gcrp[i] + sl; p < gcrp[i + 1]; p += MIS_SW) {
      uint64_t v = tag[gcci[p]];
      m = v > m ? v : m;
    }
  }
  for (int o = MIS_SW / 2; o > 0; o >>= 1) {
    uint64_t v = __shfl_xor_sync(FULL, m, o, MIS_SW);
    m = v > m ? v : m;
  }
  if (t < nl && sl == 0) m1[i] = m;
}

__global__ void k_mis_max2(int64_t nl, const int32_t* __restrict__ list, const int64_t* __restrict__ gcrp,
                           const int32_t* __restrict__ gcci, const uint64_t* __restrict__ m1,
                           uint64_t* __restrict__ tag, unsigned long long* __restrict__ undecided) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t t = gt / MIS_SW;
  const int sl = (int)(gt % MIS_SW);
  const int64_t i = t < nl ? (list ? list[t] : t) : 0;
  const uint64_t ti = t < nl ? tag[i] : 0;
  const bool active = t < nl && mis_undecided(ti);
  uint64_t m = 0;
  if (active) {
    if (sl == 0) m = m1[i];
    for (int64_t p = gcrp[i] + sl; p < gcrp[i + 1]; p += MIS_SW) {
      uint64_t v = m1[gcci[p]];
      m = v > m ? v : m;
    }
  }
  for (int o = MIS_SW / 2; o > 0; o >>= 1) {
    uint64_t v = __shfl_xor_sync(FULL, m, o, MIS_SW);
    m = v > m ? v : m;
  }
  if (active && sl == 0) {
    uint64_t nt = (m == TAG_SEL) ? 0 : (m == ti ? TAG_SEL : ti);
    tag[i] = nt;
    if (mis_undecided(nt)) atomicAdd(undecided, 1ull);
  }
}

// active sets for the later rounds: flag every undecided row of `list` and
// its G_C neighbours (the rows whose m1 a round still reads)
__global__ void k_mis_flag(int64_t nl, const int32_t* __restrict__ list, const int64_t* __restrict__ gcrp,
                           const int32_t* __restrict__ gcci, const uint64_t* __restrict__ tag,
                           uint8_t* __restrict__ flag) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t t = gt / MIS_SW;
  const int sl = (int)(gt % MIS_SW);
  if (t >= nl) return;
  const int64_t i = list ? list[t] : t;
  if (!mis_undecided(tag[i])) return;
  if (sl == 0) flag[i] = 1;
  for (int64_t p = gcrp[i] + sl; p < gcrp[i + 1]; p += MIS_SW) flag[gcci[p]] = 1;
}

// over the rows of the previous neighbourhood list: counts of the new
// undecided list and of the new neighbourhood list (both subsets of it)
__global__ void k_mis_listcount(int64_t nl, const int32_t* __restrict__ list, const uint64_t* __restrict__ tag,
                                const uint8_t* __restrict__ flag, int64_t* __restrict__ cu,
                                int64_t* __restrict__ cn) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nl) return;
  const int64_t i = list ? list[t] : t;
  cu[t + 1] = mis_undecided(tag[i]) ? 1 : 0;
  cn[t + 1] = flag[i] ? 1 : 0;
}

__global__ void k_mis_listfill(int64_t nl, const int32_t* __restrict__ list, const uint64_t* __restrict__ tag,
                               const uint8_t* __restrict__ flag, const int64_t* __restrict__ cu,
                               const int64_t* __restrict__ cn, int32_t* __restrict__ ulist,
                               int32_t* __restrict__ nlist) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nl) return;
  const int32_t i = list ? list[t] : (int32_t)t;
  if (mis_undecided(tag[i])) ulist[cu[t]] = i;
  if (flag[i]) nlist[cn[t]] = i;
}

int run_mis2(Alloc& al, int64_t n, const int64_t* gcrp, const int32_t* gcci, const uint8_t* dir, int level,
             uint32_t seed, uint64_t* tag, int* rounds, int max_rounds) {
  cudaStream_t s = al.stream;
  *rounds = 0;
  if (n <= 0) return SA_OK;
  Buf<uint64_t> m1;
  Buf<unsigned long long> cnt;
  SA_TRY(m1.alloc(&al, n));
  SA_TRY(cnt.alloc(&al, 1));
  const uint32_t salt = 0x9E3779B9u * (uint32_t)(level + 1);
  k_mis_init<<<blocks_for(n, 256), 256, 0, s>>>(n, dir, salt, seed, tag);
  SA_LAUNCHED();
  // Rounds are launched in groups between read-backs of the undecided count;
  // a round after convergence changes nothing (every node is decided).  Once
  // few nodes are undecided, the rounds run over two lists instead of all
  // rows: U, the undecided rows (the only ones max2 changes), and N, U with
  // its G_C neighbours (the only m1 values max2 reads).  Both lists are
  // rebuilt after every group from the previous N (they only shrink), in
  // ascending row order; the rounds decide exactly as over all rows.
  Buf<int32_t> ul, nla, nlb;
  Buf<uint8_t> flag;
  Buf<int64_t> cu, cn;
  const int32_t* U = nullptr;  // NULL: every row
  const int32_t* N = nullptr;
  int64_t nu = n, nn = n;
  unsigned long long h_cnt = 1;
  const int group = 4;
  while (h_cnt > 0) {
    if (*rounds >= max_rounds) return SA_ERR_CAPACITY;
    for (int g = 0; g < group; ++g) {
      SA_TRY(memset_d(cnt.p, 0, sizeof(unsigned long long), s));
      if (nn > 0) {
        k_mis_max1<<<blocks_for(nn * MIS_SW, 256), 256, 0, s>>>(nn, N, gcrp, gcci, tag, m1.p);
        SA_LAUNCHED();
      }
      if (nu > 0) {
        k_mis_max2<<<blocks_for(nu * MIS_SW, 256), 256, 0, s>>>(nu, U, gcrp, gcci, m1.p, tag, cnt.p);
        SA_LAUNCHED();
      }
      ++*rounds;
    }
    SA_TRY(copy_d2h(&h_cnt, cnt.p, sizeof(h_cnt), s));
    if (h_cnt > 0 && (int64_t)h_cnt * 8 < nn) {
      if (!flag.p) {
        SA_TRY(flag.alloc(&al, n));
        SA_TRY(ul.alloc(&al, n));
        SA_TRY(nla.alloc(&al, n));
        SA_TRY(nlb.alloc(&al, n));
        SA_TRY(cu.alloc(&al, n + 1));
        SA_TRY(cn.alloc(&al, n + 1));
      }
      SA_TRY(memset_d(flag.p, 0, flag.bytes(), s));
      k_mis_flag<<<blocks_for(nu * MIS_SW, 256), 256, 0, s>>>(nu, U, gcrp, gcci, tag, flag.p);
      SA_LAUNCHED();
      SA_TRY(memset_d(cu.p, 0, sizeof(int64_t), s));
      SA_TRY(memset_d(cn.p, 0, sizeof(int64_t), s));
      k_mis_listcount<<<blocks_for(nn, 256), 256, 0, s>>>(nn, N, tag, flag.p, cu.p, cn.p);
      SA_LAUNCHED();
      SA_TRY(scan_inplace(al, cu.p + 1, nn));
      SA_TRY(scan_inplace(al, cn.p + 1, nn));
      int32_t* nnew = (N == nla.p) ? nlb.p : nla.p;
      k_mis_listfill<<<blocks_for(nn, 256), 256, 0, s>>>(nn, N, tag, flag.p, cu.p, cn.p, ul.p, nnew);
      SA_LAUNCHED();
      int64_t tot[2] = {0, 0};
      SA_TRY(copy_d2h(&tot[0], cu.p + nn, sizeof(int64_t), s));
      SA_TRY(copy_d2h(&tot[1], cn.p + nn, sizeof(int64_t), s));
      U = ul.p;
      N = nnew;
      nu = tot[0];
      nn = tot[1];
    }
  }
  return SA_OK;
}

// ---------------------------------------------------------------------------
// a7. aggregation (Sec. 2): ids of roots by ascending index (scan of root
// flags); phase 1: root and its G_C neighbours; phase 2: a leftover node joins
// the phase-1 aggregate with the most G_C edges to it, ties to the smallest
// id.  err bit 8: a non-Dirichlet node left without an aggregate.
// ---------------------------------------------------------------------------
__global__ void k_root_count(int64_t n, const uint64_t* __restrict__ tag, int64_t* __restrict__ cnt,
                             uint8_t* __restrict__ root) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool r = tag[i] == TAG_SEL;
  cnt[i + 1] = r ? 1 : 0;
  if (root) root[i] = r ? 1 : 0;
}

__global__ void k_agg_phase1(int64_t n, const int64_t* __restrict__ gcrp, const int32_t* __restrict__ gcci,
                             const uint64_t* __restrict__ tag, const int64_t* __restrict__ rpref,
                             int32_t* __restrict__ p1) {
  const int lane = lane_id();
  for (int64_t i = global_warp(); i < n; i += warp_stride()) {
    if (tag[i] == TAG_SEL) {
      if (lane == 0) p1[i] = (int32_t)rpref[i];
      continue;
    }
    int32_t a = -1;
    for (int64_t p0 = gcrp[i]; p0 < gcrp[i + 1]; p0 += 32) {
      int64_t p = p0 + lane;
      bool r = false;
      int32_t j = 0;
      if (p < gcrp[i + 1]) { j = gcci[p]; r = tag[j] == TAG_SEL; }
      unsigned m = __ballot_sync(FULL, r);
      if (m && a < 0) {
        int32_t jr = __shfl_sync(FULL, j, __ffs(m) - 1);
        a = (int32_t)rpref[jr];
      }
    }
    if (lane == 0) p1[i] = a;
  }
}

__global__ void k_agg_phase2(int64_t n, const int64_t* __restrict__ gcrp, const int32_t* __restrict__ gcci,
                             const uint8_t* __restrict__ dir, const int32_t* __restrict__ p1,
                             int32_t* __restrict__ agg, int* __restrict__ err) {
  const int lane = lane_id();
  for (int64_t i = global_warp(); i < n; i += warp_stride()) {
    const int32_t mine = p1[i];
    if (mine >= 0 || (dir && dir[i])) {
      if (lane == 0) agg[i] = mine;
      continue;
    }
    const int64_t b = gcrp[i], e = gcrp[i + 1];
    // best = max edge count, then min id: maximise (count << 32) | ~id
    unsigned long long best = 0;
    for (int64_t p = b + lane; p < e; p += 32) {
      int32_t a = p1[gcci[p]];
      if (a < 0) continue;
      unsigned c = 0;
      for (int64_t q = b; q < e; ++q) c += (p1[gcci[q]] == a);
      unsigned long long key = ((unsigned long long)c << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)a);
      best = key > best ? key : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long t = __shfl_xor_sync(FULL, best, o);
      best = t > best ? t : best;
    }
    if (lane == 0) {
      int32_t a = best ? (int32_t)(0xFFFFFFFFu - (uint32_t)(best & 0xFFFFFFFFull)) : -1;
      agg[i] = a;
      if (a < 0) atomicOr(err, 8);
    }
  }
}

int run_aggregate(Alloc& al, int64_t n, const int64_t* gcrp, const int32_t* gcci, const uint8_t* dir,
                  const uint64_t* tag, int32_t* agg, uint8_t* root, int64_t* nc, int* err) {
  cudaStream_t s = al.stream;
  *nc = 0;
  if (n <= 0) return SA_OK;
  Buf<int64_t> pref;
  Buf<int32_t> p1;
  SA_TRY(pref.alloc(&al, n + 1));
  SA_TRY(p1.alloc(&al, n));
  SA_TRY(memset_d(pref.p, 0, sizeof(int64_t), s));
  k_root_count<<<blocks_for(n, 256), 256, 0, s>>>(n, tag, pref.p, root);
  SA_LAUNCHED();
  SA_TRY(scan_inplace(al, pref.p + 1, n));
  k_agg_phase1<<<warp_rows_grid(n), 256, 0, s>>>(n, gcrp, gcci, tag, pref.p, p1.p);
  SA_LAUNCHED();
  k_agg_phase2<<<warp_rows_grid(n), 256, 0, s>>>(n, gcrp, gcci, dir, p1.p, agg, err);
  SA_LAUNCHED();
  SA_TRY(copy_d2h(nc, pref.p + n, sizeof(int64_t), s));
  return SA_OK;
}

// ---------------------------------------------------------------------------
// a8. tentative prolongator (Sec. 2): one 1.0 per aggregated row
// ---------------------------------------------------------------------------
__global__ void k_tentative_count(int64_t n, const int32_t* __restrict__ agg, int64_t* __restrict__ cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cnt[i + 1] = agg[i] >= 0 ? 1 : 0;
}

__global__ void k_tentative_fill(int64_t n, const int32_t* __restrict__ agg, const int64_t* __restrict__ rp,
                                 int32_t* __restrict__ ci, double* __restrict__ v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) {
    ci[rp[i]] = agg[i];
    v[rp[i]] = 1.0;
  }
}

int launch_tentative_count(cudaStream_t s, int64_t n, const int32_t* agg, int64_t* cnt) {
  if (n <= 0) return SA_OK;
  k_tentative_count<<<blocks_for(n, 256), 256, 0, s>>>(n, agg, cnt);
  SA_LAUNCHED();
  return SA_OK;
}

int launch_tentative(cudaStream_t s, int64_t n, const int32_t* agg, const int64_t* rp, int32_t* ci, double* v) {
  if (n <= 0) return SA_OK;
  k_tentative_fill<<<blocks_for(n, 256), 256, 0, s>>>(n, agg, rp, ci, v);
  SA_LAUNCHED();
  return SA_OK;
}

// ---------------------------------------------------------------------------
// deterministic transpose: column counts, scan, unordered scatter, then each
// row of the result is placed in ascending source-row order by rank
// ---------------------------------------------------------------------------
__global__ void k_col_count(int64_t nnz, const int32_t* __restrict__ ci, int64_t* __restrict__ cnt) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnz) atomicAdd((unsigned long long*)&cnt[ci[p] + 1], 1ull);
}

__global__ void k_scatter_t(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, const int64_t* __restrict__ off,
                            int* __restrict__ cursor, int32_t* __restrict__ tci, double* __restrict__ tv) {
  const int lane = lane_id();
  for (int64_t i = global_warp(); i < n; i += warp_stride()) {
    for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
      int32_t j = ci[p];
      int64_t pos = off[j] + atomicAdd(&cursor[j], 1);
      tci[pos] = (int32_t)i;
      if (tv) tv[pos] = v[p];
    }
  }
}

__global__ void k_rank_sort_rows(int64_t m, const int64_t* __restrict__ rp, const int32_t* __restrict__ tci,
                                 const double* __restrict__ tv, int32_t* __restrict__ oci,
                                 double* __restrict__ ov) {
  const int lane = lane_id();
  for (int64_t r = global_warp(); r < m; r += warp_stride()) {
    const int64_t b = rp[r], e = rp[r + 1];
    for (int64_t p = b + lane; p < e; p += 32) {
      int32_t key = tci[p];
      int64_t rank = 0;
      for (int64_t q = b; q < e; ++q) rank += (tci[q] < key);
      oci[b + rank] = key;
      if (ov) ov[b + rank] = tv[p];
    }
  }
}

int run_transpose(Alloc& al, int64_t n, int64_t m, const int64_t* rp, const int32_t* ci, const double* v,
                  Buf<int64_t>& Rrp, Buf<int32_t>& Rci, Buf<double>* Rv) {
  cudaStream_t s = al.stream;
  int64_t nnz = 0;
  SA_TRY(copy_d2h(&nnz, rp + n, sizeof(int64_t), s));
  SA_TRY(Rrp.alloc(&al, m + 1));
  SA_TRY(Rci.alloc(&al, nnz));
  if (Rv) SA_TRY(Rv->alloc(&al, nnz));
  SA_TRY(memset_d(Rrp.p, 0, Rrp.bytes(), s));
  if (nnz > 0) {
    k_col_count<<<blocks_for(nnz, 256), 256, 0, s>>>(nnz, ci, Rrp.p);
    SA_LAUNCHED();
  }
  SA_TRY(scan_inplace(al, Rrp.p + 1, m));
  if (nnz == 0) return SA_OK;
  Buf<int> cursor;
  Buf<int32_t> tci;
  Buf<double> tv;
  SA_TRY(cursor.alloc(&al, m));
  SA_TRY(tci.alloc(&al, nnz));
  if (Rv) SA_TRY(tv.alloc(&al, nnz));
  SA_TRY(memset_d(cursor.p, 0, cursor.bytes(), s));
  k_scatter_t<<<warp_rows_grid(n), 256, 0, s>>>(n, rp, ci, v, Rrp.p, cursor.p, tci.p, Rv ? tv.p : nullptr);
  SA_LAUNCHED();
  k_rank_sort_rows<<<warp_rows_grid(m), 256, 0, s>>>(m, Rrp.p, tci.p, Rv ? tv.p : nullptr, Rci.p,
                                                      Rv ? Rv->p : nullptr);
  SA_LAUNCHED();
  return SA_OK;
}

}  // namespace sa
