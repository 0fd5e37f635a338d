// Per-launch CUDA-event timing of solve-phase kernels, aggregated by
// (kernel kind, level).  Events come from a reusable pool; reading the
// profile synchronises on the last recorded event.
#include <map>
#include <mutex>
#include <vector>

#include "profile.cuh"

namespace sa {

namespace {
struct Rec {
  int kind, level;
  double bytes;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
size_t g_used = 0;

cudaEvent_t take() {
  if (g_used == g_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_pool.push_back(e);
  }
  return g_pool[g_used++];
}
}  // namespace

bool prof_on() { return g_on; }

int prof_begin(cudaStream_t s, int kind, int level, double bytes) {
  if (!g_on) return -1;
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r;
  r.kind = kind;
  r.level = level;
  r.bytes = bytes;
  r.a = take();
  r.b = take();
  if (!r.a || !r.b) return -1;
  cudaEventRecord(r.a, s);
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void prof_end(cudaStream_t s, int idx) {
  if (idx < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(g_recs[idx].b, s);
}

}  // namespace sa

extern "C" {

int sa_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(sa::g_mu);
  sa::g_on = on != 0;
  sa::g_recs.clear();
  sa::g_used = 0;
  return SA_OK;
}

int sa_profile_read(int max_rows, int* kind, int* level, int64_t* launches, double* total_ms, double* bytes,
                    int* rows) {
  std::lock_guard<std::mutex> lk(sa::g_mu);
  if (!rows) return SA_ERR_INVALID_ARG;
  std::map<std::pair<int, int>, int> idx;
  std::vector<int64_t> cnt;
  std::vector<double> ms, by;
  std::vector<std::pair<int, int>> keys;
  for (const sa::Rec& r : sa::g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) {
      cudaGetLastError();
      return SA_ERR_CUDA;
    }
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    auto k = std::make_pair(r.kind, r.level);
    auto it = idx.find(k);
    int j;
    if (it == idx.end()) {
      j = (int)keys.size();
      idx[k] = j;
      keys.push_back(k);
      cnt.push_back(0);
      ms.push_back(0);
      by.push_back(0);
    } else {
      j = it->second;
    }
    cnt[j] += 1;
    ms[j] += t;
    by[j] += r.bytes;
  }
  int n = (int)keys.size();
  *rows = n;
  for (int j = 0; j < n && j < max_rows; ++j) {
    if (kind) kind[j] = keys[j].first;
    if (level) level[j] = keys[j].second;
    if (launches) launches[j] = cnt[j];
    if (total_ms) total_ms[j] = ms[j];
    if (bytes) bytes[j] = by[j];
  }
  return SA_OK;
}

}  // extern "C"
