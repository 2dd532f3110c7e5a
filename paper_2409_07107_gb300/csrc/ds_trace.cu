// Stage tracing: CUDA events around every kernel the library launches, on the launching stream.
#include <mutex>
#include <vector>

#include "ds_common.cuh"

namespace {
struct Mark {
  int stage;
  cudaEvent_t begin, end;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Mark> g_marks;      // bracketed launches since the last read
std::vector<cudaEvent_t> g_pool;
struct Open {
  int stage;
  cudaStream_t stream;
  cudaEvent_t begin;
};
std::vector<Open> g_open;         // begun, not yet ended (per stage and stream: models may overlap)

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void ds_trace_mark(int stage, int begin, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_on || stage < 0 || stage >= DS_NSTAGES) return;
  cudaEvent_t e = take_event();
  if (!e) return;
  cudaEventRecord(e, s);
  if (begin) {
    g_open.push_back({stage, s, e});
    return;
  }
  for (size_t i = 0; i < g_open.size(); ++i)
    if (g_open[i].stage == stage && g_open[i].stream == s) {
      g_marks.push_back({stage, g_open[i].begin, e});
      g_open.erase(g_open.begin() + i);
      return;
    }
  g_pool.push_back(e);
}

extern "C" ds_status ds_profile(int32_t enable) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_on = enable != 0;
  return DS_OK;
}

extern "C" ds_status ds_profile_read(double* ms, int32_t* launches) {
  if (!ms || !launches) return DS_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  for (int k = 0; k < DS_NSTAGES; ++k) { ms[k] = 0.0; launches[k] = 0; }
  ds_status st = DS_OK;
  for (const Mark& m : g_marks) {
    float t = 0.f;
    if (cudaEventSynchronize(m.end) != cudaSuccess || cudaEventElapsedTime(&t, m.begin, m.end) != cudaSuccess)
      st = DS_ECUDA;
    ms[m.stage] += t;
    launches[m.stage] += 1;
    g_pool.push_back(m.begin);
    g_pool.push_back(m.end);
  }
  g_marks.clear();
  return st;
}
