// Per-kernel timing with CUDA events recorded on the launching stream (off by default).
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pttk_internal.cuh"

namespace pttk {
namespace {

struct Pending {
  cudaEvent_t a, b;
};
struct Entry {
  std::vector<Pending> pending;
  double ms = 0.0;
  int64_t launches = 0;
};

std::mutex g_mu;
std::map<std::string, Entry> g_entries;
std::vector<cudaEvent_t> g_pool;
bool g_on = false;

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

pttk_status drain(Entry& en) {
  for (auto& p : en.pending) {
    cudaError_t err = cudaEventSynchronize(p.b);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, p.a, p.b);
    if (err != cudaSuccess) return cuda_error(err, "profile event");
    en.ms += ms;
    en.launches += 1;
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  en.pending.clear();
  return PTTK_OK;
}

}  // namespace

bool prof_on() { return g_on; }

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void* prof_begin(const char* name, cudaStream_t s) {
  if (!g_on) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  Entry& en = g_entries[name];
  Pending p{take_event(), take_event()};
  cudaEventRecord(p.a, s);
  en.pending.push_back(p);
  return &en.pending.back();
}

void prof_end(const char* name, cudaStream_t s) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Entry& en = g_entries[name];
  if (!en.pending.empty()) cudaEventRecord(en.pending.back().b, s);
}

}  // namespace pttk

using namespace pttk;

extern "C" {

pttk_status pttk_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  return PTTK_OK;
}

pttk_status pttk_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& kv : g_entries) {
    pttk_status s = drain(kv.second);
    if (s != PTTK_OK) return s;
    kv.second.ms = 0.0;
    kv.second.launches = 0;
  }
  return PTTK_OK;
}

pttk_status pttk_profile_get(const char* name, double* ms_total, int64_t* launches) {
  if (!name || !ms_total || !launches) return set_error(PTTK_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_entries.find(name);
  if (it == g_entries.end()) {
    *ms_total = 0.0;
    *launches = 0;
    return PTTK_OK;
  }
  PTTK_TRY(drain(it->second));
  *ms_total = it->second.ms;
  *launches = it->second.launches;
  return PTTK_OK;
}

int64_t pttk_launch_count(void) { return (int64_t)g_launches.load(); }

// Names of the kernels seen so far, separated by '\n', into buf (truncated to len).
pttk_status pttk_profile_names(char* buf, int64_t len) {
  if (!buf || len < 1) return set_error(PTTK_EINVAL, "bad buffer");
  std::lock_guard<std::mutex> lk(g_mu);
  std::string all;
  for (auto& kv : g_entries) all += kv.first + "\n";
  const size_t n = std::min<size_t>(all.size(), (size_t)len - 1);
  memcpy(buf, all.data(), n);
  buf[n] = 0;
  return PTTK_OK;
}

}  // extern "C"
