// profile.cu -- launch counter and per-class CUDA-event kernel timing.
//
// Timing is off by default.  When enabled, every launch of a class is
// bracketed by two events recorded on the stream it is launched on, so the
// durations are the kernels' own device times inside whatever region the
// caller is measuring.  purl_profile_read synchronises the pending events.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cstdio>
#include <iterator>

#include "profile.cuh"

namespace purl {

namespace {

struct Pending {
  int cls;
  const char *name;
  cudaEvent_t e0, e1;
  double flops, bytes;
};

struct Stats {
  long long launches = 0;
  double ms = 0.0, flops = 0.0, bytes = 0.0;
};

const char *kNames[KC_COUNT] = {"gemm_f64", "panel_qr", "gemm_tc", "split", "other"};

std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_timing{0};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
Stats g_stats[KC_COUNT];
std::map<std::string, Stats> g_named;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void drain_locked() {
  for (const Pending &p : g_pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      for (Stats *s : {&g_stats[p.cls], &g_named[p.name ? p.name : kNames[p.cls]]}) {
        s->launches += 1;
        s->ms += ms;
        s->flops += p.flops;
        s->bytes += p.bytes;
      }
    }
    g_pool.push_back(p.e0);
    g_pool.push_back(p.e1);
  }
  g_pending.clear();
}

}  // namespace

LaunchScope::LaunchScope(int cls, cudaStream_t s, double flops, double bytes, const char *name)
    : cls_(cls), name_(name), s_(s), flops_(flops), bytes_(bytes) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (g_timing.load(std::memory_order_relaxed)) {
    std::lock_guard<std::mutex> lock(g_mu);
    e0_ = take_event();
    e1_ = take_event();
    if (e0_ && e1_) cudaEventRecord(e0_, s_);
  }
}

LaunchScope::~LaunchScope() {
  if (e0_ && e1_) {
    cudaEventRecord(e1_, s_);
    std::lock_guard<std::mutex> lock(g_mu);
    g_pending.push_back({cls_, name_, e0_, e1_, flops_, bytes_});
    if (g_pending.size() > 4096) drain_locked();
  }
}

}  // namespace purl

using namespace purl;

extern "C" {

unsigned long long purl_launch_count(void) { return g_launches.load(); }

void purl_profile_enable(int on) {
  std::lock_guard<std::mutex> lock(g_mu);
  drain_locked();
  g_timing.store(on ? 1 : 0);
}

void purl_profile_reset(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  drain_locked();
  for (auto &s : g_stats) s = Stats{};
  g_named.clear();
}

int purl_profile_read(int cls, long long *launches, double *ms, double *flops, double *bytes) {
  if (cls < 0 || cls >= KC_COUNT) return -1;
  std::lock_guard<std::mutex> lock(g_mu);
  drain_locked();
  const Stats &s = g_stats[cls];
  if (launches) *launches = s.launches;
  if (ms) *ms = s.ms;
  if (flops) *flops = s.flops;
  if (bytes) *bytes = s.bytes;
  return PURL_OK;
}

int purl_profile_read_named(int index, char *name, int name_len, long long *launches, double *ms, double *flops,
                            double *bytes) {
  std::lock_guard<std::mutex> lock(g_mu);
  drain_locked();
  if (index < 0 || index >= (int)g_named.size()) return -1;
  auto it = g_named.begin();
  std::advance(it, index);
  if (name && name_len > 0) {
    std::snprintf(name, (size_t)name_len, "%s", it->first.c_str());
  }
  if (launches) *launches = it->second.launches;
  if (ms) *ms = it->second.ms;
  if (flops) *flops = it->second.flops;
  if (bytes) *bytes = it->second.bytes;
  return PURL_OK;
}

const char *purl_profile_class_name(int cls) {
  return (cls >= 0 && cls < KC_COUNT) ? kNames[cls] : "";
}

}  // extern "C"
