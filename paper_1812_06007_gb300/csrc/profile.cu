// profile.cu -- launch counter and per-class CUDA-event kernel timing.
//
// Timing is off by default.  When enabled, launches are bracketed by two
// events recorded on the stream they are launched on, so the durations are
// the kernels' own device times inside whatever region the caller is
// measuring.  With a sampling stride s > 1, the first launches of every
// kernel name and then every s-th are timed (event records between
// kernels are not free: tens of thousands per second add up), and each
// name's total time is estimated as its timed launches' time scaled by
// launches / timed launches.  purl_profile_read synchronises the pending
// events.
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

// launches seen and launches timed per kernel name (for sampling)
struct Seen {
  long long seen = 0, timed = 0;
  double flops = 0.0, bytes = 0.0;
};

const char *kNames[KC_COUNT] = {"gemm_f64", "panel_qr", "gemm_tc", "split", "other"};

std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_timing{0};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
Stats g_stats[KC_COUNT];
std::map<std::string, Stats> g_named;       // timed launches only
std::map<std::string, Seen> g_seen;         // every launch while timing is on
Seen g_seen_cls[KC_COUNT];
int g_stride = 1;
constexpr long long kAlwaysTimed = 8;       // the first launches of every name are timed

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

// Fold the first `count` pending timings (all by default) into the stats.
// The oldest launches are drained first: they have normally finished, so the
// host does not wait on the GPU (waiting on the newest launch would let the
// GPU's queue run dry in the middle of the region being measured).
void drain_locked(size_t count = (size_t)-1) {
  if (count > g_pending.size()) count = g_pending.size();
  for (size_t i = 0; i < count; ++i) {
    const Pending &p = g_pending[i];
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
  g_pending.erase(g_pending.begin(), g_pending.begin() + (long)count);
}

}  // namespace

LaunchScope::LaunchScope(int cls, cudaStream_t s, double flops, double bytes, const char *name)
    : cls_(cls), name_(name), s_(s), flops_(flops), bytes_(bytes) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (g_timing.load(std::memory_order_relaxed)) {
    std::lock_guard<std::mutex> lock(g_mu);
    Seen &sn = g_seen[name_ ? name_ : kNames[cls_]];
    Seen &sc = g_seen_cls[cls_];
    const long long k = sn.seen++;
    sn.flops += flops_;
    sn.bytes += bytes_;
    sc.seen++;
    sc.flops += flops_;
    sc.bytes += bytes_;
    if (k < kAlwaysTimed || g_stride <= 1 || (k % g_stride) == 0) {
      e0_ = take_event();
      e1_ = take_event();
      if (e0_ && e1_) {
        cudaEventRecord(e0_, s_);
        sn.timed++;
        sc.timed++;
      }
    }
  }
}

LaunchScope::~LaunchScope() {
  if (e0_ && e1_) {
    cudaEventRecord(e1_, s_);
    std::lock_guard<std::mutex> lock(g_mu);
    g_pending.push_back({cls_, name_, e0_, e1_, flops_, bytes_});
    if (g_pending.size() > 8192) drain_locked(4096);
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
  g_seen.clear();
  for (auto &s : g_seen_cls) s = Seen{};
}

void purl_profile_set_stride(int stride) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_stride = stride < 1 ? 1 : stride;
}

// Reported per class / name: every launch made while timing was on, their
// declared flops and bytes, and the device time of the timed launches scaled
// by launches / timed launches.
int purl_profile_read(int cls, long long *launches, double *ms, double *flops, double *bytes) {
  if (cls < 0 || cls >= KC_COUNT) return -1;
  std::lock_guard<std::mutex> lock(g_mu);
  drain_locked();
  const Stats &s = g_stats[cls];
  const Seen &sn = g_seen_cls[cls];
  const double scale = s.launches > 0 ? (double)sn.seen / (double)s.launches : 0.0;
  if (launches) *launches = sn.seen;
  if (ms) *ms = s.ms * scale;
  if (flops) *flops = sn.flops;
  if (bytes) *bytes = sn.bytes;
  return PURL_OK;
}

int purl_profile_read_named(int index, char *name, int name_len, long long *launches, double *ms, double *flops,
                            double *bytes) {
  std::lock_guard<std::mutex> lock(g_mu);
  drain_locked();
  if (index < 0 || index >= (int)g_seen.size()) return -1;
  auto it = g_seen.begin();
  std::advance(it, index);
  if (name && name_len > 0) {
    std::snprintf(name, (size_t)name_len, "%s", it->first.c_str());
  }
  const auto st = g_named.find(it->first);
  const double tms = st != g_named.end() ? st->second.ms : 0.0;
  const long long tl = st != g_named.end() ? st->second.launches : 0;
  if (launches) *launches = it->second.seen;
  if (ms) *ms = tl > 0 ? tms * (double)it->second.seen / (double)tl : 0.0;
  if (flops) *flops = it->second.flops;
  if (bytes) *bytes = it->second.bytes;
  return PURL_OK;
}

const char *purl_profile_class_name(int cls) {
  return (cls >= 0 && cls < KC_COUNT) ? kNames[cls] : "";
}

}  // extern "C"
