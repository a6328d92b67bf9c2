// Kernel profiler: CUDA events around every launch of the library while
// profiling is on, aggregated per kernel name with the launch's algorithmic
// flops and bytes (counted on the host from the descriptors).
#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace hif {

namespace {

struct Pending {
  std::string name;
  cudaEvent_t a, b;
  double flops, bytes;
  int64_t kernels;
};

struct Agg {
  int64_t launches = 0, kernels = 0;
  double seconds = 0, flops = 0, bytes = 0;
};

thread_local bool t_suspended = false;

struct ProfState {
  std::mutex mu;
  bool on = false;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, Agg> agg;
};

ProfState& state() {
  static ProfState s;
  return s;
}

cudaEvent_t get_event(ProfState& s) {
  if (!s.pool.empty()) {
    cudaEvent_t e = s.pool.back();
    s.pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  HIF_CUDA_TRY(cudaEventCreate(&e));
  return e;
}

void drain(ProfState& s) {
  for (auto& p : s.pending) {
    float ms = 0.f;
    HIF_CUDA_TRY(cudaEventSynchronize(p.b));
    HIF_CUDA_TRY(cudaEventElapsedTime(&ms, p.a, p.b));
    Agg& g = s.agg[p.name];
    g.launches++;
    g.kernels += p.kernels;
    g.seconds += ms * 1e-3;
    g.flops += p.flops;
    g.bytes += p.bytes;
    s.pool.push_back(p.a);
    s.pool.push_back(p.b);
  }
  s.pending.clear();
}

}  // namespace

bool prof_enabled() { return state().on; }

void prof_add(const char* name, double flops, double bytes) {
  ProfState& s = state();
  if (!s.on || t_suspended) return;
  std::lock_guard<std::mutex> lk(s.mu);
  Agg& g = s.agg[name];
  g.flops += flops;
  g.bytes += bytes;
}

ProfSuspend::ProfSuspend() : prev_(t_suspended) { t_suspended = true; }
ProfSuspend::~ProfSuspend() { t_suspended = prev_; }

ProfScope::ProfScope(const char* name, cudaStream_t st, double flops, double bytes)
    : st_(st), active_(false) {
  ProfState& s = state();
  if (!s.on || t_suspended) return;
  std::lock_guard<std::mutex> lk(s.mu);
  a_ = get_event(s);
  b_ = get_event(s);
  name_ = name;
  flops_ = flops;
  bytes_ = bytes;
  k0_ = launch_counter();
  HIF_CUDA_TRY(cudaEventRecord(a_, st_));
  active_ = true;
  nvtxRangePushA(name);   // lets a profiler select the launches of one label
}

ProfScope::~ProfScope() {
  if (!active_) return;
  nvtxRangePop();
  ProfState& s = state();
  std::lock_guard<std::mutex> lk(s.mu);
  cudaEventRecord(b_, st_);
  s.pending.push_back(Pending{name_, a_, b_, flops_, bytes_, launch_counter() - k0_});
  if (s.pending.size() > 4096) {
    try {
      drain(s);
    } catch (...) {
    }
  }
}

}  // namespace hif

extern "C" {

hif_status hif_profile_begin(void) {
  try {
    auto& s = hif::state();
    std::lock_guard<std::mutex> lk(s.mu);
    hif::drain(s);
    s.agg.clear();
    s.on = true;
    return HIF_OK;
  } catch (const hif::Error& e) {
    hif::set_last_error(e.msg);
    return e.code;
  }
}

hif_status hif_profile_end(hif_kernel_profile* out, int cap, int* count) {
  try {
    auto& s = hif::state();
    std::lock_guard<std::mutex> lk(s.mu);
    s.on = false;
    hif::drain(s);
    int i = 0;
    for (auto& kv : s.agg) {
      if (out && i < cap) {
        hif_kernel_profile& o = out[i];
        std::memset(&o, 0, sizeof(o));
        std::strncpy(o.name, kv.first.c_str(), sizeof(o.name) - 1);
        o.launches = kv.second.launches;
        o.kernels = kv.second.kernels;
        o.seconds = kv.second.seconds;
        o.flops = kv.second.flops;
        o.bytes = kv.second.bytes;
      }
      ++i;
    }
    if (count) *count = i;
    return HIF_OK;
  } catch (const hif::Error& e) {
    hif::set_last_error(e.msg);
    return e.code;
  }
}

}  // extern "C"
