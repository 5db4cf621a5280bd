// Per-kernel timing with CUDA events recorded on the launching stream (off by default), and a
// process-wide count of the kernels this library launches.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <utility>
#include <vector>

namespace cola {

struct Profiler {
  bool on = false;
  struct Rec {
    const char* name;
    cudaEvent_t start, stop;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  ~Profiler() {
    for (auto& r : recs) {
      cudaEventDestroy(r.start);
      cudaEventDestroy(r.stop);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

extern std::atomic<unsigned long long> g_launches;
extern thread_local Profiler* t_profiler;

// Wraps one kernel launch: counts it and, when the calling plan profiles, brackets it with events.
class LaunchScope {
 public:
  LaunchScope(const char* name, cudaStream_t st) : st_(st) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    Profiler* p = t_profiler;
    if (p && p->on) {
      rec_.name = name;
      rec_.start = p->get();
      rec_.stop = p->get();
      if (rec_.start && rec_.stop) {
        cudaEventRecord(rec_.start, st_);
        active_ = true;
      }
    }
  }
  ~LaunchScope() {
    if (active_) {
      cudaEventRecord(rec_.stop, st_);
      t_profiler->recs.push_back(rec_);
    }
  }

 private:
  cudaStream_t st_;
  Profiler::Rec rec_{};
  bool active_ = false;
};

// Sets the profiler of the plan used by the current API call.  A call made inside another call
// that is profiling (an ensemble running its boxes' plans) records into that outer profiler.
struct ProfilerGuard {
  explicit ProfilerGuard(Profiler* p) : prev_(t_profiler) {
    if (!(prev_ && prev_->on)) t_profiler = p;
  }
  ~ProfilerGuard() { t_profiler = prev_; }
  Profiler* prev_;
};

}  // namespace cola
