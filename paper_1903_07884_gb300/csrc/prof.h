// Optional per-kernel timing: while enabled, each instrumented launch is
// bracketed by CUDA events on its stream; totals are summed per kernel name.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

namespace vie {

extern std::atomic<int> g_prof_on;
void prof_record(const char* name, cudaStream_t st, cudaEvent_t* e0, cudaEvent_t* e1, bool begin);

struct Prof {
  const char* name;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool on;
  Prof(const char* n, cudaStream_t s) : name(n), st(s), on(g_prof_on.load(std::memory_order_relaxed) != 0) {
    if (on) prof_record(name, st, &e0, &e1, true);
  }
  ~Prof() {
    if (on) prof_record(name, st, &e0, &e1, false);
  }
};

inline bool prof_enabled() { return g_prof_on.load(std::memory_order_relaxed) != 0; }

}  // namespace vie
