// Autotuner.  For the shapes of a plan it times the candidate launch variants
// of two kernels on the plan's own buffers and keeps the fastest:
//   * the matvec's x pass (per precision): the compile-time radix-16 kernel
//     where one exists (complex FP32, L = 2048 or 4096) and the generic
//     shared-memory Stockham kernel with three radix orders of L (8s first;
//     reversed; powers of two as 4s);
//   * the kept-block product of each 1-level box: rows of a block split over
//     1, 2, 4 or 8 CTAs (every split computes each output in the same order,
//     so the results do not depend on the choice).
// Choices are cached per process and shape, so all plans of a shape run the
// same kernels (a plan solved alone and in a batch stays bitwise the same).
// VIE_AUTOTUNE=0 in the environment keeps the default rules.  The report of
// a plan's choices and timings is returned by vie_plan_tuning.
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "internal.h"

namespace vie {

bool autotune_enabled() {
  static const bool on = [] {
    const char* e = getenv("VIE_AUTOTUNE");
    return !(e && e[0] == '0');
  }();
  return on;
}

static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<int, std::string>> g_tune;

bool tune_cache_get(const TuneKey& k, int* choice, std::string* report) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *choice = it->second.first;
  *report = it->second.second;
  return true;
}

void tune_cache_put(const TuneKey& k, int choice, const std::string& report) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.emplace(k, std::make_pair(choice, report));
}

// mean device time of reps calls of f after one warm-up call, on stream st
template <class F>
static vie_status time_ms(cudaStream_t st, int reps, F f, float* ms) {
  cudaEvent_t e0, e1;
  VIE_CUDA(cudaEventCreate(&e0));
  VIE_CUDA(cudaEventCreate(&e1));
  vie_status s = f();
  if (s >= 0) {
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && s >= 0; ++r) s = f();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    *ms /= (float)reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

// alternative radix orders of L (the twiddle table of the base plan serves all)
static int radix_orders(int L, const FftPlanDev& base, FftPlanDev out[3]) {
  out[0] = base;
  out[1] = base;
  for (int i = 0; i < base.npass; ++i) out[1].radix[i] = base.radix[base.npass - 1 - i];
  fft_plan_finalize(out[1]);
  FftPlanDev q = base;
  q.npass = 0;
  int m = L, a = 0;
  while (m % 2 == 0) { m /= 2; ++a; }
  bool ok = true;
  auto push = [&](int r) {
    if (q.npass >= FFT_MAX_PASSES) ok = false;
    else q.radix[q.npass++] = r;
  };
  for (; a >= 2; a -= 2) push(4);
  if (a == 1) push(2);
  for (int r : {3, 5, 7})
    for (; m % r == 0; m /= r) push(r);
  if (!ok) return 2;
  fft_plan_finalize(q);
  out[2] = q;
  return 3;
}

static std::string radix_name(const FftPlanDev& p) {
  std::string s = "stockham[";
  for (int i = 0; i < p.npass; ++i) {
    if (i) s += ".";
    s += std::to_string(p.radix[i]);
  }
  return s + "]";
}

template <class C>
static vie_status tune_x(vie_plan_s* P, int pi) {
  const MvDims& d = P->d;
  const bool fused = pi == 0 ? P->fused_x64 : P->fused_x128;
  const FftPlanDev base = pi == 0 ? P->fL->pn32 : P->fL->pn64;
  const int nord = radix_orders(d.L, base, P->xord[pi]);
  const char* tag = pi == 0 ? "x_pass_c64" : "x_pass_c128";
  if (!fused) return VIE_OK;   // the unfused path transforms through S; nothing to choose
  const TuneKey key{0, pi, d.L, d.Py, d.Pz};
  int choice;
  std::string rep;
  if (tune_cache_get(key, &choice, &rep)) {
    P->xvar[pi] = choice;
    P->tuning += rep;
    return VIE_OK;
  }
  C* T = (C*)(pi == 0 ? P->T64.p : P->T128.p);
  C* S = (C*)(pi == 0 ? P->S64.p : P->S128.p);
  const C* spec = (const C*)(pi == 0 ? P->spec64.p : P->spec128.p);
  const long long nT = 3LL * d.Pz * d.Py * d.nx;
  VIE_CUDA(cudaMemsetAsync(T, 0, sizeof(C) * nT, P->st));
  const bool ct = pi == 0 && (d.L == 2048 || d.L == 4096);
  char buf[160];
  snprintf(buf, sizeof(buf), "%s L=%d Py=%d Pz=%d:", tag, d.L, d.Py, d.Pz);
  rep = buf;
  int best = -1;
  float tbest = 0;
  for (int v = ct ? 0 : 1; v <= nord; ++v) {
    // an order equal to an earlier one (a palindromic radix list) is not timed twice
    bool dup = false;
    for (int u = 1; u < v && !dup; ++u) {
      const FftPlanDev &a = P->xord[pi][u - 1], &b = P->xord[pi][v - 1];
      dup = a.npass == b.npass;
      for (int i = 0; dup && i < a.npass; ++i) dup = a.radix[i] == b.radix[i];
    }
    if (dup) continue;
    float ms = 0;
    VIE_TRY(time_ms(P->st, 3, [&] { return xpass<C>(P, spec, T, S, v, P->st); }, &ms));
    const std::string name = v == 0 ? std::string(d.L == 2048 ? "radix16x16x8" : "radix16x16x16")
                                    : radix_name(P->xord[pi][v - 1]);
    snprintf(buf, sizeof(buf), " %s %.4f ms;", name.c_str(), ms);
    rep += buf;
    if (best < 0 || ms < tbest) { best = v; tbest = ms; }
  }
  snprintf(buf, sizeof(buf), " chosen %d\n", best);
  rep += buf;
  tune_cache_put(key, best, rep);
  P->xvar[pi] = best;
  P->tuning += rep;
  return VIE_OK;
}

vie_status tune_matvec(vie_plan_s* P) {
  if (!autotune_enabled()) {
    // default rule, with the radix orders filled in
    radix_orders(P->d.L, P->fL->pn32, P->xord[0]);
    radix_orders(P->d.L, P->fL->pn64, P->xord[1]);
    P->tuning = "autotuning off (VIE_AUTOTUNE=0)\n";
    P->tuning_matvec = P->tuning.size();
    return VIE_OK;
  }
  VIE_TRY(tune_x<float2>(P, 0));
  VIE_TRY(tune_x<double2>(P, 1));
  VIE_CUDA(cudaStreamSynchronize(P->st));
  P->tuning_matvec = P->tuning.size();
  return VIE_OK;
}

}  // namespace vie

extern "C" const char* vie_plan_tuning(vie_plan_t P) { return P ? P->tuning.c_str() : ""; }
