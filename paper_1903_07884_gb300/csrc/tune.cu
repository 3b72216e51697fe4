// Autotuner.  For the shapes of a plan it times the candidate launch variants
// of three kernels on the plan's own buffers and keeps the fastest:
//   * the matvec's yz passes (complex FP32): 16, 8 or 4 x-columns per CTA of
//     the register kernels (power-of-two cross-sections), 1 to 16 of the
//     generic shared-memory kernels otherwise (every choice transforms the
//     same columns the same way, so results do not depend on it);
//   * the matvec's x pass (per precision): the compile-time kernels where
//     they exist (complex FP32: three passes 16x16x8 for L = 2048, 16x16x16
//     for 4096; four passes 16x16x4x4 for 4096, 16x16x8x4 for 8192) and the
//     generic shared-memory Stockham kernel with three radix orders of L (8s
//     first; reversed; powers of two as 4s);
//   * the kept-block product of each 1-level box: rows of a block split over
//     1, 2, 4 or 8 CTAs (every split computes each output in the same order,
//     so the results do not depend on the choice).
// Choices are cached per process and shape, so all plans of a shape run the
// same kernels (a plan solved alone and in a batch stays bitwise the same).
// VIE_AUTOTUNE=0 in the environment keeps the default rules; VIE_TUNE_FILE
// keeps the choices across processes.  The report of a plan's choices and
// timings is returned by vie_plan_tuning.
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

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
static bool g_tune_loaded = false;

// VIE_TUNE_FILE names a file of earlier choices ("kernel precision a b c
// choice" per line) read at the first lookup; new choices are appended to it,
// so that another process (a profiler run, say) reuses them.
static const char* tune_file() {
  const char* f = getenv("VIE_TUNE_FILE");
  return (f && f[0]) ? f : nullptr;
}

static void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* fn = tune_file();
  if (!fn) return;
  FILE* f = fopen(fn, "r");
  if (!f) return;
  int k, p, a, b, c, ch;
  while (fscanf(f, "%d %d %d %d %d %d", &k, &p, &a, &b, &c, &ch) == 6)
    g_tune.emplace(TuneKey{k, p, a, b, c}, std::make_pair(ch, std::string("(from VIE_TUNE_FILE) chosen ") +
                                                                  std::to_string(ch) + "\n"));
  fclose(f);
}

bool tune_cache_get(const TuneKey& k, int* choice, std::string* report) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *choice = it->second.first;
  *report = it->second.second;
  return true;
}

void tune_cache_put(const TuneKey& k, int choice, const std::string& report) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load_locked();
  if (!g_tune.emplace(k, std::make_pair(choice, report)).second) return;
  if (const char* fn = tune_file()) {
    if (FILE* f = fopen(fn, "a")) {
      fprintf(f, "%d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k),
              std::get<4>(k), choice);
      fclose(f);
    }
  }
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
  const bool split = pi == 0 && P->xq > 1;   // the cluster-split kernels (variants 5..7) are candidates
  if (!fused && !split) return VIE_OK;   // the unfused path transforms through S; nothing to choose
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
  const bool ct = pi == 0 && (d.L == 2048 || d.L == 4096);   // three-pass compile-time kernel (variant 0)
  const bool fp = pi == 0 && (d.L == 4096 || d.L == 8192);   // four-pass compile-time kernel (variant 4)
  char buf[160];
  snprintf(buf, sizeof(buf), "%s L=%d Py=%d Pz=%d:", tag, d.L, d.Py, d.Pz);
  rep = buf;
  int best = -1;
  float tbest = 0;
  std::vector<int> cands;
  if (ct) cands.push_back(0);
  for (int v = 1; fused && v <= nord; ++v) cands.push_back(v);
  if (fp) cands.push_back(4);
  for (int Q = P->xq; split && Q <= 8; Q *= 2) cands.push_back(4 + (Q == 2 ? 1 : Q == 4 ? 2 : 3));
  for (int v : cands) {
    // an order equal to an earlier one (a palindromic radix list) is not timed twice
    bool dup = false;
    for (int u = 1; v <= 3 && u < v && !dup; ++u) {
      const FftPlanDev &a = P->xord[pi][u - 1], &b = P->xord[pi][v - 1];
      dup = a.npass == b.npass;
      for (int i = 0; dup && i < a.npass; ++i) dup = a.radix[i] == b.radix[i];
    }
    if (dup) continue;
    float ms = 0;
    VIE_TRY(time_ms(P->st, 3, [&] { return xpass<C>(P, spec, T, S, v, P->st); }, &ms));
    const std::string name = v == 0   ? std::string(d.L == 2048 ? "radix16x16x8" : "radix16x16x16")
                             : v == 4 ? std::string(d.L == 4096 ? "radix16x16x4x4" : "radix16x16x8x4")
                             : v >= 5 ? "cluster" + std::to_string(1 << (v - 4)) + "x" + radix_name(P->fLq[v - 5]->pn32)
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

// x-columns per CTA of the register yz passes (forward and inverse timed
// together; every choice transforms the same columns the same way)
static vie_status tune_yz_generic(vie_plan_s* P);

static vie_status tune_yz(vie_plan_s* P) {
  const MvDims& d = P->d;
  if (yz_pair(P, 16, P->st) == VIE_EINVAL) {
    cudaGetLastError();
    return tune_yz_generic(P);
  }
  const TuneKey key{2, 0, d.Py, d.Pz, d.nx * 64 + d.nz};
  int choice;
  std::string rep;
  if (!tune_cache_get(key, &choice, &rep)) {
    const long long n3 = 3LL * d.nx * d.ny * d.nz;
    VIE_CUDA(cudaMemsetAsync(P->xin64.p, 0, sizeof(float2) * n3, P->st));
    char buf[160];
    snprintf(buf, sizeof(buf), "yz_passes_c64 nx=%d Py=%d Pz=%d nz=%d:", d.nx, d.Py, d.Pz, d.nz);
    rep = buf;
    int best = 0;
    float tbest = 0;
    for (int xg : {16, 8, 4}) {
      float ms = 0;
      VIE_TRY(time_ms(P->st, 3, [&] { return yz_pair(P, xg, P->st); }, &ms));
      snprintf(buf, sizeof(buf), " %d columns/CTA %.4f ms;", xg, ms);
      rep += buf;
      if (best == 0 || ms < tbest) { best = xg; tbest = ms; }
    }
    snprintf(buf, sizeof(buf), " chosen %d\n", best);
    rep += buf;
    choice = best;
    tune_cache_put(key, choice, rep);
  }
  P->yzxg = choice;
  P->tuning += rep;
  return VIE_OK;
}

// x-columns per CTA of the generic (shared-memory Stockham) yz passes, for
// cross-sections without a register variant: 1, 2, 4, 8, 16 as shared memory
// allows (each column is transformed the same way whatever the grouping)
static vie_status tune_yz_generic(vie_plan_s* P) {
  const MvDims& d = P->d;
  if (yz_pair_generic(P, 1, P->st) == VIE_EINVAL) {
    cudaGetLastError();
    return VIE_OK;
  }
  const TuneKey key{3, 0, d.Py, d.Pz, d.nx * 64 + d.nz};
  int choice;
  std::string rep;
  if (!tune_cache_get(key, &choice, &rep)) {
    const long long n3 = 3LL * d.nx * d.ny * d.nz;
    VIE_CUDA(cudaMemsetAsync(P->xin64.p, 0, sizeof(float2) * n3, P->st));
    char buf[160];
    snprintf(buf, sizeof(buf), "yz_generic_c64 nx=%d Py=%d Pz=%d nz=%d:", d.nx, d.Py, d.Pz, d.nz);
    rep = buf;
    int best = 0;
    float tbest = 0;
    for (int xg : {1, 2, 4, 8, 16}) {
      if (xg > std::max(1, d.nx)) break;
      if (2 * (size_t)xg * (d.Py * d.Pz + 1) * sizeof(float2) > 200 * 1024) break;
      float ms = 0;
      VIE_TRY(time_ms(P->st, 3, [&] { return yz_pair_generic(P, xg, P->st); }, &ms));
      snprintf(buf, sizeof(buf), " %d columns/CTA %.4f ms;", xg, ms);
      rep += buf;
      if (best == 0 || ms < tbest) { best = xg; tbest = ms; }
    }
    snprintf(buf, sizeof(buf), " chosen %d\n", best);
    rep += buf;
    choice = best;
    tune_cache_put(key, choice, rep);
  }
  P->yzxg_gen = choice;
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
  VIE_TRY(tune_yz(P));
  VIE_TRY(tune_x<float2>(P, 0));
  VIE_TRY(tune_x<double2>(P, 1));
  VIE_CUDA(cudaStreamSynchronize(P->st));
  P->tuning_matvec = P->tuning.size();
  return VIE_OK;
}

}  // namespace vie

extern "C" const char* vie_plan_tuning(vie_plan_t P) { return P ? P->tuning.c_str() : ""; }

extern "C" vie_status vie_plan_set_tuning(vie_plan_t P, const char* kernel, int choice) {
  using namespace vie;
  if (!P || !kernel) { set_error("vie_plan_set_tuning: NULL argument"); return VIE_EINVAL; }
  const std::string k = kernel;
  const MvDims& d = P->d;
  if (k == "x_pass_c64" || k == "x_pass_c128") {
    const bool c64 = k == "x_pass_c64";
    const bool fused = c64 ? P->fused_x64 : P->fused_x128;
    const bool ok = choice == -1 || (choice >= 1 && choice <= 3 && (fused || !c64 || P->xq == 1)) ||
                    (c64 && choice == 0 && (d.L == 2048 || d.L == 4096)) ||
                    (c64 && choice == 4 && (d.L == 4096 || d.L == 8192)) || (c64 && choice >= 5 && choice <= 7 && P->xq > 1 && (1 << (choice - 4)) >= P->xq);
    if (!ok) { set_error("vie_plan_set_tuning: x-pass variant %d does not exist for L = %d", choice, d.L); return VIE_EINVAL; }
    P->xvar[c64 ? 0 : 1] = choice;
  } else if (k == "yz_generic_c64") {
    if (choice < 1 || choice > 16 || (choice & (choice - 1)) ||
        2 * (size_t)choice * (d.Py * d.Pz + 1) * sizeof(float2) > 200 * 1024) {
      set_error("vie_plan_set_tuning: generic yz columns must be 1..16 (power of two, fitting shared memory)");
      return VIE_EINVAL;
    }
    P->yzxg_gen = choice;
  } else if (k == "yz_passes_c64") {
    if (choice != 16 && choice != 8 && choice != 4) { set_error("vie_plan_set_tuning: yz columns must be 16, 8 or 4"); return VIE_EINVAL; }
    P->yzxg = choice;
  } else if (k == "block_gemv") {
    if (choice != 1 && choice != 2 && choice != 4 && choice != 8) {
      set_error("vie_plan_set_tuning: CTAs per block must be 1, 2, 4 or 8");
      return VIE_EINVAL;
    }
    for (auto& B : P->bp) B->gemv_split[P->opts.precision == VIE_FP64] = choice;
  } else if (k == "rep_gemm_tc") {
    if (choice != 64 && choice != 32) { set_error("vie_plan_set_tuning: the N tile must be 64 or 32"); return VIE_EINVAL; }
    VIE_TRY(precond_set_rep_tile(P, choice));
  } else {
    set_error("vie_plan_set_tuning: unknown kernel '%s'", kernel);
    return VIE_EINVAL;
  }
  reset_graphs(P);   // captured steps hold the old launch shapes
  return VIE_OK;
}
