// C ABI of libvie: plan lifecycle, matvec / preconditioner hooks, solves,
// batched solves and the continuous-batching server.
#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"
#include "prof.h"

namespace vie {

static thread_local char g_err[1024] = "";
static thread_local cudaStream_t g_alloc_stream = nullptr;

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

// Stream-ordered allocations on the calling plan's stream: no device-wide
// synchronisation, so concurrent requests keep overlapping.
vie_status DevBuf::alloc(size_t n) {
  release();
  if (n == 0) n = 16;
  cudaError_t e = cudaMallocAsync(&p, n, g_alloc_stream);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    set_error("device allocation of %zu bytes failed: %s", n, cudaGetErrorString(e));
    return VIE_ENOMEM;
  }
  bytes = n;
  stream = g_alloc_stream;
  return VIE_OK;
}

void DevBuf::release() {
  if (p) cudaFreeAsync(p, stream);
  p = nullptr;
  bytes = 0;
}

cudaStream_t alloc_stream() { return g_alloc_stream; }
void set_alloc_stream(cudaStream_t s) { g_alloc_stream = s; }
using StreamScope = AllocScope;

static std::once_flag g_pool_once;
static void init_pool() {
  std::call_once(g_pool_once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  });
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

static bool boxes_valid(int nx, int ny, int nz, const std::vector<vie_box>& bs) {
  for (size_t i = 0; i < bs.size(); ++i) {
    const vie_box& b = bs[i];
    if (b.nx < 1 || b.ny < 1 || b.nz < 1 || b.x0 < 0 || b.y0 < 0 || b.z0 < 0) return false;
    if (b.x0 + b.nx > nx || b.y0 + b.ny > ny || b.z0 + b.nz > nz) return false;
    for (size_t j = 0; j < i; ++j) {
      const vie_box& c = bs[j];
      const bool ox = b.x0 < c.x0 + c.nx && c.x0 < b.x0 + b.nx;
      const bool oy = b.y0 < c.y0 + c.ny && c.y0 < b.y0 + b.ny;
      const bool oz = b.z0 < c.z0 + c.nz && c.z0 < b.z0 + b.nz;
      if (ox && oy && oz) return false;
    }
  }
  return true;
}

static int embed_len(int n) { return 2 * fft_next_smooth(n); }

// x-embedding (any L >= 2 nx - 1 gives the same matvec): 2 smooth(nx), whose
// three complex-FP32 lines one CTA transforms when they fit shared memory
// (or L = 4096, 8192, the compile-time kernels); past that
// L = 8 smooth(ceil(nx / 4)) >= 2 nx, a multiple of 8, and the x pass splits
// the frequencies over a cluster of Q = 2, 4 or 8 CTAs (lines of L/Q; *q is
// the smallest Q that fits, the autotuner may take a larger one); beyond
// that the unfused path through the full x-spectrum.
int embed_x(int nx, int* q) {
  const int L = embed_len(nx);
  const int lq_max = (int)((200 * 1024) / (2 * 3 * sizeof(float2)));   // three lines, two copies
  *q = 1;
  if (L <= lq_max || L == 4096 || L == 8192) return L;
  const int L8 = 8 * fft_next_smooth((nx + 3) / 4);
  for (int Q = 2; Q <= 8; Q *= 2)
    if (L8 / Q <= lq_max) { *q = Q; return L8; }
  return L;
}

std::atomic<int> g_prof_on{0};
struct ProfRec { const char* name; cudaEvent_t e0, e1; };
static std::mutex g_prof_mu;
static std::vector<ProfRec>* g_prof = nullptr;
static std::vector<cudaEvent_t>* g_ev_pool = nullptr;

static cudaEvent_t prof_event() {
  if (!g_ev_pool) g_ev_pool = new std::vector<cudaEvent_t>();
  if (!g_ev_pool->empty()) { cudaEvent_t e = g_ev_pool->back(); g_ev_pool->pop_back(); return e; }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void prof_record(const char* name, cudaStream_t st, cudaEvent_t* e0, cudaEvent_t* e1, bool begin) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (begin) {
    *e0 = prof_event();
    cudaEventRecord(*e0, st);
  } else {
    *e1 = prof_event();
    cudaEventRecord(*e1, st);
    if (!g_prof) g_prof = new std::vector<ProfRec>();
    g_prof->push_back(ProfRec{name, *e0, *e1});
  }
}

}  // namespace vie

namespace vie {

vie_status smem_optin_raw(const void* kern, size_t need) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<int, const void*>, int>> done;
  int dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  int limit = -1;
  for (const auto& d : done)
    if (d.first.first == dev && d.first.second == kern) limit = d.second;
  if (limit < 0) {
    int optin = 0;
    VIE_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    VIE_CUDA(cudaFuncGetAttributes(&fa, kern));
    limit = optin - (int)fa.sharedSizeBytes;
    VIE_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
    done.push_back({{dev, kern}, limit});
  }
  if (need > (size_t)limit) {
    set_error("kernel needs %zu bytes of shared memory, more than the %d available", need, limit);
    return VIE_EINVAL;
  }
  return VIE_OK;
}

}  // namespace vie

using namespace vie;

extern "C" {

void vie_default_opts(vie_opts* o) {
  if (!o) return;
  o->restart = 50;
  o->tol = 1e-9;
  o->max_iter = 5000;
  o->inner_tol = 1e-6;
  o->max_refine = 1000;
  o->precision = VIE_MIXED;
  o->precond = VIE_PREC_CIRCULANT;
  o->homog = VIE_HOM_REALMEAN;
  o->reduce_tol = 1e-3;
  o->boxes = nullptr;
  o->nboxes = 0;
  o->inner_restart = 0;
}

const char* vie_last_error(void) { return g_err; }

void vie_profile_enable(int on) { g_prof_on.store(on ? 1 : 0); }

void vie_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof) return;
  for (auto& r : *g_prof) {
    cudaEventSynchronize(r.e1);
    if (!g_ev_pool) g_ev_pool = new std::vector<cudaEvent_t>();
    g_ev_pool->push_back(r.e0);
    g_ev_pool->push_back(r.e1);
  }
  g_prof->clear();
}

vie_status vie_profile_query(const char* kernel, int64_t* launches, double* total_ms) {
  if (!kernel || !launches || !total_ms) { set_error("vie_profile_query: NULL argument"); return VIE_EINVAL; }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  int64_t n = 0;
  double t = 0;
  if (g_prof) {
    for (auto& r : *g_prof) {
      if (strcmp(r.name, kernel) != 0) continue;
      if (cudaEventSynchronize(r.e1) != cudaSuccess) { set_error("vie_profile_query: event failed"); return VIE_ECUDA; }
      float ms = 0;
      cudaEventElapsedTime(&ms, r.e0, r.e1);
      t += ms;
      ++n;
    }
  }
  *launches = n;
  *total_ms = t;
  return VIE_OK;
}

int vie_profile_kernels(const char** names, int cap) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  std::vector<const char*> seen;
  if (g_prof)
    for (auto& r : *g_prof) {
      bool dup = false;
      for (const char* q : seen) if (strcmp(q, r.name) == 0) { dup = true; break; }
      if (!dup) seen.push_back(r.name);
    }
  for (int i = 0; i < (int)seen.size() && i < cap; ++i) names[i] = seen[i];
  return (int)seen.size();
}

int64_t vie_kernel_launches(void) { return (int64_t)launches_total(); }

vie_status vie_plan_create(int nx, int ny, int nz, double h, double k0, double eps_bg, const vie_opts* opts,
                           void* cuda_stream, vie_plan_t* out) {
  if (!out) { set_error("vie_plan_create: out is NULL"); return VIE_EINVAL; }
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || !(h > 0) || !(k0 >= 0) || !(eps_bg > 0)) {
    set_error("vie_plan_create: invalid grid or physics (nx=%d ny=%d nz=%d h=%g k0=%g eps_bg=%g)", nx, ny, nz, h, k0,
              eps_bg);
    return VIE_EINVAL;
  }
  init_pool();
  std::unique_ptr<vie_plan_s> P(new vie_plan_s());
  P->nx = nx; P->ny = ny; P->nz = nz;
  P->h = h; P->k0 = k0; P->eps_bg = eps_bg;
  P->kb = k0 * sqrt(eps_bg);
  if (opts) P->opts = *opts; else vie_default_opts(&P->opts);
  vie_opts& o = P->opts;
  if (o.restart < 1 || o.restart > 128 || !(o.tol > 0) || o.max_iter < 1 || o.max_refine < 1 ||
      (o.precision != VIE_FP64 && o.precision != VIE_MIXED) ||
      (o.precond != VIE_PREC_NONE && o.precond != VIE_PREC_CIRCULANT) || o.homog < 1 || o.homog > 3 ||
      !(o.reduce_tol >= 0) || !(o.inner_tol > 0) || o.nboxes < 0 || (o.nboxes > 0 && !o.boxes) ||
      o.inner_restart < 0 || o.inner_restart > 128) {
    set_error("vie_plan_create: invalid options");
    return VIE_EINVAL;
  }
  if (o.nboxes > 0) P->boxes.assign(o.boxes, o.boxes + o.nboxes);
  else P->boxes.push_back(vie_box{0, 0, 0, nx, ny, nz});
  o.boxes = nullptr;
  o.nboxes = (int)P->boxes.size();
  if (!boxes_valid(nx, ny, nz, P->boxes)) { set_error("vie_plan_create: boxes out of range or overlapping"); return VIE_EINVAL; }
  P->st = (cudaStream_t)cuda_stream;
  VIE_CUDA(cudaGetDevice(&P->device));
  StreamScope scope(P->st);
  MvDims& d = P->d;
  d.nx = nx; d.ny = ny; d.nz = nz;
  d.L = embed_x(nx, &P->xq); d.Py = embed_len(ny); d.Pz = embed_len(nz);
  d.Lh = d.L / 2 + 1; d.Pyh = d.Py / 2 + 1; d.Pzh = d.Pz / 2 + 1;
  if (d.Py > fft_max_len<double2>() || d.Pz > fft_max_len<double2>()) {
    set_error("vie_plan_create: cross-section embedding %dx%d exceeds one shared-memory line", d.Py, d.Pz);
    return VIE_EINVAL;
  }
  if (3LL * nx * ny * nz >= (1LL << 31) - 64) {
    // the streaming kernels index a vector with 32-bit arithmetic
    set_error("vie_plan_create: 3*nx*ny*nz = %lld unknowns, the limit is 2^31 - 64", 3LL * nx * ny * nz);
    return VIE_EINVAL;
  }
  if (d.L > 2 * fft_max_len<double2>()) {
    set_error("vie_plan_create: nx=%d needs an x-embedding of %d > %d points", nx, d.L, 2 * fft_max_len<double2>());
    return VIE_EINVAL;
  }
  for (const vie_box& b : P->boxes) {
    if (b.levels < 0 || b.levels > 2) { set_error("vie_plan_create: box levels must be 0, 1 or 2"); return VIE_EINVAL; }
    if (P->opts.precond == VIE_PREC_NONE) continue;   // the boxes carry no blocks
    // the Chan eigenvalues are transformed in FP64; one split doubles the limit
    // (x-lines for every box, y-lines too for a 2-level box)
    for (int axis = 0; axis < (b.levels == 2 ? 2 : 1); ++axis) {
      const int nb = axis == 0 ? b.nx : b.ny;
      const FftLen* f;
      VIE_TRY(fft_get(nb, &f));
      const int len = f->bluestein ? f->M : f->n;
      if (len > 2 * fft_max_len<double2>()) {
        set_error("vie_plan_create: box length %d needs a transform of %d points (limit %d)", nb, len,
                  2 * fft_max_len<double2>());
        return VIE_EINVAL;
      }
      if (len > fft_max_len<double2>()) {
        const FftLen* h;
        VIE_TRY(fft_get(len / 2, &h));   // half length used by the split, cached before any capture
      }
    }
    if (b.levels == 2) {
      if (b.nz > 32) { set_error("vie_plan_create: 2-level box needs nz <= 32 (blocks of 3 nz rows)"); return VIE_EINVAL; }
      if ((b.nx / 2 + 1LL) * (b.ny / 2 + 1LL) > 65535) {
        set_error("vie_plan_create: 2-level box stores (nx/2+1)(ny/2+1) > 65535 blocks");
        return VIE_EINVAL;
      }
    } else if (3 * b.ny * b.nz > 864) {
      set_error("vie_plan_create: box cross-section too large (m = 3 ny nz > 864)");
      return VIE_EINVAL;
    }
  }
  VIE_TRY(fft_get(d.L, &P->fL));
  if (P->xq > 1) {
    for (int Q = P->xq, i = P->xq == 2 ? 0 : P->xq == 4 ? 1 : 2; Q <= 8; Q *= 2, ++i)
      VIE_TRY(fft_get(d.L / Q, &P->fLq[i]));
    std::vector<float2> tw(d.L);
    for (int j = 0; j < d.L; ++j) {
      const double a = -2.0 * M_PI * (double)j / (double)d.L;
      tw[j] = make_float2((float)cos(a), (float)sin(a));
    }
    VIE_TRY(P->twL64.alloc(sizeof(float2) * d.L));
    VIE_CUDA(cudaMemcpyAsync(P->twL64.p, tw.data(), sizeof(float2) * d.L, cudaMemcpyHostToDevice, P->st));
    VIE_CUDA(cudaStreamSynchronize(P->st));   // tw lives on this stack frame
  }
  if (d.L > fft_max_len<float2>() || d.L > fft_max_len<double2>()) {
    const FftLen* h;
    VIE_TRY(fft_get(d.L / 2, &h));   // half length used by the split, cached before any capture
  }
  VIE_TRY(fft_get(d.Py, &P->fPy));
  VIE_TRY(fft_get(d.Pz, &P->fPz));
  VIE_TRY(build_spectra(P.get()));
  VIE_TRY(matvec_alloc(P.get()));
  VIE_TRY(tune_matvec(P.get()));
  VIE_TRY(P->dev_err.alloc(sizeof(int)));
  VIE_CUDA(cudaMemsetAsync(P->dev_err.p, 0, sizeof(int), P->st));
  *out = P.release();
  return VIE_OK;
}

void vie_plan_destroy(vie_plan_t P) {
  if (!P) return;
  {
    StreamScope scope(P->st);
    cudaStreamSynchronize(P->st);
    krylov_free(P);
    precond_free(P);
    delete P;
  }
  cudaGetLastError();
}

vie_status vie_set_permittivity(vie_plan_t P, const void* eps) {
  if (!P || !eps) { set_error("vie_set_permittivity: NULL argument"); return VIE_EINVAL; }
  StreamScope scope(P->st);
  VIE_TRY(set_material(P, (const double2*)eps));
  precond_free(P);
  reset_graphs(P);
  P->has_eps = true;
  return VIE_OK;
}

vie_status vie_build_preconditioner(vie_plan_t P) {
  if (!P) { set_error("vie_build_preconditioner: NULL plan"); return VIE_EINVAL; }
  if (!P->has_eps) { set_error("vie_build_preconditioner: permittivity not set"); return VIE_ESTATE; }
  StreamScope scope(P->st);
  reset_graphs(P);
  VIE_TRY(precond_build(P));
  VIE_CUDA(cudaStreamSynchronize(P->st));
  return VIE_OK;
}

vie_status vie_matvec(vie_plan_t P, const void* x, void* y, int precision) {
  if (!P || !x || !y || x == y) { set_error("vie_matvec: bad arguments"); return VIE_EINVAL; }
  if (!P->has_eps) { set_error("vie_matvec: permittivity not set"); return VIE_ESTATE; }
  StreamScope scope(P->st);
  const long long n3 = 3LL * P->nx * P->ny * P->nz;
  if (precision == VIE_FP64) {
    return matvec<double2>(P, (const double2*)x, (double2*)y, P->M128.as<double2>(), P->spec128.as<double2>(),
                           P->T128.as<double2>(), P->S128.as<double2>(), P->st);
  }
  if (precision != VIE_MIXED) { set_error("vie_matvec: bad precision"); return VIE_EINVAL; }
  VIE_TRY(narrow((const double2*)x, P->xin64.as<float2>(), n3, P->st));
  VIE_TRY(matvec<float2>(P, P->xin64.as<float2>(), P->xout64.as<float2>(), P->M64.as<float2>(),
                         P->spec64.as<float2>(), P->T64.as<float2>(), P->S64.as<float2>(), P->st));
  return widen(P->xout64.as<float2>(), (double2*)y, n3, P->st);
}

vie_status vie_precond_apply(vie_plan_t P, const void* r, void* z, int precision) {
  if (!P || !r || !z || r == z) { set_error("vie_precond_apply: bad arguments"); return VIE_EINVAL; }
  if (!P->prec_built) { set_error("vie_precond_apply: preconditioner not built"); return VIE_ESTATE; }
  StreamScope scope(P->st);
  const long long n3 = 3LL * P->nx * P->ny * P->nz;
  if (precision == VIE_FP64) return precond_apply<double2>(P, (const double2*)r, (double2*)z, P->st);
  if (precision != VIE_MIXED) { set_error("vie_precond_apply: bad precision"); return VIE_EINVAL; }
  VIE_TRY(narrow((const double2*)r, P->xin64.as<float2>(), n3, P->st));
  VIE_TRY(precond_apply<float2>(P, P->xin64.as<float2>(), P->xout64.as<float2>(), P->st));
  return widen(P->xout64.as<float2>(), (double2*)z, n3, P->st);
}

vie_status vie_solve(vie_plan_t P, const void* e_inc, void* w_out, vie_info* info) {
  if (!P || !e_inc || !w_out) { set_error("vie_solve: NULL argument"); return VIE_EINVAL; }
  StreamScope scope(P->st);
  return solve(P, (const double2*)e_inc, (double2*)w_out, info);
}

vie_status vie_solve_host(vie_plan_t P, const void* eps_host, const void* e_inc_host, void* w_out_host,
                          vie_info* info) {
  if (!P || !eps_host || !e_inc_host || !w_out_host) { set_error("vie_solve_host: NULL argument"); return VIE_EINVAL; }
  StreamScope scope(P->st);
  const long long N = (long long)P->nx * P->ny * P->nz;
  // device staging buffers: allocated by the first call, kept by the plan
  DevBuf &eps = P->h_eps, &e = P->h_e, &w = P->h_w;
  if (!eps.p) VIE_TRY(eps.alloc(sizeof(double2) * N));
  if (!e.p) VIE_TRY(e.alloc(sizeof(double2) * 3 * N));
  if (!w.p) VIE_TRY(w.alloc(sizeof(double2) * 3 * N));
  VIE_CUDA(cudaMemcpyAsync(eps.p, eps_host, sizeof(double2) * N, cudaMemcpyHostToDevice, P->st));
  VIE_CUDA(cudaMemcpyAsync(e.p, e_inc_host, sizeof(double2) * 3 * N, cudaMemcpyHostToDevice, P->st));
  VIE_TRY(vie_set_permittivity(P, eps.p));
  const vie_status s = solve(P, e.as<double2>(), w.as<double2>(), info);
  if (s < 0) return s;
  VIE_CUDA(cudaMemcpyAsync(w_out_host, w.p, sizeof(double2) * 3 * N, cudaMemcpyDeviceToHost, P->st));
  VIE_CUDA(cudaStreamSynchronize(P->st));
  return s;
}

vie_status vie_solve_batch(vie_plan_t* plans, int n, const void* const* e_inc, void* const* w_out, vie_info* info) {
  if (n < 0 || (n > 0 && (!plans || !e_inc || !w_out))) { set_error("vie_solve_batch: bad arguments"); return VIE_EINVAL; }
  if (n == 0) return VIE_OK;
  int dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !e_inc[i] || !w_out[i]) { set_error("vie_solve_batch: NULL plan or vector %d", i); return VIE_EINVAL; }
    if (plans[i]->device != dev) { set_error("vie_solve_batch: plan %d belongs to another device", i); return VIE_EINVAL; }
    for (int k = 0; k < i; ++k)
      if (plans[k] == plans[i]) { set_error("vie_solve_batch: plan %d appears twice", i); return VIE_EINVAL; }
  }
  cudaStream_t st;
  VIE_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  std::vector<vie_status> status(n, VIE_OK);
  vie_status worst;
  {
    StreamScope scope(st);
    worst = solve_many(reinterpret_cast<vie_plan_s* const*>(plans), n,
                       reinterpret_cast<const double2* const*>(e_inc), reinterpret_cast<double2* const*>(w_out), info,
                       status.data(), st);
  }
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  return worst;
}

size_t vie_estimate_bytes(int nx, int ny, int nz, const vie_opts* opts) {
  vie_opts o;
  if (opts) o = *opts; else vie_default_opts(&o);
  const double N = (double)nx * ny * nz;
  int xq = 1;
  const double L = embed_x(nx, &xq), Py = 2.0 * fft_next_smooth(ny), Pz = 2.0 * fft_next_smooth(nz);
  const double spec = 6.0 * (L / 2 + 1) * (Py / 2 + 1) * (Pz / 2 + 1) * (16 + 8);
  const double full = L * Py * Pz * 16;                  // spectra assembly scratch
  const double T = 3.0 * Pz * Py * nx * (16 + 8) + ((double)Py * Pz > 4096 ? 3.0 * nz * Py * nx * (16 + 8) : 0);
  // full x-spectra of the unfused x pass (complex FP32 only without a cluster split)
  const double Sx = (3.0 * L * 16 > 200 * 1024 ? 3.0 * Pz * Py * L * 16 : 0) +
                    (3.0 * L * 8 > 200 * 1024 && xq == 1 ? 3.0 * Pz * Py * L * 8 : 0);
  const double Xs = (L > 12736) ? 3.0 * Pz * Py * L * 16 + L * Py * Pz * 16 : 0;   // long-line split scratch
  const double vec = N * 3 * (16 * 6 + 8 * 8) + N * 24;
  const int R = o.precision == VIE_MIXED ? (o.inner_restart > 0 ? o.inner_restart : std::min(2 * o.restart, 128))
                                         : o.restart;
  const double basis = N * 3 * (R + 1) * (o.precision == VIE_MIXED ? 8 : 16);
  double prec = 0;
  if (o.precond == VIE_PREC_CIRCULANT) {
    std::vector<vie_box> bs;
    if (o.nboxes > 0 && o.boxes) bs.assign(o.boxes, o.boxes + o.nboxes);
    else bs.push_back(vie_box{0, 0, 0, nx, ny, nz});
    for (const vie_box& b : bs) {
      if (b.levels == 2) {
        const double m2 = 3.0 * b.nz, nblk = (b.nx / 2 + 1.0) * (b.ny / 2 + 1.0);
        const double lam = 6.0 * (2 * b.nz - 1) * b.ny * b.nx * 16 * 2;
        prec += lam + nblk * m2 * m2 * (16 + (o.precision == VIE_MIXED ? 8 : 16)) + 4.0 * b.nx * b.ny * m2 * 16;
        continue;
      }
      const double m = 3.0 * b.ny * b.nz;
      const double half = b.nx / 2 + 1;
      const double kept = o.reduce_tol > 0 ? std::min(half, 0.3 * half + 2) : half;
      const double lam = 6.0 * (2 * b.ny - 1) * (2 * b.nz - 1) * b.nx * 16 * 2;
      const double blocks = kept * m * m * (16 + (o.precision == VIE_MIXED ? 8 : 16));
      prec += lam + blocks + 4.0 * b.nx * m * 16;
    }
  }
  return (size_t)(spec + full + T + Sx + Xs + vec + basis + prec + 64.0 * 1024 * 1024);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// continuous-batching server
//
// Requests wait in a FIFO queue until their estimated device footprint fits
// the budget and fewer than max_inflight are admitted.  Preparation workers
// (threads) each take an admitted request: plan creation on the request's
// own stream, the upload of its permittivity and incident field, the
// preconditioner build and the start of its solve.  One driver thread keeps
// every prepared request in a lockstep set: each pass runs a chunk of Arnoldi
// steps of all of them as one step graph (the step kernels as single launches
// over the work-list of the set), and requests join the set between passes
// as they become ready and leave it as they finish, so the batch on the GPU
// changes continuously.  A finished request's result is copied to its host
// buffer, its plan released, and its status published.
// ---------------------------------------------------------------------------
struct SrvReq {
  int64_t id;
  int nx, ny, nz;
  double h, k0, eps_bg;
  vie_opts opts;
  std::vector<vie_box> boxes;
  std::vector<double2> eps, e;
  void* w_out;
  size_t est;
  vie_status status = VIE_PENDING;
  vie_info info{};
  std::string err;
  // while admitted (owned by one thread at a time: worker, then driver)
  cudaStream_t st = nullptr;
  vie_plan_t plan = nullptr;
  vie::Run* run = nullptr;
  vie_info run_info{};
};

struct vie_server_s {
  size_t budget = 0;
  int max_inflight = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_ready;
  std::deque<SrvReq*> queue;              // submitted, not admitted
  std::deque<SrvReq*> ready;              // prepared, waiting to join the lockstep set
  std::map<int64_t, std::unique_ptr<SrvReq>> all;
  size_t reserved = 0;
  int running = 0;                        // admitted and not finished
  int64_t next_id = 1;
  bool stop = false;
  std::vector<std::thread> workers;
  std::thread driver;
};

// release an admitted request's resources (on the thread that owns it)
static void server_release(SrvReq* R) {
  if (R->run) vie::run_delete(R->run);
  R->run = nullptr;
  if (R->plan) vie_plan_destroy(R->plan);
  R->plan = nullptr;
  if (R->st) cudaStreamDestroy(R->st);
  R->st = nullptr;
}

// publish a finished request (status last, under the mutex: a poller that
// sees it also sees info, the result and the error text)
static void server_publish(vie_server_s* S, SrvReq* R, vie_status st, const vie_info& info, const std::string& err) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    R->info = info;
    R->err = err;
    R->status = st;
    R->eps.clear(); R->eps.shrink_to_fit();
    R->e.clear(); R->e.shrink_to_fit();
    S->reserved -= R->est;
    S->running -= 1;
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
}

// preparation: plan, inputs, preconditioner, start of the solve
static vie_status server_prepare(SrvReq* R) {
  VIE_CUDA(cudaStreamCreateWithFlags(&R->st, cudaStreamNonBlocking));
  VIE_TRY(vie_plan_create(R->nx, R->ny, R->nz, R->h, R->k0, R->eps_bg, &R->opts, R->st, &R->plan));
  vie_plan_s* P = R->plan;
  StreamScope scope(P->st);
  const long long N = (long long)P->nx * P->ny * P->nz;
  VIE_TRY(P->h_eps.alloc(sizeof(double2) * N));
  VIE_TRY(P->h_e.alloc(sizeof(double2) * 3 * N));
  VIE_TRY(P->h_w.alloc(sizeof(double2) * 3 * N));
  VIE_CUDA(cudaMemcpyAsync(P->h_eps.p, R->eps.data(), sizeof(double2) * N, cudaMemcpyHostToDevice, P->st));
  VIE_CUDA(cudaMemcpyAsync(P->h_e.p, R->e.data(), sizeof(double2) * 3 * N, cudaMemcpyHostToDevice, P->st));
  VIE_TRY(vie_set_permittivity(P, P->h_eps.p));
  VIE_CUDA(cudaStreamSynchronize(P->st));   // host copies of the inputs may go
  R->run = vie::run_new(P, P->h_e.as<double2>(), P->h_w.as<double2>(), &R->run_info);
  return vie::run_start(R->run);
}

static void server_worker(vie_server_s* S) {
  cudaSetDevice(S->device);
  for (;;) {
    SrvReq* R = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // admit the oldest request once its footprint fits the budget
      S->cv_work.wait(lk, [&] {
        return S->stop || (!S->queue.empty() && S->running < S->max_inflight &&
                           S->reserved + S->queue.front()->est <= S->budget);
      });
      if (S->stop) break;
      R = S->queue.front();
      S->queue.pop_front();
      S->reserved += R->est;
      S->running += 1;
    }
    const vie_status s = server_prepare(R);
    if (s < 0 || vie::run_finished(R->run)) {
      // failed, or finished at once (a zero right-hand side)
      std::string err = s < 0 ? std::string(vie_last_error()) : std::string();
      vie_status st = s;
      if (s >= 0) {
        st = vie::run_status(R->run, &err);
        if (st >= 0 && cudaMemcpy(R->w_out, R->plan->h_w.p, sizeof(double2) * 3 * (size_t)R->nx * R->ny * R->nz,
                                  cudaMemcpyDeviceToHost) != cudaSuccess) {
          st = VIE_ECUDA;
          err = "vie_server: result copy failed";
        }
      } else if (R->run) {
        vie::run_status(R->run, &err);
      }
      const vie_info info = R->run_info;
      server_release(R);
      server_publish(S, R, st, info, err);
      continue;
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->ready.push_back(R);
    }
    S->cv_ready.notify_all();
  }
}

static void server_driver(vie_server_s* S) {
  cudaSetDevice(S->device);
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  vie::Lockstep* L = nullptr;
  {
    StreamScope scope(st);
    L = vie::lockstep_new();
  }
  std::vector<SrvReq*> active;
  std::vector<vie::Run*> runs;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (active.empty()) S->cv_ready.wait(lk, [&] { return S->stop || !S->ready.empty(); });
      if (S->stop) break;
      while (!S->ready.empty()) {   // requests join the set between passes
        active.push_back(S->ready.front());
        S->ready.pop_front();
      }
    }
    runs.clear();
    for (SrvReq* R : active) runs.push_back(R->run);
    bool stepped;
    {
      StreamScope scope(st);
      stepped = vie::lockstep_pass(L, runs, st);
    }
    if (!stepped) {
      // every run of the set is either in a cycle or finished; a run in
      // neither state would never progress: fail it rather than spin
      for (SrvReq* R : active)
        if (!vie::run_finished(R->run)) vie::run_abort(R->run, "vie_server: request lost its GMRES cycle");
    }
    // requests that finished leave the set
    for (size_t i = 0; i < active.size();) {
      SrvReq* R = active[i];
      if (!vie::run_finished(R->run)) { ++i; continue; }
      std::string err;
      vie_status s = vie::run_status(R->run, &err);
      if (s >= 0) {
        vie_plan_s* P = R->plan;
        if (cudaMemcpyAsync(R->w_out, P->h_w.p, sizeof(double2) * 3 * (size_t)P->nx * P->ny * P->nz,
                            cudaMemcpyDeviceToHost, P->st) != cudaSuccess ||
            cudaStreamSynchronize(P->st) != cudaSuccess) {
          s = VIE_ECUDA;
          err = "vie_server: result copy failed";
        }
      }
      const vie_info info = R->run_info;
      server_release(R);
      server_publish(S, R, s, info, err);
      active.erase(active.begin() + i);
    }
  }
  for (SrvReq* R : active) {
    server_release(R);
    server_publish(S, R, VIE_EREJECTED, vie_info{}, "server destroyed");
  }
  {
    StreamScope scope(st);
    vie::lockstep_release(L);
    vie::lockstep_free(L);
  }
  cudaStreamDestroy(st);
}

extern "C" {

vie_status vie_server_create(size_t budget_bytes, int max_inflight, vie_server_t* out) {
  if (!out || budget_bytes == 0 || max_inflight < 1 || max_inflight > 256) {
    set_error("vie_server_create: bad arguments");
    return VIE_EINVAL;
  }
  init_pool();
  vie_server_s* S = new vie_server_s();
  S->budget = budget_bytes;
  S->max_inflight = max_inflight;
  cudaGetDevice(&S->device);
  // preparation workers: up to four plans built at once beside the solves
  for (int i = 0; i < std::min(max_inflight, 4); ++i) S->workers.emplace_back(server_worker, S);
  S->driver = std::thread(server_driver, S);
  *out = S;
  return VIE_OK;
}

vie_status vie_server_submit(vie_server_t S, int nx, int ny, int nz, double h, double k0, double eps_bg,
                             const vie_opts* opts, const void* eps_host, const void* e_inc_host, void* w_out_host,
                             int64_t* ticket) {
  if (!S || !eps_host || !e_inc_host || !w_out_host || !ticket || nx < 1 || ny < 1 || nz < 1) {
    set_error("vie_server_submit: bad arguments");
    return VIE_EINVAL;
  }
  std::unique_ptr<SrvReq> R(new SrvReq());
  R->nx = nx; R->ny = ny; R->nz = nz; R->h = h; R->k0 = k0; R->eps_bg = eps_bg;
  if (opts) R->opts = *opts; else vie_default_opts(&R->opts);
  if (R->opts.nboxes > 0 && R->opts.boxes) R->boxes.assign(R->opts.boxes, R->opts.boxes + R->opts.nboxes);
  R->opts.boxes = R->boxes.empty() ? nullptr : R->boxes.data();
  R->opts.nboxes = (int)R->boxes.size();
  R->est = vie_estimate_bytes(nx, ny, nz, &R->opts);
  const size_t N = (size_t)nx * ny * nz;
  R->w_out = w_out_host;
  std::lock_guard<std::mutex> lk(S->mu);
  R->id = S->next_id++;
  *ticket = R->id;
  if (R->est > S->budget) {
    R->status = VIE_EREJECTED;
    R->err = "request footprint exceeds the server budget";
    S->all[R->id] = std::move(R);
    set_error("vie_server_submit: request footprint exceeds the server budget");
    return VIE_EREJECTED;
  }
  R->eps.assign((const double2*)eps_host, (const double2*)eps_host + N);
  R->e.assign((const double2*)e_inc_host, (const double2*)e_inc_host + 3 * N);
  S->queue.push_back(R.get());
  S->all[R->id] = std::move(R);
  S->cv_work.notify_all();
  return VIE_OK;
}

vie_status vie_server_poll(vie_server_t S, int64_t ticket, vie_info* info) {
  if (!S) { set_error("vie_server_poll: NULL server"); return VIE_EINVAL; }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) { set_error("vie_server_poll: unknown ticket"); return VIE_EINVAL; }
  SrvReq* R = it->second.get();
  if (R->status == VIE_PENDING) return VIE_PENDING;
  if (info) *info = R->info;
  if (R->status < 0) set_error("%s", R->err.c_str());
  return R->status;
}

vie_status vie_server_drain(vie_server_t S, double timeout_ms) {
  if (!S) { set_error("vie_server_drain: NULL server"); return VIE_EINVAL; }
  std::unique_lock<std::mutex> lk(S->mu);
  const auto pred = [&] { return S->queue.empty() && S->running == 0; };
  if (timeout_ms < 0) { S->cv_done.wait(lk, pred); return VIE_OK; }
  if (!S->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred)) {
    set_error("vie_server_drain: timed out");
    return VIE_ETIMEOUT;
  }
  return VIE_OK;
}

size_t vie_server_reserved_bytes(vie_server_t S) {
  if (!S) return 0;
  std::lock_guard<std::mutex> lk(S->mu);
  return S->reserved;
}

void vie_server_destroy(vie_server_t S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (SrvReq* R : S->queue) { R->status = VIE_EREJECTED; R->err = "server destroyed"; }
    S->queue.clear();
  }
  S->cv_work.notify_all();
  S->cv_ready.notify_all();
  for (auto& t : S->workers) t.join();
  S->driver.join();
  // prepared requests that never joined the set
  for (SrvReq* R : S->ready) {
    server_release(R);
    R->status = VIE_EREJECTED;
    R->err = "server destroyed";
  }
  delete S;
}

}  // extern "C"
