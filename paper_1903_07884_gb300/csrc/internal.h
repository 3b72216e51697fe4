// Internal declarations shared by the libvie translation units.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "fft.cuh"
#include "vie_common.cuh"

namespace vie {

// Device allocation owned by a plan (freed on destruction).  Allocations are
// stream-ordered on the stream of the API call that makes them.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release();
  vie_status alloc(size_t n);
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

// Stream of this thread's stream-ordered allocations (DevBuf::alloc) and a
// scope that sets it; buffers are freed on the stream they were allocated on.
cudaStream_t alloc_stream();
void set_alloc_stream(cudaStream_t s);
struct AllocScope {
  cudaStream_t prev;
  explicit AllocScope(cudaStream_t s) : prev(alloc_stream()) { set_alloc_stream(s); }
  ~AllocScope() { set_alloc_stream(prev); }
};

// Matvec geometry passed to kernels.
struct MvDims {
  int nx, ny, nz;       // grid
  int L, Py, Pz;        // circulant embedding lengths
  int Lh, Pyh, Pzh;     // stored (non-negative) spectral octant: L/2+1, ...
};

// One partition box of the preconditioner with its factorised blocks.
struct BoxPrec {
  vie_box b{};
  int levels = 1;            // 1: 1-level circulant; 2: 2-level (blocks per (f_x, f_y))
  int m = 0;                 // 3 * ny * nz
  int n = 0;                 // nx of the box (circulant length)
  int nhalf = 0;             // frequencies 0..nhalf-1 carry stored blocks (S1 symmetry)
  int rep = 0;               // representative frequency ceil(n/2) - 1
  int nblk = 0;              // stored blocks: kept f <= n/2 plus the representative
  int nkept = 0;             // kept frequencies (full range 0..n-1)
  int ndisc = 0;             // discarded frequencies (use the representative)
  DevBuf Mt;                 // double2 [nz][ny] homogenised M~
  DevBuf lam;                // double2 [6][2nz-1][2ny-1][n] Chan eigenvalues
  DevBuf vhat;               // double  [n]
  DevBuf fmap;               // int [n]: block slot for f (S1 folded), -1 -> representative
  DevBuf fsgn;               // int [n]: 1 if f uses S D S (f > n/2)
  DevBuf disc;               // int [ndisc]: discarded frequencies
  DevBuf blkf;               // int [nblk]: frequency of each stored block
  DevBuf inv64;              // float2  [nblk][m][m] row-major D_f^{-1} (mixed path)
  DevBuf inv128;             // double2 [nblk][m][m] row-major D_f^{-1} (FP64 path)
  DevBuf rhat64, rhat128;    // [m][n] line-major spectra of the box unknowns
  DevBuf zhat64, zhat128;
  DevBuf tmp64, tmp128;      // transform scratch (Bluestein and/or long-line split)
  DevBuf bpack, apack;       // tensor-core operands of the representative-block product (packed tf32 hi/lo)
  int tc_n = 64;             // N tile of that product (64 or 32; set by the autotuner)
  int gemv_split[2] = {0, 0};  // kept-block product: CTAs per block, complex FP32 / FP64 (0: the default
                               // rule; set by the autotuner)
  const FftLen* fx = nullptr;
  // 2-level boxes: blocks of m2 = 3 nz rows for f <= n/2, g <= ny/2, slot
  // g * nfs + f, inverses column-major in inv64 / inv128; rhat/zhat [m2][ny][n]
  int m2 = 0, nfs = 0, ngs = 0;
  const FftLen* fy = nullptr;
};

struct Krylov;   // krylov.cu

}  // namespace vie

struct vie_plan_s {
  int nx = 0, ny = 0, nz = 0;
  double h = 0, k0 = 0, eps_bg = 1, kb = 0;
  vie_opts opts{};
  std::vector<vie_box> boxes;
  cudaStream_t st = nullptr;
  int device = 0;
  // second stream and events for the fork inside a preconditioner application
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  vie::MvDims d{};
  const vie::FftLen *fL = nullptr, *fPy = nullptr, *fPz = nullptr;
  bool fused_x128 = true, fused_x64 = true;   // fused x-pass fits shared memory
  // complex-FP32 x pass split over a cluster of Q CTAs (Q = 2, 4 or 8; xq is
  // the smallest Q whose lines fit shared memory, 1 = no split): each CTA
  // transforms every Q-th frequency of the three lines with length L / Q
  // (fLq[log2 Q - 1]) and the twiddles W_L^j, j < L (twL64)
  int xq = 1;
  const vie::FftLen* fLq[3] = {nullptr, nullptr, nullptr};
  vie::DevBuf twL64;
  // x-pass variant per precision [c64, c128] chosen by the autotuner (-1:
  // untuned, the default rule; 0: compile-time radix-16 kernel; k >= 1: the
  // generic Stockham kernel with radix order xord[.][k - 1])
  int xvar[2] = {-1, -1};
  vie::FftPlanDev xord[2][3]{};
  int yzxg = 0;                        // x-columns per CTA of the register yz passes (0: 16)
  int yzxg_gen = 0;                    // x-columns per CTA of the generic yz passes, complex FP32 (0: default rule)
  std::string tuning;                  // the autotuner's report (vie_plan_tuning)
  size_t tuning_matvec = 0;            // length of its matvec part (the rest belongs to the last build)
  vie::DevBuf spec128, spec64;         // [6][Pzh][Pyh][Lh] scaled generator spectra
  vie::DevBuf M128, M64;               // [nz][ny][nx] material M
  vie::DevBuf T128, T64;               // [3][Pz][Py][nx] matvec intermediate
  vie::DevBuf S128, S64;               // [3][Pz][Py][L] full x-spectrum (unfused path only)
  vie::DevBuf X128, X64;               // split scratch for x-lines longer than shared memory
  bool yz_split = false;               // Py*Pz > 4096: y and z transforms as separate line passes
  vie::DevBuf U128, U64;               // [3][nz][Py][nx] y-spectrum of the unpadded z rows (yz_split)
  vie::DevBuf xin64, xout64;           // c64 staging for vie_matvec / precond (mixed)
  vie::DevBuf dev_err;                 // int: set by a kernel whose bounded wait ran out
  vie::DevBuf h_eps, h_e, h_w;         // device staging of vie_solve_host (first call allocates)
  bool has_eps = false;
  bool prec_built = false;
  std::vector<std::unique_ptr<vie::BoxPrec>> bp;
  size_t precond_bytes = 0;
  long long precond_blocks = 0, precond_discarded = 0;
  double kept_fraction = 1.0;
  float t_setup_ms = 0;
  std::unique_ptr<vie::Krylov> kry;
  size_t bytes_allocated = 0;
  vie_plan_s();
  ~vie_plan_s();
};

namespace vie {

long long launches_total();
long long launches_thread();   // launches counted by the calling thread

// greens.cu
vie_status build_spectra(vie_plan_s* P);
vie_status set_material(vie_plan_s* P, const double2* eps);

// matvec.cu
template <class C>
vie_status matvec(vie_plan_s* P, const C* x, C* y, const C* Mv, const C* spec, C* T, C* S, cudaStream_t st);
vie_status matvec_alloc(vie_plan_s* P);
template <class C>
vie_status xpass(vie_plan_s* P, const C* spec, C* T, C* S, int variant, cudaStream_t st);
// both register yz passes (complex FP32) with xg x-columns per CTA on the
// plan's staging buffers (autotuner timing); VIE_EINVAL if the cross-section
// has no register variant
vie_status yz_pair(vie_plan_s* P, int xg, cudaStream_t st);
// both generic yz passes (complex FP32, shared-memory Stockham) with xg
// x-columns per CTA on the plan's staging buffers; VIE_EINVAL if the plan
// takes the register or the split-line passes, or xg columns do not fit
vie_status yz_pair_generic(vie_plan_s* P, int xg, cudaStream_t st);

// tune.cu: per-shape choice among launch variants, by timing on the plan's
// own buffers (cached per process and shape)
using TuneKey = std::tuple<int, int, int, int, int>;   // kernel, precision, shape...
bool tune_cache_get(const TuneKey& k, int* choice, std::string* report);
void tune_cache_put(const TuneKey& k, int choice, const std::string& report);
vie_status tune_matvec(vie_plan_s* P);
bool autotune_enabled();
// device time of one call of f on stream st: after one warm-up call, the
// least of three trials of reps back-to-back calls (a trial another stream's
// work slowed down does not decide)
template <class F>
inline vie_status time_ms(cudaStream_t st, int reps, F f, float* ms) {
  cudaEvent_t e0, e1;
  VIE_CUDA(cudaEventCreate(&e0));
  VIE_CUDA(cudaEventCreate(&e1));
  vie_status s = f();
  *ms = 0;
  for (int trial = 0; trial < 3 && s >= 0; ++trial) {
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && s >= 0; ++r) s = f();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    t /= (float)reps;
    if (trial == 0 || t < *ms) *ms = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}


// precond.cu
vie_status precond_build(vie_plan_s* P);
template <class C>
vie_status precond_apply(vie_plan_s* P, const C* r, C* z, cudaStream_t st);
void precond_free(vie_plan_s* P);
vie_status precond_add_fp64(vie_plan_s* P);
vie_status precond_set_rep_tile(vie_plan_s* P, int tn);
// x-embedding length of nx points and the cluster split of its complex-FP32
// x pass (1, 2 or 4)
int embed_x(int nx, int* q);
vie_status box_homogenise(vie_plan_s* P, const vie_box& b, DevBuf& Mt, bool plane);
vie_status factor_invert_blocks(vie_plan_s* P, DevBuf& LU, int m, int nblk, bool want64, DevBuf* inv64, bool want128,
                                DevBuf* inv128);

// precond2.cu (2-level boxes)
vie_status build_box2(vie_plan_s* P, BoxPrec& B, bool want64, bool want128);
template <class C>
vie_status apply_box2(vie_plan_s* P, BoxPrec& B, const C* r, C* z, C* inv, C* rh, C* zh, C* tmp, cudaStream_t st);

// krylov.cu
vie_status solve(vie_plan_s* P, const double2* e_inc, double2* w, vie_info* info);
vie_status solve_many(vie_plan_s* const* P, int n, const double2* const* e_inc, double2* const* w_out,
                      vie_info* info, vie_status* status, cudaStream_t st);
void krylov_free(vie_plan_s* P);
void reset_graphs(vie_plan_s* P);
// resumable solves ("runs") and the lockstep driver, for the server
struct Run;
struct Lockstep;
Run* run_new(vie_plan_s* P, const double2* e_inc, double2* w_out, vie_info* info);
void run_delete(Run* R);
vie_status run_start(Run* R);          // right-hand side, preconditioner, first cycle (plan stream)
bool run_finished(const Run* R);
void run_abort(Run* R, const char* why);   // mark a run failed
vie_status run_status(const Run* R, std::string* err);
vie_plan_s* run_plan(const Run* R);
Lockstep* lockstep_new();
void lockstep_free(Lockstep* L);
void lockstep_release(Lockstep* L);    // frees its device buffers, streams and graph
bool lockstep_pass(Lockstep* L, std::vector<Run*>& runs, cudaStream_t st);

// conversions
vie_status widen(const float2* a, double2* b, long long n, cudaStream_t st);
vie_status narrow(const double2* a, float2* b, long long n, cudaStream_t st);

}  // namespace vie
