// Right-preconditioned restarted GMRES (the Krylov solver of Sec. 1 / Sec. 3)
// and FP64 iterative refinement around a complex-FP32 inner GMRES.
//
// One Arnoldi step with classical Gram-Schmidt and one re-orthogonalisation
// (CGS2): z = P^-1 v_j, w = A z, h = V^H w, w -= V h (twice), h_{j+1,j} =
// ||w||, v_{j+1} = w / h_{j+1,j}.  The Hessenberg column is reduced by complex
// Givens rotations on the device; |g_{j+1}| is the residual estimate.  All
// reductions are two-stage and fixed-order, so results are bitwise
// reproducible for a given size and launch shape.
//
// The iteration index j, the rotations and the stop flag live in device
// memory; one captured CUDA graph replays a whole Arnoldi step, and the host
// only polls the stop flag between chunks of steps.
#include <math.h>

#include <cmath>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

#include "internal.h"
#include "prof.h"

namespace vie {

constexpr int RMAX = 128;      // largest supported restart length
constexpr int NPART = 152;     // CTAs of the reduction kernels (one 1024-thread block per SM)
constexpr int RED_THREADS = 1024;

constexpr int PST = 2 * (RMAX + 1);   // per-block stride of the reduction partials

struct GmresDev {
  double2 H[(RMAX + 1) * RMAX];   // column j at H[j*(RMAX+1) + i], after rotations
  double2 Hr[(RMAX + 1) * RMAX];  // the same columns before rotations (Arnoldi relation)
  double cs[RMAX];
  double2 sn[RMAX];
  double2 g[RMAX + 1];
  double2 y[RMAX];
  double2 cs_s[RMAX + 1];         // update coefficients of the current step: s (re-orthogonalisation
  double2 cs_c[RMAX + 1];         //   of u_j) and c (projection of w)
  double2 cu;                     // coefficient of u_j in the projection of w
  double inv_beta;                // 1 / ||u_j - Q s||
  double nu;                      // ||w''|| of the last update: h_{j,j-1} before its correction
  double beta;                    // norm of the cycle's starting residual
  double tol_abs;                 // stop when |g_k| <= tol_abs
  double hnext;                   // scale of the next basis vector
  double inv_next;                // 1 / hnext, in FP64 ...
  float inv_next32;               // ... and rounded to FP32 (read by the scaling without FP64 work)
  double resest;                  // |g_k|
  int j;                          // current step
  int k;                          // final columns of the finished cycle
  int done;                       // 1: cycle finished (converged, full, or breakdown)
  int restart;
  int iters;                      // Arnoldi columns formed by this state
  int reorth;                     // unused (kept for the layout of older callers)
  int reorths;                    // re-orthogonalised vectors
  int arrive_dot;                 // arrival counters of the fused grid reductions
  int arrive_upd;
  int pad[3];
};

struct Lockstep;
void lockstep_free(Lockstep* L);
struct LockstepDeleter { void operator()(Lockstep* L) const { lockstep_free(L); } };

struct Krylov {
  int restart = 0;
  int rs64 = 0, rs128 = 0;        // restart lengths of the complex-FP32 and FP64 cycles
  long long n3 = 0;
  long long ld = 0;               // column stride of the basis (n3 rounded up to 32)
  DevBuf V64, V128;               // (restart + 1) * ld basis
  DevBuf u64, u128, z64, z128, w64, w128;
  DevBuf partial;                 // double2 [NPART][PST] (norms of the cycle and refinement steps)
  DevBuf p1, p2;                  // Arnoldi partials: dot [PST][NPART], norm [NPART] (accumulator precision)
  DevBuf red;                     // [PST] the dot partials summed over the CTAs
  DevBuf arn64, arn128;           // one ArnPlan descriptor per precision (device)
  int nparts = 0;                 // CTAs of the plan in the Arnoldi launches
  DevBuf state;                   // GmresDev
  DevBuf x128, r128, b128, d64, rhs64, r64, t128;
  DevBuf xbest;                   // best iterate of a multi-cycle (FP64) solve
  DevBuf scal;                    // double [8]: norms
  int* hflag = nullptr;           // pinned host mirror: done, iters
  std::unique_ptr<Lockstep, LockstepDeleter> lock;  // step graph of this plan's own solves
  cudaEvent_t ev = nullptr;
  cudaStream_t cap = nullptr;     // private stream for graph capture
  cudaStream_t side = nullptr;    // second stream of a step (Hessenberg bookkeeping)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  ~Krylov() {
    if (cap) cudaStreamDestroy(cap);
    if (side) cudaStreamDestroy(side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev) cudaEventDestroy(ev);
    if (hflag) cudaFreeHost(hflag);
  }
};

void krylov_free(vie_plan_s* P) { P->kry.reset(); }

}  // namespace vie

vie_plan_s::vie_plan_s() = default;
vie_plan_s::~vie_plan_s() {
  if (side) cudaStreamDestroy(side);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
}

namespace vie {

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <class C> struct Acc;   // per-thread accumulator type
template <> struct Acc<float2> { using T = float; };
template <> struct Acc<double2> { using T = double; };

__device__ __forceinline__ double2 block_sum2(double2 v, double2* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double2 t = make_double2(0, 0);
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t.x += sh[w].x; t.y += sh[w].y; }
  return t;   // valid in thread 0
}

// sum of partial[b][i] over b by one warp, reading through L2 (the partials
// were just written by other blocks); fixed order: lane-strided sums, then a
// butterfly
__device__ __forceinline__ double2 warp_sum_partials_cg(const double2* __restrict__ partial, int nparts, int i) {
  const int lane = threadIdx.x & 31;
  double2 t = make_double2(0, 0);
#pragma unroll 4
  for (int b = lane; b < nparts; b += 32) {
    const double2 p = __ldcg(partial + (long long)b * PST + i);
    t.x += p.x;
    t.y += p.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
    t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
  }
  return t;
}

// Called by every thread of a block after it wrote its partials: returns
// true in the last block to arrive (which then owns the grid reduction) and
// resets the counter there.
__device__ __forceinline__ bool last_block(int* counter) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (is_last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0;
  }
  return is_last;
}

// As last_block, for the n CTAs of one plan in a launch over a work-list.
__device__ __forceinline__ bool last_block_of(int* counter, int n) {
  __shared__ int is_last_of;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last_of = (atomicAdd(counter, 1) == n - 1);
  __syncthreads();
  if (is_last_of) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0;
  }
  return is_last_of;
}

// As givens_column, run by one warp (lane 0 takes the sequential chain), so
// that the rest of the block can work meanwhile.  The arithmetic is in T: the
// complex-FP32 solve rotates its FP32-accurate Hessenberg entries in FP32
// (FP64 issues at a small fraction of the FP32 rate on this part, and the
// chain is sequential); the matrix, rotations and residual estimate are
// stored in FP64 either way.
template <class T>
__device__ void givens_column_warp(GmresDev* __restrict__ s, int jc) {
  using CT = typename cplx_of<T>::type;
  __shared__ CT colw[RMAX + 1];
  __shared__ T csw[RMAX];
  __shared__ CT snw[RMAX];
  const int lane = threadIdx.x & 31;
  const double2* hr = s->Hr + (long long)jc * (RMAX + 1);
  for (int i = lane; i <= jc + 1; i += 32) colw[i] = cconv<CT>(hr[i]);
  for (int i = lane; i < jc; i += 32) { csw[i] = (T)s->cs[i]; snw[i] = cconv<CT>(s->sn[i]); }
  __syncwarp();
  if (lane == 0) {
    // the rotated row i + 1 is carried in registers (the chain's only
    // dependency); rows i + 1 of the input and the rotations are read ahead
    CT a = colw[0];
#pragma unroll 4
    for (int i = 0; i < jc; ++i) {
      const CT b = colw[i + 1];
      const T c = csw[i];
      const CT sn = snw[i];
      colw[i] = cmake<CT>(c * a.x + (sn.x * b.x - sn.y * b.y), c * a.y + (sn.x * b.y + sn.y * b.x));
      a = cmake<CT>(-(sn.x * a.x + sn.y * a.y) + c * b.x, -(sn.x * a.y - sn.y * a.x) + c * b.y);
    }
    const CT bb = colw[jc + 1];
    const T b = sqrt(bb.x * bb.x + bb.y * bb.y);
    T c;
    CT sn;
    const T aa = sqrt(a.x * a.x + a.y * a.y);
    if (b == (T)0) { c = 1; sn = cmake<CT>(0, 0); }
    else if (aa == (T)0) { c = 0; sn = cmake<CT>(1, 0); }
    else {
      const T r = hypot(aa, b);
      c = aa / r;
      sn = cmake<CT>(a.x * b / (aa * r), a.y * b / (aa * r));
    }
    s->cs[jc] = (double)c;
    s->sn[jc] = make_double2((double)sn.x, (double)sn.y);
    colw[jc] = cmake<CT>(c * a.x + sn.x * b, c * a.y + sn.y * b);
    colw[jc + 1] = cmake<CT>(0, 0);
    const CT gj = cconv<CT>(s->g[jc]);
    const CT g1 = cmake<CT>(-(sn.x * gj.x + sn.y * gj.y), -(sn.x * gj.y - sn.y * gj.x));
    s->g[jc + 1] = make_double2((double)g1.x, (double)g1.y);
    s->g[jc] = make_double2((double)(c * gj.x), (double)(c * gj.y));
    s->resest = (double)sqrt(g1.x * g1.x + g1.y * g1.y);
  }
  __syncwarp();
  double2* H = s->H + (long long)jc * (RMAX + 1);
  for (int i = lane; i <= jc + 1; i += 32) H[i] = make_double2((double)colw[i].x, (double)colw[i].y);
}

// Rotations for the final raw column jc (rows 0..jc+1 in Hr): apply the
// earlier rotations, form rotation jc, update g and the residual estimate,
// store the rotated column in H.  Run by one whole block.
__device__ void givens_column(GmresDev* __restrict__ s, int jc) {
  __shared__ double2 col[RMAX + 1];
  __shared__ double csv[RMAX];
  __shared__ double2 snv[RMAX];
  const double2* hr = s->Hr + (long long)jc * (RMAX + 1);
  for (int i = threadIdx.x; i <= jc + 1; i += blockDim.x) col[i] = hr[i];
  for (int i = threadIdx.x; i < jc; i += blockDim.x) { csv[i] = s->cs[i]; snv[i] = s->sn[i]; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < jc; ++i) {
      const double2 a = col[i], b = col[i + 1];
      const double c = csv[i];
      const double2 sn = snv[i];
      // [c s; -conj(s) c] [a; b]
      col[i] = make_double2(c * a.x + (sn.x * b.x - sn.y * b.y), c * a.y + (sn.x * b.y + sn.y * b.x));
      col[i + 1] = make_double2(-(sn.x * a.x + sn.y * a.y) + c * b.x, -(sn.x * a.y - sn.y * a.x) + c * b.y);
    }
    const double2 a = col[jc];
    const double2 bb = col[jc + 1];
    const double b = sqrt(bb.x * bb.x + bb.y * bb.y);   // the subdiagonal is real and >= 0
    double c;
    double2 sn;
    const double aa = sqrt(a.x * a.x + a.y * a.y);
    if (b == 0.0) { c = 1.0; sn = make_double2(0, 0); }
    else if (aa == 0.0) { c = 0.0; sn = make_double2(1.0, 0.0); }
    else {
      const double r = hypot(aa, b);
      c = aa / r;
      // s = a conj(b) / (|a| r), b real
      sn = make_double2(a.x * b / (aa * r), a.y * b / (aa * r));
    }
    s->cs[jc] = c;
    s->sn[jc] = sn;
    col[jc] = make_double2(c * a.x + sn.x * b, c * a.y + sn.y * b);
    col[jc + 1] = make_double2(0, 0);
    const double2 gj = s->g[jc];
    // g_{jc+1} = -conj(s) g_jc ; g_jc = c g_jc
    const double2 g1 = make_double2(-(sn.x * gj.x + sn.y * gj.y), -(sn.x * gj.y - sn.y * gj.x));
    s->g[jc + 1] = g1;
    s->g[jc] = make_double2(c * gj.x, c * gj.y);
    s->resest = sqrt(g1.x * g1.x + g1.y * g1.y);
  }
  __syncthreads();
  double2* H = s->H + (long long)jc * (RMAX + 1);
  for (int i = threadIdx.x; i <= jc + 1; i += blockDim.x) H[i] = col[i];
  __syncthreads();
}

// sum of partial[b][i] over b by one warp (fixed order: lane-strided sums,
// then a butterfly)
__device__ __forceinline__ double2 warp_sum_partials(const double2* __restrict__ partial, int nparts, int i) {
  const int lane = threadIdx.x & 31;
  double2 t = make_double2(0, 0);
  for (int b = lane; b < nparts; b += 32) {
    const double2 p = partial[(long long)b * PST + i];
    t.x += p.x;
    t.y += p.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
    t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
  }
  return t;
}


// ---------------------------------------------------------------------------
// Arnoldi step kernels over a work-list of plans.
//
// One launch of each kernel serves every plan of a batch: plan p owns the
// CTAs [part0_p, part0_p + nparts_p) of the grid, and each of those CTAs a
// contiguous range of the plan's vectors (columns of stride ld, a multiple of
// 32 elements).  A CTA cuts its range into sub-chunks of ARN_SUB bytes per
// column; per sub-chunk a thread visits the same KPT elements of w, u_j = V_j
// and V_0 .. V_{j-1}, four columns at a time, and issues the loads of the next
// four columns before it reduces the current ones, so that two groups of
// loads are in flight per thread.  (A variant that streamed the columns
// through a ring of shared-memory tiles with cp.async.bulk is described with
// the concurrency finding of the design notes; the direct coalesced loads are
// as fast here.)
//
// The serial work between the passes is small: the dot pass writes per-CTA
// partials and the plan's last CTA sums them (fixed order) into one vector
// of dots; every CTA of the update pass derives the same coefficients from
// it; one CTA per plan, on a second stream beside the update, keeps the
// Hessenberg matrix and the Givens rotations; one CTA per plan at the step end
// sums the norm partials (fixed order) and advances the step index.  The
// new direction w'' is left unnormalised in u
// (the input of the next step's preconditioner); the step kernels scale u
// and w = A P^-1 u by 1 / ||w''|| as they load them, so no pass rewrites the
// vector after its norm is known.
// ---------------------------------------------------------------------------
constexpr int ARN_SUB = 16384;                  // bytes of one column per sub-chunk
constexpr int ARN_THREADS = 512;                // streaming threads of the dot and update passes
constexpr int STEP_END_THREADS = 128;

// The vectors of one plan for the step kernels.
template <class C>
struct ArnPlan {
  C* V;            // basis: restart + 1 columns of stride ld
  C* w;            // A P^-1 u_j, scaled by 1 / ||u_j|| (the GmresDev field inv_next)
  C* u;            // u_j, unnormalised (w'' of step j - 1): input of P^-1; the update pass
                   // writes w'' there
  GmresDev* s;     // GMRES state of the plan
  C* p1;           // [PST][NPART] dot partials (accumulator precision): row v, part b at v * NPART + b
  C* p2;           // [nparts] partials of ||w''||^2 (real part)
  C* red;          // [PST] the plan's sums of the dot partials (s_i / alpha, z_i / zeta)
  long long ld;
  int n3;
  int part0;       // first CTA of the plan in a launch over the work-list
  int nparts;      // CTAs of the plan
  int pad;
};

// CTAs per plan: one per 2048 elements of the vector, at most NPART (one wave
// of one CTA per SM).  A function of n3 alone, so a plan's reductions run in
// the same order whether it is solved alone or in a batch.
inline int arn_parts(long long n3) {
  return (int)std::min<long long>(NPART, std::max<long long>(1, (n3 + 2047) / 2048));
}

// the plan of this CTA (descriptors sorted by part0) and the CTA's part in it
template <class C>
__device__ __forceinline__ const ArnPlan<C>* arn_find(const ArnPlan<C>* __restrict__ D, int nd, int& part) {
  int lo = 0, hi = nd - 1;
  const int b = (int)blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (D[mid].part0 <= b) lo = mid;
    else hi = mid - 1;
  }
  part = b - D[lo].part0;
  return D + lo;
}

struct ArnRange {
  int c0, c1;   // the CTA's element range
  int nsub, sc; // sub-chunks and elements per sub-chunk (multiple of 32)
};

// (32-bit arithmetic: vectors hold fewer than 2^31 elements, checked at plan
// creation, and a 64-bit division would run as an FP64 subroutine)
template <class C>
__device__ __forceinline__ ArnRange arn_range(int n3, int nparts, int part) {
  const unsigned n = (unsigned)n3;
  const unsigned per = ((n + nparts - 1) / (unsigned)nparts + 31) / 32 * 32;
  ArnRange g;
  const unsigned c0 = min(n, (unsigned)part * per), c1 = min(n, c0 + per);
  g.c0 = (int)c0;
  g.c1 = (int)c1;
  const unsigned maxe = ARN_SUB / (unsigned)sizeof(C);
  const unsigned len = c1 - c0;
  g.nsub = (int)((len + maxe - 1) / maxe);
  g.sc = g.nsub > 0 ? (int)(((len + (unsigned)g.nsub - 1) / (unsigned)g.nsub + 31) / 32 * 32) : 0;
  return g;
}

// elements q of columns i0 .. i0 + nt - 1 (nt <= 4) of the sub-chunk at start
template <class C, int KPT>
__device__ __forceinline__ void arn_load4(C (&v)[4][KPT], const C* __restrict__ V, long long ld, long long start,
                                          int i0, int nt, int ct, int cnt) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const C* col = V + (long long)(i0 + t) * ld + start;
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const int e = ct + q * ARN_THREADS;
      v[t][q] = (t < nt && e < cnt) ? col[e] : czero<C>();
    }
  }
}

// the dots of four columns with u_j and w, reduced over the warp into its row
template <class C, class T, int KPT>
__device__ __forceinline__ void arn_dot4(const C (&v)[4][KPT], const C (&xu)[KPT], const C (&xw)[KPT], T* my, int i0,
                                         int nt, int lane) {
  T a[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) a[q] = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      a[4 * t + 0] += v[t][q].x * xu[q].x + v[t][q].y * xu[q].y;
      a[4 * t + 1] += v[t][q].x * xu[q].y - v[t][q].y * xu[q].x;
      a[4 * t + 2] += v[t][q].x * xw[q].x + v[t][q].y * xw[q].y;
      a[4 * t + 3] += v[t][q].x * xw[q].y - v[t][q].y * xw[q].x;
    }
  const T r = warp_reduce16<T>(a, lane);
  const int qq = lane >> 1, col = i0 + (qq >> 2), part = qq & 3;
  if ((lane & 1) == 0 && (qq >> 2) < nt) my[(part < 2 ? 0 : 2 * (RMAX + 1)) + 2 * col + (part & 1)] += r;
  __syncwarp();
}

// columns top, top - 1, .., top - nt + 1 (nt <= 4), for the update's
// descending sweep
template <class C, int KPT>
__device__ __forceinline__ void arn_load4r(C (&v)[4][KPT], const C* __restrict__ V, long long ld, long long start,
                                           int top, int nt, int ct, int cnt) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const C* col = V + (long long)(top - t) * ld + start;
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const int e = ct + q * ARN_THREADS;
      v[t][q] = (t < nt && e < cnt) ? col[e] : czero<C>();
    }
  }
}

// the update of four columns: as += s_i V_i, ac += c_i V_i
template <class C, int KPT>
__device__ __forceinline__ void arn_axpy4(const C (&v)[4][KPT], const C* sco, const C* cco, C (&as)[KPT],
                                          C (&ac)[KPT], int top, int nt) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const C hs = t < nt ? sco[top - t] : czero<C>(), hc = t < nt ? cco[top - t] : czero<C>();
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      cfma(as[q], hs, v[t][q]);
      cfma(ac[q], hc, v[t][q]);
    }
  }
}

// Sum the dot partials of a plan over its CTAs, in a fixed order (lane-
// strided, then a butterfly): sv[i] = s_i (alpha at i = j), zv[i] = z_i (zeta
// at i = j), one warp per row, RB rows of loads in flight per warp.  The
// order of one row's sum does not depend on RB or on the number of warps.
template <class C, int RB>
__device__ __forceinline__ void arn_reduce_dots(const C* __restrict__ p1, int np, int j, C* __restrict__ sv,
                                                C* __restrict__ zv) {
  constexpr int NPL = (NPART + 31) / 32;   // partials per lane
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i0 = warp * RB; i0 <= j; i0 += nw * RB) {
    C pa[RB][NPL], pz[RB][NPL];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
      for (int q = 0; q < NPL; ++q) {
        const int bk = lane + 32 * q, i = i0 + r;
        const bool ok = bk < np && i <= j;
        pa[r][q] = ok ? __ldcg(p1 + (long long)i * NPART + bk) : czero<C>();
        pz[r][q] = ok ? __ldcg(p1 + (long long)(RMAX + 1 + i) * NPART + bk) : czero<C>();
      }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      C a = czero<C>(), b = czero<C>();
#pragma unroll
      for (int q = 0; q < NPL; ++q) { a.x += pa[r][q].x; a.y += pa[r][q].y; b.x += pz[r][q].x; b.y += pz[r][q].y; }
      for (int o = 16; o > 0; o >>= 1) {
        a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
        a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
        b.x += __shfl_xor_sync(0xffffffffu, b.x, o);
        b.y += __shfl_xor_sync(0xffffffffu, b.y, o);
      }
      if (lane == 0 && i0 + r <= j) { sv[i0 + r] = a; zv[i0 + r] = b; }
    }
  }
}

// Delayed classical Gram-Schmidt with re-orthogonalisation (one global
// reduction and one update per Arnoldi step).  Step j enters with Q = [q_0 ..
// q_{j-1}] final and u_j = V_j, which step j-1 orthogonalised once and scaled
// by nu = ||w''||, and with w = A P^{-1} u_j.  One pass over the basis gives
//   s = Q^H u_j, alpha = u_j^H u_j, z = Q^H w, zeta = u_j^H w;
// then q_j = (u_j - Q s) / beta with beta^2 = alpha - |s|^2, the previous
// column is final (h_{:,j-1} += nu s, h_{j,j-1} = nu beta), and, writing
// t = (zeta - s^H z) / beta, the projection of A P^{-1} q_j is
//   h_{:,j} = ([z; t] - H_{0:j,0:j-1} s) / beta,
//   w'' = (w - Q (z - s t / beta) - u_j t / beta) / beta,
// by the Arnoldi relation A P^{-1} Q = Q_{j+1} H.  The update pass forms q_j
// and w'' together; u_{j+1} = w'' / ||w''|| is orthogonalised again (its s)
// at step j + 1.  Column j thus becomes final one step later, so the
// residual estimate lags by one step; at restart length a last reduction
// (step j = restart) only finalises the last column.
//
// Dot pass: per CTA the partials [i] = (s_i, or alpha at i = j) and
// [RMAX + 1 + i] = (z_i, or zeta at i = j), summed over the CTA's warps.
template <class C>
__global__ void __launch_bounds__(ARN_THREADS) k_arn_dot(const ArnPlan<C>* __restrict__ D, int nd) {
  using T = typename Acc<C>::T;
  constexpr int KPT = ARN_SUB / (int)sizeof(C) / ARN_THREADS;   // elements per thread per sub-chunk
  constexpr int ROW = 4 * (RMAX + 1) + 4;                       // per warp: s (2 per column), z (2), alpha, zeta
  extern __shared__ __align__(16) unsigned char dot_smem[];
  T* wsum = reinterpret_cast<T*>(dot_smem);                     // [ARN_THREADS / 32][ROW]
  int part;
  const ArnPlan<C>* dp = arn_find(D, nd, part);
  const GmresDev* s = dp->s;
  if (s->done) return;
  const int j = s->j;
  const C* __restrict__ V = dp->V;
  const C* __restrict__ w = dp->w;
  const C* __restrict__ u = dp->u;
  // u holds u_j unnormalised (w'' of the previous step) and w = A P^-1 of it:
  // both are scaled by rho = 1 / ||w''|| as they are loaded
  using R = typename real_of<C>::type;
  const R rho = sizeof(R) == 4 ? (R)s->inv_next32 : (R)s->inv_next;
  const long long ld = dp->ld;
  const ArnRange g = arn_range<C>(dp->n3, dp->nparts, part);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ct = threadIdx.x;
  T* my = wsum + (size_t)warp * ROW;
  for (int i = lane; i < ROW; i += 32) my[i] = 0;
  __syncwarp();
  T al = 0, zr = 0, zi = 0;
  for (int sb = 0; sb < g.nsub; ++sb) {
    const long long start = g.c0 + (long long)sb * g.sc;
    const int cnt = min(g.sc, g.c1 - (int)start);
    const C* wv = w + start;
    const C* uv = u + start;
    C xw[KPT], xu[KPT];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const int e = ct + q * ARN_THREADS;
      xw[q] = e < cnt ? cscale(wv[e], rho) : czero<C>();
      xu[q] = e < cnt ? cscale(uv[e], rho) : czero<C>();
    }
    C va[4][KPT], vb[4][KPT];
    if (j > 0) arn_load4<C, KPT>(va, V, ld, start, 0, min(4, j), ct, cnt);
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      al += xu[q].x * xu[q].x + xu[q].y * xu[q].y;
      zr += xu[q].x * xw[q].x + xu[q].y * xw[q].y;
      zi += xu[q].x * xw[q].y - xu[q].y * xw[q].x;
    }
    for (int i0 = 0; i0 < j; i0 += 8) {
      const int n1 = min(4, j - i0 - 4), n2 = min(4, j - i0 - 8);
      if (n1 > 0) arn_load4<C, KPT>(vb, V, ld, start, i0 + 4, n1, ct, cnt);
      arn_dot4<C, T, KPT>(va, xu, xw, my, i0, min(4, j - i0), lane);
      if (n2 > 0) arn_load4<C, KPT>(va, V, ld, start, i0 + 8, n2, ct, cnt);
      if (n1 > 0) arn_dot4<C, T, KPT>(vb, xu, xw, my, i0 + 4, n1, lane);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    zr += __shfl_xor_sync(0xffffffffu, zr, o);
    zi += __shfl_xor_sync(0xffffffffu, zi, o);
  }
  if (lane == 0) { my[4 * (RMAX + 1)] = al; my[4 * (RMAX + 1) + 1] = zr; my[4 * (RMAX + 1) + 2] = zi; }
  __syncthreads();
  // block sums over the warps, in the accumulator precision (FP32 for a
  // complex-FP32 basis; FP64 issues at a small fraction of the FP32 rate here)
  C* pb = dp->p1 + part;   // row v at pb[v * NPART]
  for (int v = threadIdx.x; v < 2 * (j + 1); v += blockDim.x) {
    // v < j: s_v; v == j: alpha; v = j + 1 + i: z_i; v = 2 j + 1: zeta
    int sr, si, dst;
    if (v < j) { sr = 2 * v; si = sr + 1; dst = v; }
    else if (v == j) { sr = 4 * (RMAX + 1); si = -1; dst = j; }
    else if (v < 2 * j + 1) { sr = 2 * (RMAX + 1) + 2 * (v - j - 1); si = sr + 1; dst = RMAX + 1 + (v - j - 1); }
    else { sr = 4 * (RMAX + 1) + 1; si = sr + 1; dst = RMAX + 1 + j; }
    T re = 0, im = 0;
    for (int w2 = 0; w2 < ARN_THREADS / 32; ++w2) {
      re += wsum[(size_t)w2 * ROW + sr];
      if (si >= 0) im += wsum[(size_t)w2 * ROW + si];
    }
    pb[(long long)dst * NPART] = cmake<C>(re, im);
  }
  // the plan's last CTA to finish sums the partials over the CTAs, in a
  // fixed order, once for all readers (update pass, Hessenberg bookkeeping)
  GmresDev* sm = const_cast<GmresDev*>(s);
  if (!last_block_of(&sm->arrive_dot, dp->nparts)) return;
  arn_reduce_dots<C, sizeof(C) == 8 ? 4 : 2>(dp->p1, dp->nparts, j, dp->red, dp->red + RMAX + 1);
}

// the plan's reduced dots (written by the last CTA of the dot pass) into
// shared memory
template <class C>
__device__ __forceinline__ void arn_load_dots(const C* __restrict__ red, int j, C* sv, C* zv) {
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    sv[i] = __ldcg(red + i);
    zv[i] = __ldcg(red + RMAX + 1 + i);
  }
}

// beta = sqrt(alpha - |s|^2) (warp 0) and t = (zeta - s^H z) / beta (warp 1)
// from the reduced dots; valid in every thread after the call
template <class C, class T>
__device__ __forceinline__ void arn_beta_t(const C* sv, const C* zv, int j, T& beta, C& t) {
  __shared__ T sc_beta, sc_t[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp == 0) {
    T ss = 0;
    for (int i = lane; i < j; i += 32) ss += sv[i].x * sv[i].x + sv[i].y * sv[i].y;
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    // u_j is already orthogonal to Q up to rounding, so |s|^2 << alpha
    if (lane == 0) sc_beta = sqrt(fmax(sv[j].x - ss, (T)1e-12 * sv[j].x));
  } else if (warp == 1) {
    T tr = 0, ti = 0;
    for (int i = lane; i < j; i += 32) {
      tr += sv[i].x * zv[i].x + sv[i].y * zv[i].y;
      ti += sv[i].x * zv[i].y - sv[i].y * zv[i].x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      tr += __shfl_xor_sync(0xffffffffu, tr, o);
      ti += __shfl_xor_sync(0xffffffffu, ti, o);
    }
    if (lane == 0) { sc_t[0] = zv[j].x - tr; sc_t[1] = zv[j].y - ti; }
  }
  __syncthreads();
  beta = sc_beta;
  const T ib = (T)1 / beta;
  t = cmake<C>(sc_t[0] * ib, sc_t[1] * ib);
}

// Hessenberg bookkeeping of step j, one CTA per plan, launched on a second
// stream beside the update pass (both only read the dot partials): the
// previous column becomes final (h_{:,j-1} += nu s, h_{j,j-1} = nu beta), the
// tentative column j = ([z; t] - H_{0:j,0:j-1} s) / beta, then the rotation of
// column j - 1 and the stop test on the residual estimate it gives.
// (4 warps of at most 96 registers: what an SM has left beside one update CTA)
constexpr int HESS_THREADS = 128;
template <class C>
__global__ void __maxnreg__(96) k_arn_hess(const ArnPlan<C>* __restrict__ D) {
  using T = typename Acc<C>::T;
  constexpr int RPL = (RMAX + 1 + 31) / 32;   // rows per lane
  constexpr int NW = HESS_THREADS / 32;
  __shared__ C sv[RMAX + 1], zv[RMAX + 1];
  __shared__ T hsum[NW][2][RMAX + 1];
  const ArnPlan<C>* dp = D + blockIdx.x;
  GmresDev* s = dp->s;
  if (s->done) return;
  const int j = s->j;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  arn_load_dots<C>(dp->red, j, sv, zv);
  __syncthreads();
  T beta;
  C t;
  arn_beta_t<C, T>(sv, zv, j, beta, t);
  const T ib = (T)1 / beta;
  if (j > 0) {
    const double nu = s->nu;
    double2* hp = s->Hr + (long long)(j - 1) * (RMAX + 1);
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      hp[i].x += nu * (double)sv[i].x;
      hp[i].y += nu * (double)sv[i].y;
    }
    if (threadIdx.x == 0) hp[j] = make_double2(nu * (double)beta, 0.0);
  }
  __syncthreads();
  // at j = restart only column j - 1 is finalised (column j is never used and
  // has no slot when restart = RMAX)
  if (j < s->restart) {
    // H_{0:j,0:j-1} s: warp w takes the columns l = w (mod NW) with coalesced
    // column loads (lanes over rows; H[r][l] = 0 for r > l + 1), then the
    // warps' sums are added in a fixed order
    T ar[RPL], ai[RPL];
#pragma unroll
    for (int k = 0; k < RPL; ++k) { ar[k] = 0; ai[k] = 0; }
#pragma unroll 4
    for (int l = warp; l < j; l += NW) {
      const double2* hc = s->Hr + (long long)l * (RMAX + 1);
      const C sl = sv[l];
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        const int r = lane + 32 * k;
        if (r <= min(l + 1, j)) {
          const double2 hd = hc[r];
          const T hx = (T)hd.x, hy = (T)hd.y;
          ar[k] += hx * sl.x - hy * sl.y;
          ai[k] += hx * sl.y + hy * sl.x;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int r = lane + 32 * k;
      if (r <= RMAX) { hsum[warp][0][r] = ar[k]; hsum[warp][1][r] = ai[k]; }
    }
    __syncthreads();
    double2* hj = s->Hr + (long long)j * (RMAX + 1);
    for (int r = threadIdx.x; r <= j; r += blockDim.x) {
      T sr = 0, si = 0;
      for (int w2 = 0; w2 < NW; ++w2) { sr += hsum[w2][0][r]; si += hsum[w2][1][r]; }
      const C zr = r < j ? zv[r] : t;
      hj[r] = make_double2((double)((zr.x - sr) * ib), (double)((zr.y - si) * ib));
    }
  }
  __syncthreads();
  if (j == 0 || warp != 0) return;
  givens_column_warp<T>(s, j - 1);
  if (lane == 0) {
    s->k = j;
    s->reorths += 1;
    if (s->resest <= s->tol_abs || j >= s->restart) s->done = 1;
  }
}

// Update pass: every CTA sums its plan's dot partials (s, z, alpha, zeta),
// forms beta, t and the coefficients s, c = z - s t / beta, cu = t / beta, then
// streams q_j = (u_j - Q s) / beta into V_j and w'' = (w - Q c - cu u_j) / beta
// into w, and writes its partial of ||w''||^2.
// (104 registers at most, so that the Hessenberg CTA of the second stream
// fits beside one update CTA on an SM and the two run concurrently)
template <class C>
__global__ void __maxnreg__(104) k_arn_update(const ArnPlan<C>* __restrict__ D, int nd) {
  using T = typename Acc<C>::T;
  constexpr int KPT = ARN_SUB / (int)sizeof(C) / ARN_THREADS;
  constexpr int NW = ARN_THREADS / 32;
  __shared__ C sv[RMAX + 1], zv[RMAX + 1], sco[RMAX + 1], cco[RMAX + 1];
  __shared__ T shn[NW];
  int part;
  const ArnPlan<C>* dp = arn_find(D, nd, part);
  const GmresDev* s = dp->s;
  if (s->done) return;
  const int j = s->j;
  // at j = restart the cycle ends: q_j and w'' are not needed
  if (j >= s->restart) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int np = dp->nparts;
  arn_load_dots<C>(dp->red, j, sv, zv);
  __syncthreads();
  T beta;
  C t;
  arn_beta_t<C, T>(sv, zv, j, beta, t);
  const T ib = (T)1 / beta;
  const C tb = cmake<C>(t.x * ib, t.y * ib);           // cu = t / beta
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    const C si = sv[i], zi = zv[i];
    sco[i] = si;
    cco[i] = cmake<C>(zi.x - (si.x * tb.x - si.y * tb.y), zi.y - (si.x * tb.y + si.y * tb.x));
  }
  __syncthreads();
  T nrm = 0;
  {
    const ArnRange g = arn_range<C>(dp->n3, np, part);
    C* __restrict__ V = dp->V;
    const C* __restrict__ w = dp->w;
    C* __restrict__ u = dp->u;
    const long long ld = dp->ld;
    using R = typename real_of<C>::type;
    const R ibr = (R)ib;
    const R rho = sizeof(R) == 4 ? (R)s->inv_next32 : (R)s->inv_next;   // scale of u and w (see the dot pass)
    const int ct = threadIdx.x;
    C* Vj = V + (long long)j * ld;
    // the sweep runs backwards (last sub-chunk, highest column first): the
    // dot pass just read the basis forwards, so the columns it read last are
    // the likeliest still in L2, and the next dot pass starts on the columns
    // this pass reads last
    for (int sb = g.nsub - 1; sb >= 0; --sb) {
      const long long start = g.c0 + (long long)sb * g.sc;
      const int cnt = min(g.sc, g.c1 - (int)start);
      C as[KPT], ac[KPT];
#pragma unroll
      for (int q = 0; q < KPT; ++q) {
        as[q] = czero<C>();
        ac[q] = czero<C>();
      }
      C va[4][KPT], vb[4][KPT];
      if (j > 0) arn_load4r<C, KPT>(va, V, ld, start, j - 1, min(4, j), ct, cnt);
      for (int v0 = 0; v0 < j; v0 += 8) {
        const int n1 = min(4, j - v0 - 4), n2 = min(4, j - v0 - 8);
        if (n1 > 0) arn_load4r<C, KPT>(vb, V, ld, start, j - 1 - (v0 + 4), n1, ct, cnt);
        arn_axpy4<C, KPT>(va, sco, cco, as, ac, j - 1 - v0, min(4, j - v0));
        if (n2 > 0) arn_load4r<C, KPT>(va, V, ld, start, j - 1 - (v0 + 8), n2, ct, cnt);
        if (n1 > 0) arn_axpy4<C, KPT>(vb, sco, cco, as, ac, j - 1 - (v0 + 4), n1);
      }
      // w and u_j only now, so that their registers are free during the sweep
      C xw[KPT], xu[KPT];
#pragma unroll
      for (int q = 0; q < KPT; ++q) {
        const int e = ct + q * ARN_THREADS;
        xw[q] = e < cnt ? cscale(w[start + e], rho) : czero<C>();
        xu[q] = e < cnt ? cscale(u[start + e], rho) : czero<C>();
      }
#pragma unroll
      for (int q = 0; q < KPT; ++q) {
        const int e = ct + q * ARN_THREADS;
        if (e < cnt) {
          const C qj = cmake<C>((xu[q].x - as[q].x) * ibr, (xu[q].y - as[q].y) * ibr);
          C x = csub(xw[q], ac[q]);
          x.x -= (R)tb.x * xu[q].x - (R)tb.y * xu[q].y;
          x.y -= (R)tb.x * xu[q].y + (R)tb.y * xu[q].x;
          x.x *= ibr;
          x.y *= ibr;
          Vj[start + e] = qj;
          u[start + e] = x;   // u_{j+1} unnormalised: the next step scales it by 1 / ||w''||
          nrm += x.x * x.x + x.y * x.y;
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (lane == 0) shn[warp] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    T tt = 0;
    for (int w2 = 0; w2 < NW; ++w2) tt += shn[w2];
    dp->p2[part] = cmake<C>(tt, 0);
  }
}

// Step end, one CTA per plan (after the update pass and the Hessenberg
// bookkeeping): nu = ||w''|| from the norm partials (fixed order) becomes the
// tentative h_{j+1,j} and 1 / nu the scale at which the next step reads
// u_{j+1} = w'' (left unnormalised in u by the update pass) and w = A P^-1 of
// it; j advances.  nu = 0 is a breakdown: the Krylov space is invariant,
// column j is final, and the cycle ends.
template <class C>
__global__ void __launch_bounds__(STEP_END_THREADS) k_arn_step_end(const ArnPlan<C>* __restrict__ D) {
  using T = typename Acc<C>::T;
  constexpr int NPL = (NPART + 31) / 32;
  const ArnPlan<C>* dp = D + blockIdx.x;
  GmresDev* s = dp->s;
  if (s->done) return;
  const int j = s->j;
  const int lane = threadIdx.x & 31;
  __shared__ double nn_s;
  if (threadIdx.x < 32) {
    const C* p2 = dp->p2;
    T v[NPL];
#pragma unroll
    for (int q = 0; q < NPL; ++q) {
      const int bk = lane + 32 * q;
      v[q] = bk < dp->nparts ? __ldcg(p2 + bk).x : (T)0;
    }
    T a = 0;
#pragma unroll
    for (int q = 0; q < NPL; ++q) a += v[q];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) nn_s = (double)a;
  }
  __syncthreads();
  const double nu = sqrt(nn_s);
  if (nu == 0.0) {
    if (threadIdx.x == 0) {
      s->nu = 0.0;
      s->Hr[(long long)j * (RMAX + 1) + j + 1] = make_double2(0.0, 0.0);
      s->iters += 1;
    }
    __syncthreads();
    givens_column(s, j);
    if (threadIdx.x == 0) { s->k = j + 1; s->done = 1; }
    return;
  }
  if (threadIdx.x == 0) {
    s->nu = nu;
    s->Hr[(long long)j * (RMAX + 1) + j + 1] = make_double2(nu, 0.0);
    s->hnext = nu;
    s->inv_next = 1.0 / nu;
    s->inv_next32 = (float)s->inv_next;
    s->iters += 1;
    s->j = j + 1;
  }
}

// cycle start: beta = ||r||, V_0 = u = r / beta, g = beta e_1
template <class C>
__global__ void k_norm_partial(const C* __restrict__ r, long long n3, double2* __restrict__ partial) {
  __shared__ double2 sh[32];
  const long long chunk = ((unsigned)n3 + gridDim.x - 1) / gridDim.x;   // 32-bit division
  const long long c0 = blockIdx.x * chunk, c1 = min(n3, c0 + chunk);
  double nrm = 0;   // FP64 per thread: called once per cycle
  for (long long e = c0 + threadIdx.x; e < c1; e += blockDim.x) nrm += (double)r[e].x * r[e].x + (double)r[e].y * r[e].y;
  const double2 t = block_sum2(make_double2(nrm, 0), sh);
  if (threadIdx.x == 0) partial[(long long)blockIdx.x * PST] = t;
}

__global__ void k_cycle_init(GmresDev* __restrict__ s, const double2* __restrict__ partial, int nparts, double tol_abs,
                             int restart) {
  const double nn = warp_sum_partials(partial, nparts, 0).x;
  if (threadIdx.x != 0) return;
  const double beta = sqrt(nn);
  s->beta = beta;
  s->tol_abs = tol_abs;
  s->restart = restart;
  s->j = 0;
  s->k = 0;
  s->resest = beta;
  s->reorth = 0;
  s->nu = 0;
  s->inv_next = 1.0;      // V_0 = u = r / beta is stored normalised
  s->inv_next32 = 1.0f;
  s->arrive_dot = 0;
  s->arrive_upd = 0;
  for (int i = 0; i <= restart; ++i) s->g[i] = make_double2(0, 0);
  s->g[0] = make_double2(beta, 0);
  s->done = (beta <= tol_abs || beta == 0.0) ? 1 : 0;
}

template <class C>
__global__ void k_cycle_v0(const C* __restrict__ r, C* __restrict__ V, C* __restrict__ u, long long n3,
                           const GmresDev* __restrict__ s) {
  using T = typename real_of<C>::type;
  const T inv = s->beta > 0 ? (T)1 / (T)s->beta : (T)0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x) {
    const C v = cscale(r[e], inv);
    V[e] = v;
    u[e] = v;
  }
}

// y = H(0:k,0:k)^{-1} g(0:k)
// Back substitution R y = g on the rotated Hessenberg matrix: the upper
// triangle is staged in shared memory (column l holds rows 0..l at offset
// l (l + 1) / 2) by the whole block, then one warp solves from the bottom row
// up, each row's sum split over the lanes.
constexpr int SOLVE_THREADS = 256;
__global__ void __launch_bounds__(SOLVE_THREADS) k_solve_y(GmresDev* __restrict__ s) {
  extern __shared__ __align__(16) unsigned char solve_smem[];
  double2* R = reinterpret_cast<double2*>(solve_smem);
  __shared__ double2 ys[RMAX];
  const int k = s->k;
  const int tri = k * (k + 1) / 2;
  for (int e = threadIdx.x; e < tri; e += blockDim.x) {
    // column l = the largest l with l (l + 1) / 2 <= e
    int l = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
    while (l * (l + 1) / 2 > e) --l;
    while ((l + 1) * (l + 2) / 2 <= e) ++l;
    const int r = e - l * (l + 1) / 2;
    R[e] = s->H[(long long)l * (RMAX + 1) + r];
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  for (int i = k - 1; i >= 0; --i) {
    double2 t = make_double2(0, 0);
    for (int l = i + 1 + lane; l < k; l += 32) {
      const double2 h = R[l * (l + 1) / 2 + i];
      const double2 y = ys[l];
      t.x += h.x * y.x - h.y * y.y;
      t.y += h.x * y.y + h.y * y.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
      t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
    }
    if (lane == 0) {
      const double2 g = s->g[i];
      const double2 y = cmul(make_double2(g.x - t.x, g.y - t.y), cinv(R[i * (i + 1) / 2 + i]));
      ys[i] = y;
      s->y[i] = y;
    }
    __syncwarp();
  }
}

// u = sum_{i<k} y_i V_i
template <class C>
__global__ void k_combine(const C* __restrict__ V, long long ld, C* __restrict__ u, long long n3,
                          const GmresDev* __restrict__ s) {
  __shared__ C ys[RMAX];
  const int k = s->k;
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = cconv<C>(s->y[i]);
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x) {
    C acc = czero<C>();
    for (int i = 0; i < k; ++i) cfma(acc, ys[i], V[(long long)i * ld + e]);
    u[e] = acc;
  }
}

// x += sgn * scale * z   (x FP64, z any precision)
template <class C>
__global__ void k_axpy_to64(double2* __restrict__ x, const C* __restrict__ z, long long n3, const double* __restrict__ sc,
                            int sidx, double sgn) {
  const double a = sgn * (sc ? sc[sidx] : 1.0);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x) {
    x[e].x += a * (double)z[e].x;
    x[e].y += a * (double)z[e].y;
  }
}

// r = b - t (FP64)
__global__ void k_sub(const double2* __restrict__ b, const double2* __restrict__ t, double2* __restrict__ r, long long n3) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x)
    r[e] = make_double2(b[e].x - t[e].x, b[e].y - t[e].y);
}
__global__ void k_sub64(const float2* __restrict__ b, const float2* __restrict__ t, float2* __restrict__ r, long long n3) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x)
    r[e] = make_float2(b[e].x - t[e].x, b[e].y - t[e].y);
}

// out[idx] = sqrt(sum partial)
__global__ void k_norm_final(const double2* __restrict__ partial, int nparts, double* __restrict__ out, int idx) {
  const double nn = warp_sum_partials(partial, nparts, 0).x;
  if (threadIdx.x != 0) return;
  out[idx] = sqrt(nn);
}

// rhs64 = r / ||r||
__global__ void k_narrow_scaled(const double2* __restrict__ r, float2* __restrict__ o, long long n3,
                                const double* __restrict__ sc, int sidx) {
  const double n = sc[sidx];
  const double inv = n > 0 ? 1.0 / n : 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x)
    o[e] = make_float2((float)(r[e].x * inv), (float)(r[e].y * inv));
}

// b = M e_inc
__global__ void k_rhs(const double2* __restrict__ M, const double2* __restrict__ e, double2* __restrict__ b, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * N; i += (long long)gridDim.x * blockDim.x)
    b[i] = cmul(M[i % N], e[i]);
}

template <class C>
__global__ void k_axpy_same(C* __restrict__ x, const C* __restrict__ z, long long n3) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x)
    x[e] = cadd(x[e], z[e]);
}
template <class C>
__global__ void k_sub_same(const C* __restrict__ b, const C* __restrict__ t, C* __restrict__ r, long long n3) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x)
    r[e] = csub(b[e], t[e]);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 8); }

template <class C>
static vie_status axpy_same(C* x, const C* z, long long n3, cudaStream_t st) {
  k_axpy_same<C><<<grid_for(n3), 256, 0, st>>>(x, z, n3);
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}
template <class C>
static vie_status sub_same(const C* b, const C* t, C* r, long long n3, cudaStream_t st) {
  k_sub_same<C><<<grid_for(n3), 256, 0, st>>>(b, t, r, n3);
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

template <class C> struct KB;
template <> struct KB<float2> {
  static float2* V(Krylov& K) { return K.V64.as<float2>(); }
  static float2* u(Krylov& K) { return K.u64.as<float2>(); }
  static float2* z(Krylov& K) { return K.z64.as<float2>(); }
  static float2* w(Krylov& K) { return K.w64.as<float2>(); }
  static const ArnPlan<float2>* arn(Krylov& K) { return K.arn64.as<ArnPlan<float2>>(); }
  static int restart(const Krylov& K) { return K.rs64; }
  static const float2* M(vie_plan_s* P) { return P->M64.as<float2>(); }
  static const float2* spec(vie_plan_s* P) { return P->spec64.as<float2>(); }
  static float2* T(vie_plan_s* P) { return P->T64.as<float2>(); }
  static float2* S(vie_plan_s* P) { return P->S64.as<float2>(); }
};
template <> struct KB<double2> {
  static double2* V(Krylov& K) { return K.V128.as<double2>(); }
  static double2* u(Krylov& K) { return K.u128.as<double2>(); }
  static double2* z(Krylov& K) { return K.z128.as<double2>(); }
  static double2* w(Krylov& K) { return K.w128.as<double2>(); }
  static const ArnPlan<double2>* arn(Krylov& K) { return K.arn128.as<ArnPlan<double2>>(); }
  static int restart(const Krylov& K) { return K.rs128; }
  static const double2* M(vie_plan_s* P) { return P->M128.as<double2>(); }
  static const double2* spec(vie_plan_s* P) { return P->spec128.as<double2>(); }
  static double2* T(vie_plan_s* P) { return P->T128.as<double2>(); }
  static double2* S(vie_plan_s* P) { return P->S128.as<double2>(); }
};

template <class C>
static vie_status op_A(vie_plan_s* P, const C* x, C* y) {
  return matvec<C>(P, x, y, KB<C>::M(P), KB<C>::spec(P), KB<C>::T(P), KB<C>::S(P), P->st);
}

template <class C>
static vie_status op_Pinv(vie_plan_s* P, const C* r, C* z) {
  return precond_apply<C>(P, r, z, P->st);
}

template <class C>
static vie_status arn_upload(vie_plan_s* P, DevBuf& buf);

static vie_status krylov_alloc(vie_plan_s* P, bool need64, bool need128) {
  if (!P->kry) P->kry.reset(new Krylov());
  Krylov& K = *P->kry;
  const long long n3 = 3LL * P->nx * P->ny * P->nz;
  // the complex-FP32 inner cycles of the mixed solve are longer than the FP64
  // restart (by default twice, capped at RMAX): their basis then takes the
  // bytes of an FP64 GMRES(restart) basis
  const int R128 = P->opts.restart;
  const int R64 = P->opts.inner_restart > 0 ? P->opts.inner_restart : std::min(2 * R128, RMAX);
  K.restart = need64 ? R64 : R128;
  K.rs64 = R64;
  K.rs128 = R128;
  K.n3 = n3;
  K.ld = (n3 + 31) / 32 * 32;
  const long long ld = K.ld;
  if (!K.state.p) {
    VIE_TRY(K.state.alloc(sizeof(GmresDev)));
    // stream-ordered like the allocation (a legacy-stream memset would not be
    // ordered with the plan's non-blocking stream)
    VIE_CUDA(cudaMemsetAsync(K.state.p, 0, sizeof(GmresDev), P->st));
    VIE_TRY(K.partial.alloc(sizeof(double2) * NPART * PST));
    VIE_TRY(K.p1.alloc(sizeof(double2) * NPART * PST));
    VIE_TRY(K.p2.alloc(sizeof(double2) * NPART));
    VIE_TRY(K.red.alloc(sizeof(double2) * PST));
    K.nparts = arn_parts(n3);
    VIE_TRY(K.scal.alloc(sizeof(double) * 8));
    VIE_TRY(K.x128.alloc(sizeof(double2) * n3));
    VIE_TRY(K.r128.alloc(sizeof(double2) * n3));
    VIE_TRY(K.b128.alloc(sizeof(double2) * n3));
    VIE_TRY(K.t128.alloc(sizeof(double2) * n3));
    VIE_CUDA(cudaHostAlloc((void**)&K.hflag, sizeof(int) * 4, cudaHostAllocDefault));
    VIE_CUDA(cudaEventCreateWithFlags(&K.ev, cudaEventDisableTiming));
    VIE_CUDA(cudaStreamCreateWithFlags(&K.cap, cudaStreamNonBlocking));
    VIE_CUDA(cudaStreamCreateWithFlags(&K.side, cudaStreamNonBlocking));
    VIE_CUDA(cudaEventCreateWithFlags(&K.ev_fork, cudaEventDisableTiming));
    VIE_CUDA(cudaEventCreateWithFlags(&K.ev_join, cudaEventDisableTiming));
  }
  if (need64 && !K.V64.p) {
    VIE_TRY(K.V64.alloc(sizeof(float2) * ld * (R64 + 1)));
    VIE_TRY(K.u64.alloc(sizeof(float2) * n3));
    VIE_TRY(K.z64.alloc(sizeof(float2) * n3));
    VIE_TRY(K.w64.alloc(sizeof(float2) * ld));
    VIE_TRY(K.d64.alloc(sizeof(float2) * n3));
    VIE_TRY(K.rhs64.alloc(sizeof(float2) * n3));
    VIE_TRY(K.r64.alloc(sizeof(float2) * n3));
    VIE_TRY(arn_upload<float2>(P, K.arn64));
  }
  if (need128 && !K.V128.p) {
    VIE_TRY(K.V128.alloc(sizeof(double2) * ld * (R128 + 1)));
    VIE_TRY(K.u128.alloc(sizeof(double2) * n3));
    VIE_TRY(K.z128.alloc(sizeof(double2) * n3));
    VIE_TRY(K.w128.alloc(sizeof(double2) * ld));
    VIE_TRY(K.xbest.alloc(sizeof(double2) * n3));
    VIE_TRY(arn_upload<double2>(P, K.arn128));
  }
  return VIE_OK;
}

template <class C>
static size_t dot_smem() {
  return (size_t)(ARN_THREADS / 32) * (4 * (RMAX + 1) + 4) * sizeof(typename Acc<C>::T);
}

// the plan's Arnoldi descriptor (fixed pointers; written once per allocation)
template <class C>
static ArnPlan<C> arn_desc(vie_plan_s* P) {
  Krylov& K = *P->kry;
  ArnPlan<C> d{};
  d.V = KB<C>::V(K);
  d.w = KB<C>::w(K);
  d.u = KB<C>::u(K);
  d.s = K.state.as<GmresDev>();
  d.p1 = K.p1.as<C>();
  d.p2 = K.p2.as<C>();
  d.red = K.red.as<C>();
  d.ld = K.ld;
  d.n3 = (int)K.n3;
  d.part0 = 0;
  d.nparts = K.nparts;
  return d;
}

template <class C>
static vie_status arn_upload(vie_plan_s* P, DevBuf& buf) {
  if (!buf.p) VIE_TRY(buf.alloc(sizeof(ArnPlan<C>)));
  const ArnPlan<C> d = arn_desc<C>(P);
  VIE_CUDA(cudaMemcpyAsync(buf.p, &d, sizeof(d), cudaMemcpyHostToDevice, P->st));
  VIE_CUDA(cudaStreamSynchronize(P->st));   // d lives on this stack frame
  return VIE_OK;
}

// the three Arnoldi kernels of one step over a work-list of nd plans (total
// CTAs ncta), descriptors D on the device
template <class C>
static vie_status arn_launch(const ArnPlan<C>* D, int nd, int ncta, cudaStream_t st, cudaStream_t side,
                             cudaEvent_t ev_fork, cudaEvent_t ev_join) {
  VIE_TRY(smem_optin(k_arn_dot<C>, dot_smem<C>()));
  {
    Prof pf_(sizeof(C) == 8 ? "arnoldi_dot_c64" : "arnoldi_dot_c128", st);
    k_arn_dot<C><<<ncta, ARN_THREADS, dot_smem<C>(), st>>>(D, nd);
  }
  // the Hessenberg bookkeeping beside the update pass (both read the dot partials)
  VIE_CUDA(cudaEventRecord(ev_fork, st));
  VIE_CUDA(cudaStreamWaitEvent(side, ev_fork, 0));
  { Prof pf_("arnoldi_hessenberg", side); k_arn_hess<C><<<nd, HESS_THREADS, 0, side>>>(D); }
  VIE_CUDA(cudaEventRecord(ev_join, side));
  {
    Prof pf_(sizeof(C) == 8 ? "arnoldi_update_c64" : "arnoldi_update_c128", st);
    k_arn_update<C><<<ncta, ARN_THREADS, 0, st>>>(D, nd);
  }
  VIE_CUDA(cudaStreamWaitEvent(st, ev_join, 0));
  { Prof pf_("arnoldi_step_end", st); k_arn_step_end<C><<<nd, STEP_END_THREADS, 0, st>>>(D); }
  count_launch(4);
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

// ---------------------------------------------------------------------------
// Solves as resumable runs, advanced in lockstep.
//
// A run is one plan's solve.  The driver advances a set of runs one GMRES
// cycle at a time: every run in a cycle takes its Arnoldi steps together with
// the others -- one captured step graph holds each run's preconditioner and
// matvec as parallel branches and then the step kernels of all of them, each
// one launch over a work-list of the plans -- and the host polls the device
// stop flags between chunks of steps.  A run whose cycle ended does its host
// work (update of the iterate, true residual, refinement step, next cycle)
// and rejoins the steps.  A solve on its own is a set of one run; a batch
// (vie_solve_batch) or the server puts many plans in one set.  A plan's
// kernels see the same CTA ranges in either case, so its result is bitwise
// the same alone and in a batch.
// ---------------------------------------------------------------------------
struct Run {
  vie_plan_s* P = nullptr;
  const double2* e_inc = nullptr;
  double2* w_out = nullptr;
  vie_info* info = nullptr;
  std::chrono::steady_clock::time_point t0;
  bool mixed = false;
  bool finished = false;
  vie_status status = VIE_OK;
  std::string err;
  double bnorm = 0;
  int inner = 0, outer = 0;
  // FP64 iterative refinement of a mixed solve
  double rn = 0, rn_prev = 0;
  int ir_stalls = 0;
  // the mixed solve fell back to FP64 GMRES (its iterations in that run)
  bool fallback = false;
  int fallback_iters = 0;
  // ||b - A x|| when r128 holds that residual of the current x128 (FP64),
  // else negative: the final residual is then not evaluated again
  double res_norm = -1;
  // the GMRES run in progress (complex FP32 inner cycle, or the FP64 solve)
  double gnorm = 0, gtol = 0;
  int gmax_iter = 0, gmax_cycles = 0, gtotal = 0, gcycles = 0, gstalls = 0;
  double rr = 1, rr_best = 1;
  bool have_best = false;
  bool in_cycle = false;
  int cyc_len = 0, steps = 0;   // steps allowed / launched in the current cycle
};

// GMRES vectors of a run by precision: right-hand side, iterate, residual
template <class C> struct GB;
template <> struct GB<float2> {
  static float2* rhs(Krylov& K) { return K.rhs64.as<float2>(); }
  static float2* x(Krylov& K) { return K.d64.as<float2>(); }
  static float2* rw(Krylov& K) { return K.r64.as<float2>(); }
};
template <> struct GB<double2> {
  static double2* rhs(Krylov& K) { return K.b128.as<double2>(); }
  static double2* x(Krylov& K) { return K.x128.as<double2>(); }
  static double2* rw(Krylov& K) { return K.r128.as<double2>(); }
};

static vie_status norm128(vie_plan_s* P, const double2* v, int idx, double* out) {
  Krylov& K = *P->kry;
  double2* part = K.partial.as<double2>();
  k_norm_partial<double2><<<NPART, RED_THREADS, 0, P->st>>>(v, K.n3, part);
  k_norm_final<<<1, 32, 0, P->st>>>(part, NPART, K.scal.as<double>(), idx);
  count_launch(2);
  VIE_CHECK_LAUNCH();
  VIE_CUDA(cudaMemcpyAsync(out, K.scal.as<double>() + idx, sizeof(double), cudaMemcpyDeviceToHost, P->st));
  VIE_CUDA(cudaStreamSynchronize(P->st));
  return VIE_OK;
}

static vie_status run_finish(Run& R);
static vie_status ir_next(Run& R);

// cycle start from the run's current residual: beta = ||r||, V_0 = u = r / beta
template <class C>
static vie_status cycle_begin(Run& R) {
  vie_plan_s* P = R.P;
  Krylov& K = *P->kry;
  cudaStream_t st = P->st;
  const long long n3 = K.n3;
  const int len = std::min(KB<C>::restart(K), R.gmax_iter - R.gtotal);
  k_norm_partial<C><<<NPART, RED_THREADS, 0, st>>>(GB<C>::rw(K), n3, K.partial.as<double2>());
  k_cycle_init<<<1, 32, 0, st>>>(K.state.as<GmresDev>(), K.partial.as<double2>(), NPART, R.gtol * R.gnorm, len);
  k_cycle_v0<C><<<grid_for(n3), 256, 0, st>>>(GB<C>::rw(K), KB<C>::V(K), KB<C>::u(K), n3, K.state.as<GmresDev>());
  count_launch(3);
  VIE_CHECK_LAUNCH();
  // restart columns take restart + 1 steps: the last reduction finalises the last column
  R.cyc_len = len + 1;
  R.steps = 0;
  R.in_cycle = true;
  return VIE_OK;
}

// the GMRES run ended (its iterate is in GB<C>::x): the FP64 solve is done,
// a complex-FP32 inner cycle feeds one refinement step
template <class C>
static vie_status gmres_done(Run& R);

template <>
vie_status gmres_done<double2>(Run& R) {
  if (R.fallback) {
    R.fallback_iters = R.gtotal;
    R.inner += R.gtotal;
    ++R.outer;
  } else {
    R.inner = R.gtotal;
    R.outer = 1;
  }
  return run_finish(R);
}

// A mixed solve whose refinement stopped making progress goes on as FP64
// GMRES(restart) from its current iterate, with the complex-FP64 inverses of
// the same preconditioner.  The complex-FP32 inner solve fails when the
// operator or a preconditioner block is too ill-conditioned for FP32
// (a correction that raises the FP64 residual, or steps that gain less than
// 1%); FP64 GMRES then converges as the FP64 solve of the same system does.
static vie_status fallback_fp64(Run& R) {
  vie_plan_s* P = R.P;
  if (R.rn <= P->opts.tol * R.bnorm || R.inner >= P->opts.max_iter) return run_finish(R);
  {
    AllocScope a(P->st);
    VIE_TRY(krylov_alloc(P, true, true));
    VIE_TRY(precond_add_fp64(P));
  }
  Krylov& K = *P->kry;
  R.mixed = false;
  R.fallback = true;
  // r128 = b - A x of the current iterate; A x = b from x (the best iterate
  // so far, kept in xbest)
  R.gnorm = R.bnorm;
  R.gtol = P->opts.tol;
  R.gmax_iter = P->opts.max_iter - R.inner;
  R.gmax_cycles = 1 << 30;
  R.gtotal = 0;
  R.gcycles = 0;
  R.gstalls = 0;
  R.rr = R.rn / R.bnorm;
  R.rr_best = R.rr;
  VIE_CUDA(cudaMemcpyAsync(K.xbest.p, K.x128.p, sizeof(double2) * K.n3, cudaMemcpyDeviceToDevice, P->st));
  R.have_best = true;
  return cycle_begin<double2>(R);
}

template <>
vie_status gmres_done<float2>(Run& R) {
  vie_plan_s* P = R.P;
  Krylov& K = *P->kry;
  cudaStream_t st = P->st;
  const long long n3 = K.n3;
  const int it = R.gtotal;
  R.inner += it;
  double2* x = K.x128.as<double2>();
  double2* r = K.r128.as<double2>();
  double2* t = K.t128.as<double2>();
  double* scal = K.scal.as<double>();
  // x += ||r|| d (scal[3] = ||r|| of the step's right-hand side)
  R.res_norm = -1;
  k_axpy_to64<float2><<<grid_for(n3), 256, 0, st>>>(x, K.d64.as<float2>(), n3, scal, 3, 1.0);
  count_launch();
  VIE_TRY(op_A<double2>(P, x, t));
  k_sub<<<grid_for(n3), 256, 0, st>>>(K.b128.as<double2>(), t, r, n3);
  count_launch();
  VIE_CHECK_LAUNCH();
  ++R.outer;
  const double rn_step = R.rn;
  VIE_TRY(norm128(P, r, 5, &R.rn));
  if (!std::isfinite(R.rn)) {
    int herr = 0;
    VIE_CUDA(cudaMemcpyAsync(&herr, P->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    VIE_CUDA(cudaStreamSynchronize(st));
    if (herr) {
      set_error("vie_solve: a bounded wait in a kernel ran out (code %d); results invalid", herr);
      return VIE_ETIMEOUT;
    }
    set_error("vie_solve: refinement diverged (non-finite residual)");
    return VIE_ECUDA;
  }
  if (R.rn > rn_step && it > 0) {
    // the correction raised the FP64 residual: take it back (x -= ||r|| d,
    // scal[3] still holds ||r||) and go on in FP64
    k_axpy_to64<float2><<<grid_for(n3), 256, 0, st>>>(x, K.d64.as<float2>(), n3, scal, 3, -1.0);
    count_launch();
    VIE_TRY(op_A<double2>(P, x, t));
    k_sub<<<grid_for(n3), 256, 0, st>>>(K.b128.as<double2>(), t, r, n3);
    count_launch();
    VIE_CHECK_LAUNCH();
    VIE_TRY(norm128(P, r, 3, &R.rn));
    R.res_norm = R.rn;
    return fallback_fp64(R);
  }
  R.res_norm = R.rn;
  VIE_CUDA(cudaMemcpyAsync(scal + 3, scal + 5, sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (it == 0) return run_finish(R);
  // three refinement steps in a row that do not reduce the FP64 residual by
  // 1% mean the complex-FP32 inner solve has nothing left to give (the rule
  // of the FP64 GMRES restarts; a hard operator may gain only a few percent
  // per cycle and still converge)
  if (R.rn > 0.99 * R.rn_prev) {
    if (++R.ir_stalls >= 3) return fallback_fp64(R);
  } else {
    R.ir_stalls = 0;
  }
  R.rn_prev = R.rn;
  return ir_next(R);
}

// GMRES on A x = rhs (precision C) from x = 0: a true relative residual
// (rhs - A x, precision C) <= tol ends it, as do max_iter steps or
// max_cycles cycles (then the caller evaluates the residual itself)
template <class C>
static vie_status gmres_begin(Run& R, double tol, int max_iter, int max_cycles) {
  vie_plan_s* P = R.P;
  Krylov& K = *P->kry;
  cudaStream_t st = P->st;
  const long long n3 = K.n3;
  double* scal = K.scal.as<double>();
  k_norm_partial<C><<<NPART, RED_THREADS, 0, st>>>(GB<C>::rhs(K), n3, K.partial.as<double2>());
  k_norm_final<<<1, 32, 0, st>>>(K.partial.as<double2>(), NPART, scal, 0);
  count_launch(2);
  VIE_CUDA(cudaMemsetAsync(GB<C>::x(K), 0, sizeof(C) * n3, st));
  VIE_CUDA(cudaMemcpyAsync(GB<C>::rw(K), GB<C>::rhs(K), sizeof(C) * n3, cudaMemcpyDeviceToDevice, st));
  VIE_CUDA(cudaMemcpyAsync(K.hflag + 2, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  VIE_CUDA(cudaStreamSynchronize(st));
  R.gnorm = *reinterpret_cast<double*>(K.hflag + 2);
  R.gtol = tol;
  R.gmax_iter = max_iter;
  R.gmax_cycles = max_cycles;
  R.gtotal = 0;
  R.gcycles = 0;
  R.gstalls = 0;
  R.rr = 1.0;        // x0 = 0 has the residual ||rhs||
  R.rr_best = 1.0;
  R.have_best = false;
  if (R.gnorm == 0.0 || max_iter <= 0) {
    R.rr = 0.0;
    return gmres_done<C>(R);
  }
  return cycle_begin<C>(R);
}

// end of a cycle: x += P^-1 (V y), then the true residual decides
template <class C>
static vie_status cycle_end(Run& R) {
  vie_plan_s* P = R.P;
  Krylov& K = *P->kry;
  cudaStream_t st = P->st;
  const long long n3 = K.n3;
  GmresDev* s = K.state.as<GmresDev>();
  C* V = KB<C>::V(K);
  C* u = KB<C>::u(K);
  C* z = KB<C>::z(K);
  C* w = KB<C>::w(K);
  C* x = GB<C>::x(K);
  C* rhs = GB<C>::rhs(K);
  C* rw = GB<C>::rw(K);
  double* scal = K.scal.as<double>();
  R.in_cycle = false;
  VIE_CUDA(cudaMemcpyAsync(K.hflag + 1, &s->k, sizeof(int), cudaMemcpyDeviceToHost, st));
  {
    const int rs = KB<C>::restart(K);
    const size_t smem = sizeof(double2) * (size_t)rs * (rs + 1) / 2;
    VIE_TRY(smem_optin(k_solve_y, smem));
    k_solve_y<<<1, SOLVE_THREADS, smem, st>>>(s);
  }
  k_combine<C><<<grid_for(n3), 256, 0, st>>>(V, K.ld, u, n3, s);
  count_launch(2);
  VIE_TRY(op_Pinv<C>(P, u, z));
  VIE_TRY(axpy_same<C>(x, z, n3, st));
  R.res_norm = -1;
  VIE_CUDA(cudaStreamSynchronize(st));
  const int hk = K.hflag[1];
  if (++R.gcycles >= R.gmax_cycles) {
    // the caller evaluates the residual itself (in higher precision)
    R.gtotal += hk;
    R.rr = -1.0;
    return gmres_done<C>(R);
  }
  // true residual rw = rhs - A x
  VIE_TRY(op_A<C>(P, x, w));
  VIE_TRY(sub_same<C>(rhs, w, rw, n3, st));
  k_norm_partial<C><<<NPART, RED_THREADS, 0, st>>>(rw, n3, K.partial.as<double2>());
  k_norm_final<<<1, 32, 0, st>>>(K.partial.as<double2>(), NPART, scal, 1);
  count_launch(2);
  VIE_CUDA(cudaMemcpyAsync(K.hflag + 2, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
  VIE_CUDA(cudaStreamSynchronize(st));
  VIE_CHECK_LAUNCH();
  R.gtotal += hk;
  R.rr = *reinterpret_cast<double*>(K.hflag + 2) / R.gnorm;
  // an FP64 run works on A x = b itself: rw = r128 is the final residual
  if (sizeof(C) == 16) R.res_norm = *reinterpret_cast<double*>(K.hflag + 2);
  bool stop = R.rr <= R.gtol || hk == 0;
  if (!stop) {
    // a cycle cannot raise the true residual in exact arithmetic (y = 0 is
    // feasible), but on an ill-conditioned operator the basis can lose
    // orthogonality and it does; the next cycle still starts from the new
    // residual (a different Krylov space), and the best iterate is kept
    if (R.rr < R.rr_best) {
      VIE_CUDA(cudaMemcpyAsync(K.xbest.p, x, sizeof(C) * n3, cudaMemcpyDeviceToDevice, st));
      R.have_best = true;
    }
    // restarted GMRES may converge slowly, but three cycles in a row that
    // do not improve the best residual by 1% mean stagnation (or the
    // rounding floor of this precision): stop and report the residual
    if (R.rr > 0.99 * R.rr_best) {
      if (++R.gstalls >= 3) stop = true;
    } else {
      R.gstalls = 0;
    }
    if (!stop) R.rr_best = std::min(R.rr, R.rr_best);
  }
  if (!stop && R.gtotal < R.gmax_iter) return cycle_begin<C>(R);
  if (R.rr > R.rr_best) {
    // end on the best iterate (x0 = 0 when no cycle went below ||rhs||)
    if (R.have_best) VIE_CUDA(cudaMemcpyAsync(x, K.xbest.p, sizeof(C) * n3, cudaMemcpyDeviceToDevice, st));
    else VIE_CUDA(cudaMemsetAsync(x, 0, sizeof(C) * n3, st));
    VIE_TRY(op_A<C>(P, x, w));
    VIE_TRY(sub_same<C>(rhs, w, rw, n3, st));
    R.rr = R.rr_best;
    R.res_norm = -1;
  }
  return gmres_done<C>(R);
}

// next refinement step: one complex-FP32 GMRES cycle on A d = r / ||r||,
// stopped early once its Arnoldi residual estimate reaches eta
static vie_status ir_next(Run& R) {
  vie_plan_s* P = R.P;
  Krylov& K = *P->kry;
  const double tol = P->opts.tol;
  if (R.outer >= P->opts.max_refine || R.inner >= P->opts.max_iter || R.rn <= tol * R.bnorm) return run_finish(R);
  const double eta = std::max(P->opts.inner_tol, 0.5 * tol * R.bnorm / R.rn);
  k_narrow_scaled<<<grid_for(K.n3), 256, 0, P->st>>>(K.r128.as<double2>(), K.rhs64.as<float2>(), K.n3,
                                                      K.scal.as<double>(), 3);
  count_launch();
  return gmres_begin<float2>(R, eta, std::min(K.rs64, P->opts.max_iter - R.inner), 1);
}

// final FP64 residual, result and info
static vie_status run_finish(Run& R) {
  vie_plan_s* P = R.P;
  Krylov& K = *P->kry;
  cudaStream_t st = P->st;
  const long long n3 = K.n3;
  double2* b = K.b128.as<double2>();
  double2* x = K.x128.as<double2>();
  double2* r = K.r128.as<double2>();
  double2* t = K.t128.as<double2>();
  GmresDev* sdev = K.state.as<GmresDev>();
  R.in_cycle = false;
  double rn = R.res_norm;
  if (rn < 0) {
    VIE_TRY(op_A<double2>(P, x, t));
    k_sub<<<grid_for(n3), 256, 0, st>>>(b, t, r, n3);
    count_launch();
    VIE_CHECK_LAUNCH();
    VIE_TRY(norm128(P, r, 4, &rn));
  }
  const double relres = R.bnorm > 0 ? rn / R.bnorm : 0.0;
  VIE_CUDA(cudaMemcpyAsync(R.w_out, x, sizeof(double2) * n3, cudaMemcpyDeviceToDevice, st));
  int herr = 0, hreorth = 0;
  VIE_CUDA(cudaMemcpyAsync(&herr, P->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  VIE_CUDA(cudaMemcpyAsync(&hreorth, &sdev->reorths, sizeof(int), cudaMemcpyDeviceToHost, st));
  VIE_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    cudaMemsetAsync(P->dev_err.p, 0, sizeof(int), st);
    set_error("vie_solve: a bounded wait in a kernel ran out (code %d); results invalid", herr);
    return VIE_ETIMEOUT;
  }
  const float ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - R.t0).count();
  if (R.info) {
    vie_info* info = R.info;
    info->iters_inner = R.inner;
    info->iters_outer = R.outer;
    info->relres = relres;
    info->precond_bytes = P->precond_bytes;
    info->kept_fraction = P->kept_fraction;
    info->t_setup_ms = P->t_setup_ms;
    info->t_solve_ms = ms;
    info->precond_blocks = P->precond_blocks;
    info->precond_discarded = P->precond_discarded;
    info->reorth_passes = hreorth;
    info->iters_fp64_fallback = R.fallback_iters;
  }
  R.finished = true;
  R.status = relres <= P->opts.tol ? VIE_OK : VIE_ENOCONV;
  return R.status;
}

// (I - M N) w = M e_inc: right-hand side, preconditioner, first GMRES run
static vie_status run_begin(Run& R) {
  vie_plan_s* P = R.P;
  R.t0 = std::chrono::steady_clock::now();
  if (!P->has_eps) { set_error("vie_solve: permittivity not set"); return VIE_ESTATE; }
  R.mixed = P->opts.precision == VIE_MIXED;
  VIE_TRY(krylov_alloc(P, R.mixed, !R.mixed));
  Krylov& K = *P->kry;
  cudaStream_t st = P->st;
  const long long n3 = K.n3;
  const long long N = n3 / 3;
  double2* b = K.b128.as<double2>();
  double2* x = K.x128.as<double2>();
  k_rhs<<<grid_for(n3), 256, 0, st>>>(P->M128.as<double2>(), R.e_inc, b, N);
  count_launch();
  VIE_CHECK_LAUNCH();
  VIE_TRY(norm128(P, b, 2, &R.bnorm));
  if (!std::isfinite(R.bnorm)) {
    set_error("vie_solve: non-finite right-hand side (check the permittivity and incident field)");
    return VIE_EINVAL;
  }
  if (!P->prec_built) VIE_TRY(precond_build(P));
  VIE_CUDA(cudaMemsetAsync(&K.state.as<GmresDev>()->reorths, 0, sizeof(int), st));
  R.inner = 0;
  R.outer = 0;
  if (R.bnorm == 0.0) {
    VIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * n3, st));
    return run_finish(R);
  }
  if (!R.mixed) return gmres_begin<double2>(R, P->opts.tol, P->opts.max_iter, 1 << 30);
  // GMRES-IR: each refinement step runs one complex-FP32 GMRES cycle on
  // A d = r / ||r|| (stopped early once its Arnoldi residual estimate
  // reaches eta), then x += ||r|| d and r = b - A x in FP64.  Restarts thus
  // happen in FP64 and the FP32 rounding floor of the inner residual never
  // limits the outer accuracy.
  VIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * n3, st));
  VIE_CUDA(cudaMemcpyAsync(K.r128.p, b, sizeof(double2) * n3, cudaMemcpyDeviceToDevice, st));
  VIE_TRY(norm128(P, K.r128.as<double2>(), 3, &R.rn));   // scal[3] = ||r||, read by the narrowing and the update
  R.rn_prev = 2.0 * R.bnorm;
  R.ir_stalls = 0;
  return ir_next(R);
}

// A run's host step failed: record it and take the run out of the set.
static void run_fail(Run& R, vie_status s) {
  R.status = s;
  R.err = vie_last_error();
  R.finished = true;
  R.in_cycle = false;
}

// ---------------------------------------------------------------------------
// lockstep driver
// ---------------------------------------------------------------------------
struct Lockstep {
  int device = 0;
  cudaStream_t cap = nullptr;                 // capture stream; the step graph is launched on `st`
  cudaStream_t side = nullptr;                // Hessenberg bookkeeping beside the update pass
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_root = nullptr;
  std::vector<cudaStream_t> br;               // one branch per run of the set (preconditioner + matvec)
  std::vector<cudaEvent_t> ev_br;
  DevBuf d64, d128;                           // descriptor arrays of the set by precision
  DevBuf done_dev;                            // int [n]: stop flags gathered by k_gather_done
  int* done_host = nullptr;                   // pinned mirror
  cudaGraphExec_t exec = nullptr;
  std::vector<Run*> members;                  // the set the graph was captured for
  std::vector<char> modes;                    // and each member's precision then (1 = mixed)
  int nd64 = 0, ncta64 = 0, nd128 = 0, ncta128 = 0;   // work-lists of the captured set
  int step_launches = 0;
  ~Lockstep() { release(); }
  void release() {
    d64.release();
    d128.release();
    done_dev.release();
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    members.clear();
    modes.clear();
    for (auto s : br) cudaStreamDestroy(s);
    for (auto e : ev_br) cudaEventDestroy(e);
    br.clear();
    ev_br.clear();
    if (cap) cudaStreamDestroy(cap);
    if (side) cudaStreamDestroy(side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_root) cudaEventDestroy(ev_root);
    if (done_host) cudaFreeHost(done_host);
    cap = side = nullptr;
    ev_fork = ev_join = ev_root = nullptr;
    done_host = nullptr;
  }
};

void lockstep_free(Lockstep* L) { delete L; }

// gather the stop flags of a set of GMRES states
__global__ void k_gather_done(GmresDev* const* __restrict__ s, int n, int* __restrict__ out) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = s[i]->done;
}

// layout of done_dev for a set of n runs: the stop flags (int), then, at a
// 16-byte aligned offset, the runs' GMRES state pointers
static size_t flags_off(size_t n) { return (sizeof(int) * std::max<size_t>(n, 8) + 15) / 16 * 16; }
static size_t flags_bytes(size_t n) { return flags_off(n) + sizeof(GmresDev*) * std::max<size_t>(n, 8); }

static vie_status lockstep_init(Lockstep& L, int n) {
  if (!L.cap) {
    VIE_CUDA(cudaGetDevice(&L.device));
    VIE_CUDA(cudaStreamCreateWithFlags(&L.cap, cudaStreamNonBlocking));
    VIE_CUDA(cudaStreamCreateWithFlags(&L.side, cudaStreamNonBlocking));
    VIE_CUDA(cudaEventCreateWithFlags(&L.ev_fork, cudaEventDisableTiming));
    VIE_CUDA(cudaEventCreateWithFlags(&L.ev_join, cudaEventDisableTiming));
    VIE_CUDA(cudaEventCreateWithFlags(&L.ev_root, cudaEventDisableTiming));
  }
  while ((int)L.br.size() < n) {
    cudaStream_t s;
    cudaEvent_t e;
    VIE_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    VIE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    L.br.push_back(s);
    L.ev_br.push_back(e);
  }
  if (L.done_dev.bytes < flags_bytes(n)) {
    VIE_TRY(L.done_dev.alloc(flags_bytes(n)));
    VIE_CUDA(cudaStreamSynchronize(L.done_dev.stream));   // used on other streams
    if (L.done_host) cudaFreeHost(L.done_host);
    L.done_host = nullptr;
    VIE_CUDA(cudaHostAlloc((void**)&L.done_host, sizeof(int) * (size_t)std::max(n, 8), cudaHostAllocDefault));
  }
  return VIE_OK;
}

// descriptor array of the members of one precision (part0 = running CTA count)
template <class C>
static vie_status lockstep_desc(Lockstep& L, const std::vector<Run*>& m, DevBuf& buf, int* nd, int* ncta,
                                cudaStream_t st) {
  std::vector<ArnPlan<C>> h;
  int parts = 0;
  for (Run* R : m) {
    if ((sizeof(C) == 8) != R->mixed) continue;
    ArnPlan<C> d = arn_desc<C>(R->P);
    d.part0 = parts;
    parts += d.nparts;
    h.push_back(d);
  }
  *nd = (int)h.size();
  *ncta = parts;
  if (h.empty()) return VIE_OK;
  if (buf.bytes < sizeof(ArnPlan<C>) * h.size()) {
    VIE_TRY(buf.alloc(sizeof(ArnPlan<C>) * std::max<size_t>(h.size(), 8)));
    VIE_CUDA(cudaStreamSynchronize(buf.stream));   // used on other streams
  }
  VIE_CUDA(cudaMemcpyAsync(buf.p, h.data(), sizeof(ArnPlan<C>) * h.size(), cudaMemcpyHostToDevice, st));
  VIE_CUDA(cudaStreamSynchronize(st));   // h lives on this stack frame
  return VIE_OK;
}

// one Arnoldi step of every member: preconditioner and matvec per member on
// its branch, then the step kernels of each precision over its work-list
static vie_status lockstep_enqueue(Lockstep& L, const std::vector<Run*>& m, cudaStream_t st, int nd64, int ncta64,
                                   int nd128, int ncta128) {
  VIE_CUDA(cudaEventRecord(L.ev_root, st));
  for (size_t i = 0; i < m.size(); ++i) {
    vie_plan_s* P = m[i]->P;
    Krylov& K = *P->kry;
    cudaStream_t b = L.br[i];
    VIE_CUDA(cudaStreamWaitEvent(b, L.ev_root, 0));
    cudaStream_t keep = P->st;
    P->st = b;
    vie_status s;
    if (m[i]->mixed) {
      s = op_Pinv<float2>(P, K.u64.as<float2>(), K.z64.as<float2>());
      if (s >= 0) s = op_A<float2>(P, K.z64.as<float2>(), K.w64.as<float2>());
    } else {
      s = op_Pinv<double2>(P, K.u128.as<double2>(), K.z128.as<double2>());
      if (s >= 0) s = op_A<double2>(P, K.z128.as<double2>(), K.w128.as<double2>());
    }
    P->st = keep;
    if (s < 0) return s;
    VIE_CUDA(cudaEventRecord(L.ev_br[i], b));
  }
  for (size_t i = 0; i < m.size(); ++i) VIE_CUDA(cudaStreamWaitEvent(st, L.ev_br[i], 0));
  if (nd64) VIE_TRY(arn_launch<float2>(L.d64.as<ArnPlan<float2>>(), nd64, ncta64, st, L.side, L.ev_fork, L.ev_join));
  if (nd128)
    VIE_TRY(arn_launch<double2>(L.d128.as<ArnPlan<double2>>(), nd128, ncta128, st, L.side, L.ev_fork, L.ev_join));
  return VIE_OK;
}

// One pass over the runs (each already begun): a chunk of Arnoldi steps of
// every run in a cycle, launched on `st` as the set's step graph (captured
// again whenever the set changes), then the cycle ends of the runs whose
// cycle finished.  Returns false when no run is in a cycle.
static bool lockstep_pass_impl(Lockstep& L, std::vector<Run*>& runs, cudaStream_t st) {
  std::vector<Run*> m;
  int& nd64 = L.nd64;
  int& ncta64 = L.ncta64;
  int& nd128 = L.nd128;
  int& ncta128 = L.ncta128;
  {
    for (Run* R : runs)
      if (!R->finished && R->in_cycle) m.push_back(R);
    if (m.empty()) return false;
    vie_status s = lockstep_init(L, (int)m.size());
    std::vector<char> md;
    for (Run* R : m) md.push_back(R->mixed ? 1 : 0);
    // a mixed run that fell back to FP64 changes its step kernels
    if (s >= 0 && (m != L.members || md != L.modes)) {
      // (re)capture the step graph for this set
      if (L.exec) { cudaGraphExecDestroy(L.exec); L.exec = nullptr; }
      L.members.clear();
      s = lockstep_desc<float2>(L, m, L.d64, &nd64, &ncta64, st);
      if (s >= 0) s = lockstep_desc<double2>(L, m, L.d128, &nd128, &ncta128, st);
      if (s >= 0) {
        GmresDev** sp = reinterpret_cast<GmresDev**>(L.done_dev.as<char>() + flags_off(m.size()));
        std::vector<GmresDev*> hs;
        for (Run* R : m) hs.push_back(R->P->kry->state.as<GmresDev>());
        if (cudaMemcpyAsync(sp, hs.data(), sizeof(GmresDev*) * hs.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
          set_error("lockstep: descriptor upload failed");
          s = VIE_ECUDA;
        }
      }
      if (s >= 0 && !prof_enabled()) {
        // one step as a graph: its kernels read j and the stop flags from
        // device memory, so the same graph serves every step of the set
        cudaGraph_t graph;
        cudaError_t cb = cudaStreamBeginCapture(L.cap, cudaStreamCaptureModeRelaxed);
        if (cb != cudaSuccess) {
          set_error("graph capture: %s", cudaGetErrorString(cb));
          s = VIE_ECUDA;
        } else {
          const long long before = launches_thread();
          s = lockstep_enqueue(L, m, L.cap, nd64, ncta64, nd128, ncta128);
          L.step_launches = (int)(launches_thread() - before);
          count_launch(-L.step_launches);
          cudaError_t ce = cudaStreamEndCapture(L.cap, &graph);
          if (s >= 0 && ce != cudaSuccess) { set_error("graph capture: %s", cudaGetErrorString(ce)); s = VIE_ECUDA; }
          if (s >= 0) {
            cudaError_t ie = cudaGraphInstantiate(&L.exec, graph, 0);
            if (ie != cudaSuccess) { set_error("graph instantiate: %s", cudaGetErrorString(ie)); s = VIE_ECUDA; }
          }
          if (ce == cudaSuccess) cudaGraphDestroy(graph);
        }
      }
      if (s >= 0) {
        L.members = m;
        L.modes = md;
      }
    }
    if (s < 0) {
      for (Run* R : m) run_fail(*R, s);
      return true;
    }
    // every member's own stream is idle here (its cycle start was enqueued
    // there): order the step graph after it
    for (Run* R : m) {
      if (cudaEventRecord(L.ev_root, R->P->st) != cudaSuccess || cudaStreamWaitEvent(st, L.ev_root, 0) != cudaSuccess) {
        s = VIE_ECUDA;
        set_error("lockstep: stream ordering failed");
      }
    }
    // run steps in chunks, polling the stop flags
    int chunk = 4;
    for (Run* R : m) chunk = std::min(chunk, R->cyc_len - R->steps);
    chunk = std::max(chunk, 1);
    for (int c = 0; c < chunk && s >= 0; ++c) {
      if (prof_enabled()) s = lockstep_enqueue(L, m, st, nd64, ncta64, nd128, ncta128);
      else if (cudaGraphLaunch(L.exec, st) != cudaSuccess) { s = VIE_ECUDA; set_error("graph launch failed"); }
      else count_launch(L.step_launches);
    }
    int* dd = L.done_dev.as<int>();
    GmresDev** sp = reinterpret_cast<GmresDev**>(L.done_dev.as<char>() + flags_off(m.size()));
    if (s >= 0) {
      k_gather_done<<<1, 128, 0, st>>>(sp, (int)m.size(), dd);
      count_launch();
      if (cudaMemcpyAsync(L.done_host, dd, sizeof(int) * m.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        s = VIE_ECUDA;
        set_error("lockstep: stop-flag poll failed: %s", cudaGetErrorString(cudaGetLastError()));
      }
    }
    if (s < 0) {
      for (Run* R : m) run_fail(*R, s);
      return true;
    }
    for (size_t i = 0; i < m.size(); ++i) {
      Run& R = *m[i];
      R.steps += chunk;
      if (!L.done_host[i] && R.steps < R.cyc_len) continue;
      const vie_status cs = R.mixed ? cycle_end<float2>(R) : cycle_end<double2>(R);
      if (cs < 0) run_fail(R, cs);
    }
  }
  return true;
}

// Advance the runs until all are finished.
static void lockstep_drive(Lockstep& L, std::vector<Run*>& runs, cudaStream_t st) {
  while (lockstep_pass_impl(L, runs, st)) {
  }
}

// --- interface for the server (api.cu) ---
Run* run_new(vie_plan_s* P, const double2* e_inc, double2* w_out, vie_info* info) {
  Run* R = new Run();
  R->P = P;
  R->e_inc = e_inc;
  R->w_out = w_out;
  R->info = info;
  return R;
}
void run_delete(Run* R) { delete R; }
vie_status run_start(Run* R) {
  vie_status s;
  {
    AllocScope a(R->P->st);
    s = run_begin(*R);
  }
  if (s < 0) run_fail(*R, s);
  return s;
}
bool run_finished(const Run* R) { return R->finished; }
void run_abort(Run* R, const char* why) {
  set_error("%s", why);
  run_fail(*R, VIE_ECUDA);
}
vie_status run_status(const Run* R, std::string* err) {
  if (err) *err = R->err;
  return R->status;
}
vie_plan_s* run_plan(const Run* R) { return R->P; }
Lockstep* lockstep_new() { return new Lockstep(); }
bool lockstep_pass(Lockstep* L, std::vector<Run*>& runs, cudaStream_t st) { return lockstep_pass_impl(*L, runs, st); }
void lockstep_release(Lockstep* L) { L->release(); }

void reset_graphs(vie_plan_s* P) {
  if (!P->kry || !P->kry->lock) return;
  Lockstep& L = *P->kry->lock;
  if (L.exec) { cudaGraphExecDestroy(L.exec); L.exec = nullptr; }
  L.members.clear();
}

// One solve: a lockstep set of one run, on the plan's stream.
vie_status solve(vie_plan_s* P, const double2* e_inc, double2* w_out, vie_info* info) {
  Run R;
  R.P = P;
  R.e_inc = e_inc;
  R.w_out = w_out;
  R.info = info;
  vie_status s = run_begin(R);
  if (s < 0) return s;
  if (!R.finished) {
    Krylov& K = *P->kry;
    if (!K.lock) K.lock.reset(new Lockstep());
    std::vector<Run*> runs{&R};
    // the graph holds the plan's buffers: recapture when the set changes
    reset_graphs(P);
    lockstep_drive(*K.lock, runs, P->st);
    if (R.status < 0) {
      set_error("%s", R.err.c_str());
      return R.status;
    }
  }
  return R.status;
}

// Several solves in lockstep (plans on the current device; each plan's own
// stream carries its host-side work, the step graphs run on st, whose
// allocations scope is active).  status[i] receives each run's status.
vie_status solve_many(vie_plan_s* const* P, int n, const double2* const* e_inc, double2* const* w_out,
                      vie_info* info, vie_status* status, cudaStream_t st) {
  std::vector<Run> runs(n);
  std::vector<Run*> ptr;
  for (int i = 0; i < n; ++i) {
    Run& R = runs[i];
    R.P = P[i];
    R.e_inc = e_inc[i];
    R.w_out = w_out[i];
    R.info = info ? info + i : nullptr;
    vie_status s;
    {
      AllocScope a(R.P->st);   // the plan's buffers live on the plan's stream
      s = run_begin(R);
    }
    if (s < 0) run_fail(R, s);
    ptr.push_back(&R);
  }
  {
    Lockstep L;
    lockstep_drive(L, ptr, st);
    cudaStreamSynchronize(st);
    L.release();
  }
  vie_status worst = VIE_OK;
  for (int i = 0; i < n; ++i) {
    status[i] = runs[i].status;
    if (runs[i].status < 0 && (worst >= 0 || runs[i].status < worst)) {
      worst = runs[i].status;
      set_error("%s", runs[i].err.c_str());
    } else if (worst == VIE_OK && runs[i].status > 0) {
      worst = runs[i].status;
    }
  }
  return worst;
}

}  // namespace vie
