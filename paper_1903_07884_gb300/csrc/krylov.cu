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

struct Krylov {
  int restart = 0;
  long long n3 = 0;
  long long ld = 0;               // column stride of the basis (n3 rounded up to 32)
  DevBuf V64, V128;               // (restart + 1) * ld basis
  DevBuf u64, u128, z64, z128, w64, w128;
  DevBuf partial;                 // double2 [NPART][PST]
  DevBuf state;                   // GmresDev
  DevBuf x128, r128, b128, d64, rhs64, r64, t128;
  DevBuf xbest;                   // best iterate of a multi-cycle solve (allocated on first use)
  DevBuf scal;                    // double [8]: norms
  int* hflag = nullptr;           // pinned host mirror: done, iters
  cudaGraphExec_t g64 = nullptr, g128 = nullptr;
  int step_launches = 0;
  cudaEvent_t ev = nullptr;
  cudaStream_t cap = nullptr;     // private stream for graph capture
  ~Krylov() {
    if (cap) cudaStreamDestroy(cap);
    if (g64) cudaGraphExecDestroy(g64);
    if (g128) cudaGraphExecDestroy(g128);
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

// As givens_column, run by one warp (lane 0 takes the sequential chain), so
// that the rest of the block can work meanwhile.
__device__ void givens_column_warp(GmresDev* __restrict__ s, int jc) {
  __shared__ double2 colw[RMAX + 1];
  __shared__ double csw[RMAX];
  __shared__ double2 snw[RMAX];
  const int lane = threadIdx.x & 31;
  const double2* hr = s->Hr + (long long)jc * (RMAX + 1);
  for (int i = lane; i <= jc + 1; i += 32) colw[i] = hr[i];
  for (int i = lane; i < jc; i += 32) { csw[i] = s->cs[i]; snw[i] = s->sn[i]; }
  __syncwarp();
  if (lane == 0) {
    for (int i = 0; i < jc; ++i) {
      const double2 a = colw[i], b = colw[i + 1];
      const double c = csw[i];
      const double2 sn = snw[i];
      colw[i] = make_double2(c * a.x + (sn.x * b.x - sn.y * b.y), c * a.y + (sn.x * b.y + sn.y * b.x));
      colw[i + 1] = make_double2(-(sn.x * a.x + sn.y * a.y) + c * b.x, -(sn.x * a.y - sn.y * a.x) + c * b.y);
    }
    const double2 a = colw[jc];
    const double2 bb = colw[jc + 1];
    const double b = sqrt(bb.x * bb.x + bb.y * bb.y);
    double c;
    double2 sn;
    const double aa = sqrt(a.x * a.x + a.y * a.y);
    if (b == 0.0) { c = 1.0; sn = make_double2(0, 0); }
    else if (aa == 0.0) { c = 0.0; sn = make_double2(1.0, 0.0); }
    else {
      const double r = hypot(aa, b);
      c = aa / r;
      sn = make_double2(a.x * b / (aa * r), a.y * b / (aa * r));
    }
    s->cs[jc] = c;
    s->sn[jc] = sn;
    colw[jc] = make_double2(c * a.x + sn.x * b, c * a.y + sn.y * b);
    colw[jc + 1] = make_double2(0, 0);
    const double2 gj = s->g[jc];
    const double2 g1 = make_double2(-(sn.x * gj.x + sn.y * gj.y), -(sn.x * gj.y - sn.y * gj.x));
    s->g[jc + 1] = g1;
    s->g[jc] = make_double2(c * gj.x, c * gj.y);
    s->resest = sqrt(g1.x * g1.x + g1.y * g1.y);
  }
  __syncwarp();
  double2* H = s->H + (long long)jc * (RMAX + 1);
  for (int i = lane; i <= jc + 1; i += 32) H[i] = colw[i];
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
// Arnoldi passes over the basis (columns of stride ld, a multiple of 32
// elements).  Each block owns a contiguous range of the vector cut into
// sub-chunks of at most SUB_BYTES; per sub-chunk a thread visits the same KPT
// elements of w, u_j = V_j and V_0 .. V_{j-1} in that order, reading them with
// coalesced loads, several columns at a time so that enough loads are in
// flight.  (A variant that streamed the columns into a ring of shared-memory
// tiles with cp.async.bulk and mbarriers gave run-to-run different results
// when several plans shared the GPU; the direct reads are deterministic.)
// ---------------------------------------------------------------------------
constexpr int SUB_BYTES = 16384;                // bytes of one column per sub-chunk
constexpr int ST_CONS = 512;                    // threads doing the arithmetic
constexpr int ST_THREADS = ST_CONS;
constexpr int UPD_THREADS = ST_CONS + 32;       // k_update: + one warp for the Hessenberg bookkeeping

struct StreamGeom {
  long long c0, c1;   // the block's element range
  int nsub, sc;       // sub-chunks and elements per sub-chunk (multiple of 32)
};

// (32-bit arithmetic: vectors hold fewer than 2^31 elements, checked at plan
// creation, and a 64-bit division would run as an FP64 subroutine)
template <class C>
__device__ __forceinline__ StreamGeom stream_geom(long long n3) {
  const unsigned n = (unsigned)n3;
  const unsigned per = ((n + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
  StreamGeom g;
  const unsigned c0 = min(n, blockIdx.x * per), c1 = min(n, c0 + per);
  g.c0 = c0;
  g.c1 = c1;
  const unsigned maxe = SUB_BYTES / (unsigned)sizeof(C);
  const unsigned len = c1 - c0;
  g.nsub = (int)((len + maxe - 1) / maxe);
  g.sc = g.nsub > 0 ? (int)(((len + (unsigned)g.nsub - 1) / (unsigned)g.nsub + 31) / 32 * 32) : 0;
  return g;
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
// Reduction: tiles per sub-chunk are w, u_j = V_j, then V_0 .. V_{j-1}; a
// consumer keeps its elements of w and u_j in registers and accumulates four
// columns (two complex dots each) at a time, reduced over the warp by a
// butterfly into the warp's row of shared memory.  Partials per block:
// [i] = (s_i or alpha at i = j), [RMAX + 1 + i] = (z_i or zeta at i = j).
template <class C>
__global__ void __launch_bounds__(ST_THREADS) k_dot_partial(const C* __restrict__ V, long long ld,
                                                            const C* __restrict__ w, long long n3,
                                                            GmresDev* __restrict__ s, double2* __restrict__ partial) {
  using T = typename Acc<C>::T;
  constexpr int KPT = SUB_BYTES / (int)sizeof(C) / ST_CONS;   // elements per thread per sub-chunk
  constexpr int ROW = 4 * (RMAX + 1) + 4;                     // per warp: s (2 per column), z (2), alpha, zeta
  extern __shared__ __align__(16) unsigned char dot_smem[];
  T* wsum = reinterpret_cast<T*>(dot_smem);                   // [16][ROW]
  if (s->done) return;
  const int j = s->j;
  const StreamGeom g = stream_geom<C>(n3);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ct = threadIdx.x;
  T* my = wsum + (size_t)warp * ROW;
  for (int i = lane; i < ROW; i += 32) my[i] = 0;
  __syncwarp();
  T al = 0, zr = 0, zi = 0;
  for (int sb = 0; sb < g.nsub; ++sb) {
    const long long start = g.c0 + (long long)sb * g.sc;
    const int cnt = (int)min((long long)g.sc, g.c1 - start);
    const C* wv = w + start;
    const C* uv = V + (long long)j * ld + start;
    C xw[KPT], xu[KPT];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const int e = ct + q * ST_CONS;
      xw[q] = e < cnt ? wv[e] : czero<C>();
      xu[q] = e < cnt ? uv[e] : czero<C>();
      al += xu[q].x * xu[q].x + xu[q].y * xu[q].y;
      zr += xu[q].x * xw[q].x + xu[q].y * xw[q].y;
      zi += xu[q].x * xw[q].y - xu[q].y * xw[q].x;
    }
    for (int i0 = 0; i0 < j; i0 += 4) {
      T a[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) a[q] = 0;
      const int nt = min(4, j - i0);
      C v[4][KPT];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const C* col = V + (long long)(i0 + t) * ld + start;
#pragma unroll
        for (int q = 0; q < KPT; ++q) {
          const int e = ct + q * ST_CONS;
          v[t][q] = (t < nt && e < cnt) ? col[e] : czero<C>();
        }
      }
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
      const int q = lane >> 1, col = i0 + (q >> 2), part = q & 3;
      if ((lane & 1) == 0 && (q >> 2) < nt) my[(part < 2 ? 0 : 2 * (RMAX + 1)) + 2 * col + (part & 1)] += r;
      __syncwarp();
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    zr += __shfl_xor_sync(0xffffffffu, zr, o);
    zi += __shfl_xor_sync(0xffffffffu, zi, o);
  }
  if (lane == 0) { my[4 * (RMAX + 1)] = al; my[4 * (RMAX + 1) + 1] = zr; my[4 * (RMAX + 1) + 2] = zi; }
  __syncthreads();
  // block sums over the consumer warps.  Partials and the scalar work of the
  // last block stay in the accumulator precision (FP32 for a complex-FP32
  // basis): FP64 issues at a small fraction of the FP32 rate on this part,
  // and the tail runs on one SM while the others wait.  The Hessenberg
  // matrix itself is stored in FP64.
  C* pc = reinterpret_cast<C*>(partial);
  C* pb = pc + (long long)blockIdx.x * PST;
  for (int v = threadIdx.x; v < 2 * (j + 1); v += blockDim.x) {
    // v < j: s_v; v == j: alpha; v = j + 1 + i: z_i; v = 2 j + 1: zeta
    int sr, si, dst;
    if (v < j) { sr = 2 * v; si = sr + 1; dst = v; }
    else if (v == j) { sr = 4 * (RMAX + 1); si = -1; dst = j; }
    else if (v < 2 * j + 1) { sr = 2 * (RMAX + 1) + 2 * (v - j - 1); si = sr + 1; dst = RMAX + 1 + (v - j - 1); }
    else { sr = 4 * (RMAX + 1) + 1; si = sr + 1; dst = RMAX + 1 + j; }
    T re = 0, im = 0;
    for (int w2 = 0; w2 < ST_CONS / 32; ++w2) {
      re += wsum[(size_t)w2 * ROW + sr];
      if (si >= 0) im += wsum[(size_t)w2 * ROW + si];
    }
    pb[dst] = cmake<C>(re, im);
  }
  // the last block: s, z, beta, t, the final column j - 1 and the tentative
  // column j, the update coefficients
  GmresDev* sm = const_cast<GmresDev*>(s);
  if (!last_block(&sm->arrive_dot)) return;
  __shared__ C sv[RMAX + 1], zv[RMAX + 1];
  __shared__ T sc_beta, sc_t[2];
  const int nw = blockDim.x >> 5;
  for (int i = warp; i <= j; i += nw) {
    // s_i and z_i together: every lane keeps all its loads in flight
    C a = czero<C>(), b = czero<C>();
    C pa[(NPART + 31) / 32], pz[(NPART + 31) / 32];
#pragma unroll
    for (int q = 0; q < (NPART + 31) / 32; ++q) {
      const int bk = lane + 32 * q;
      pa[q] = bk < (int)gridDim.x ? __ldcg(pc + (long long)bk * PST + i) : czero<C>();
      pz[q] = bk < (int)gridDim.x ? __ldcg(pc + (long long)bk * PST + RMAX + 1 + i) : czero<C>();
    }
#pragma unroll
    for (int q = 0; q < (NPART + 31) / 32; ++q) { a.x += pa[q].x; a.y += pa[q].y; b.x += pz[q].x; b.y += pz[q].y; }
    for (int o = 16; o > 0; o >>= 1) {
      a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
      a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
      b.x += __shfl_xor_sync(0xffffffffu, b.x, o);
      b.y += __shfl_xor_sync(0xffffffffu, b.y, o);
    }
    if (lane == 0) { sv[i] = a; zv[i] = b; }
  }
  __syncthreads();
  // beta^2 = alpha - |s|^2 (warp 0) and s^H z (warp 1), lane-strided with a butterfly
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
  const T beta = sc_beta;
  const T ib = (T)1 / beta;
  const C t = cmake<C>(sc_t[0] * ib, sc_t[1] * ib);   // t = (zeta - s^H z) / beta
  if (j > 0) {   // column j - 1 becomes final: h_{:,j-1} += nu s, h_{j,j-1} = nu beta
    const double nu = sm->nu;
    double2* hp = sm->Hr + (long long)(j - 1) * (RMAX + 1);
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      hp[i].x += nu * (double)sv[i].x;
      hp[i].y += nu * (double)sv[i].y;
    }
    if (threadIdx.x == 0) hp[j] = make_double2(nu * (double)beta, 0.0);
  }
  __syncthreads();
  // tentative column j: rows 0..j of ([z; t] - H_{0:j,0:j-1} s) / beta, one
  // warp per row, lanes over the columns
  for (int r = warp; r <= j; r += nw) {
    T ar = 0, ai = 0;
    for (int l = max(r - 1, 0) + lane; l < j; l += 32) {   // H[r][l] = 0 for r > l + 1
      const double2 hd = sm->Hr[(long long)l * (RMAX + 1) + r];
      const T hx = (T)hd.x, hy = (T)hd.y;
      ar += hx * sv[l].x - hy * sv[l].y;
      ai += hx * sv[l].y + hy * sv[l].x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) {
      const C zr = r < j ? zv[r] : t;
      sm->Hr[(long long)j * (RMAX + 1) + r] = make_double2((double)((zr.x - ar) * ib), (double)((zr.y - ai) * ib));
    }
  }
  // update coefficients: s, c = z - s t / beta, cu = t / beta, 1 / beta; the
  // rotation of column j - 1 (a sequential chain) and the stop test run beside
  // the update (k_update, block 0), off this kernel's critical path
  const C tb = cmake<C>(t.x * ib, t.y * ib);
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    const C si = sv[i], zi = zv[i];
    sm->cs_s[i] = make_double2((double)si.x, (double)si.y);
    sm->cs_c[i] = make_double2((double)(zi.x - (si.x * tb.x - si.y * tb.y)), (double)(zi.y - (si.x * tb.y + si.y * tb.x)));
  }
  if (threadIdx.x == 0) {
    sm->cu = make_double2((double)tb.x, (double)tb.y);
    sm->inv_beta = (double)ib;
    sm->reorths += (j > 0) ? 1 : 0;
  }
}


// Hessenberg bookkeeping of step j, run by one warp of block 0 of k_update
// while the other warps stream: the rotation of the now final column j - 1
// and the stop test on the residual estimate it gives.
__device__ void hessenberg_side(GmresDev* __restrict__ s, int j) {
  if (j == 0) return;
  givens_column_warp(s, j - 1);
  if ((threadIdx.x & 31) == 0) {
    s->k = j;
    if (s->resest <= s->tol_abs || j >= s->restart) s->done = 1;
  }
}

// q_j = (u_j - Q s) / beta into V_j and w'' = (w - Q c - cu u_j) / beta into
// w, streamed like the reduction (tiles w, u_j, V_0 .. V_{j-1}); then ||w''||
// as h_{j+1,j} (tentative) and the scale of u_{j+1}.
template <class C>
__global__ void __launch_bounds__(UPD_THREADS) k_update(C* __restrict__ V, long long ld, C* __restrict__ w,
                                                       long long n3, GmresDev* __restrict__ s,
                                                       double2* __restrict__ partial) {
  using T = typename Acc<C>::T;
  constexpr int KPT = SUB_BYTES / (int)sizeof(C) / ST_CONS;
  __shared__ C sco[RMAX + 1], cco[RMAX + 1];
  __shared__ T shn[UPD_THREADS / 32];
  if (s->done) return;
  const int j = s->j;
  for (int i = threadIdx.x; i < j; i += blockDim.x) { sco[i] = cconv<C>(s->cs_s[i]); cco[i] = cconv<C>(s->cs_c[i]); }
  const C cu = cconv<C>(s->cu);
  using R = typename real_of<C>::type;
  const R ib = (R)s->inv_beta;
  const StreamGeom g = stream_geom<C>(n3);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  T nrm = 0;
  if (warp == ST_CONS / 32) {
    if (blockIdx.x == 0) hessenberg_side(const_cast<GmresDev*>(s), j);
  } else {
    const int ct = threadIdx.x;
    C* Vj = V + (long long)j * ld;
    for (int sb = 0; sb < g.nsub; ++sb) {
      const long long start = g.c0 + (long long)sb * g.sc;
      const int cnt = (int)min((long long)g.sc, g.c1 - start);
      C xw[KPT], xu[KPT], as[KPT], ac[KPT];
#pragma unroll
      for (int q = 0; q < KPT; ++q) {
        const int e = ct + q * ST_CONS;
        xw[q] = e < cnt ? w[start + e] : czero<C>();
        xu[q] = e < cnt ? Vj[start + e] : czero<C>();
        as[q] = czero<C>();
        ac[q] = czero<C>();
      }
      for (int i0 = 0; i0 < j; i0 += 4) {
        const int nt = min(4, j - i0);
        C v[4][KPT];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const C* col = V + (long long)(i0 + t) * ld + start;
#pragma unroll
          for (int q = 0; q < KPT; ++q) {
            const int e = ct + q * ST_CONS;
            v[t][q] = (t < nt && e < cnt) ? col[e] : czero<C>();
          }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const C hs = t < nt ? sco[i0 + t] : czero<C>(), hc = t < nt ? cco[i0 + t] : czero<C>();
#pragma unroll
          for (int q = 0; q < KPT; ++q) {
            cfma(as[q], hs, v[t][q]);
            cfma(ac[q], hc, v[t][q]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < KPT; ++q) {
        const int e = ct + q * ST_CONS;
        if (e < cnt) {
          const C qj = cmake<C>((xu[q].x - as[q].x) * ib, (xu[q].y - as[q].y) * ib);
          C x = csub(xw[q], ac[q]);
          x.x -= cu.x * xu[q].x - cu.y * xu[q].y;
          x.y -= cu.x * xu[q].y + cu.y * xu[q].x;
          x.x *= ib;
          x.y *= ib;
          Vj[start + e] = qj;
          w[start + e] = x;
          nrm += x.x * x.x + x.y * x.y;
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (lane == 0) shn[warp] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = 0;
    for (int w2 = 0; w2 < UPD_THREADS / 32; ++w2) t += shn[w2];
    partial[(long long)blockIdx.x * PST] = make_double2((double)t, 0.0);
  }
  GmresDev* sm = const_cast<GmresDev*>(s);
  if (!last_block(&sm->arrive_upd)) return;
  __shared__ double nn_s;
  if (warp == 0) {
    const double nn = warp_sum_partials_cg(partial, gridDim.x, 0).x;
    if (lane == 0) nn_s = nn;
  }
  __syncthreads();
  const double nu = sqrt(nn_s);
  if (threadIdx.x == 0) {
    sm->nu = nu;
    sm->Hr[(long long)j * (RMAX + 1) + j + 1] = make_double2(nu, 0.0);
    sm->hnext = nu;
    sm->inv_next = nu > 0.0 ? 1.0 / nu : 0.0;
    sm->inv_next32 = (float)sm->inv_next;
    sm->iters += 1;
  }
  if (nu == 0.0) {
    // breakdown: the Krylov space is invariant and column j is already final
    __syncthreads();
    givens_column(sm, j);
    if (threadIdx.x == 0) { sm->k = j + 1; sm->done = 1; }
    return;
  }
  if (threadIdx.x == 0) sm->j = j + 1;
}

// V_{j} = w / h (j already advanced) and u = V_j
template <class C>
__global__ void k_scale_next(C* __restrict__ V, long long ld, const C* __restrict__ w, C* __restrict__ u,
                             long long n3, const GmresDev* __restrict__ s) {
  if (s->done) return;
  const int j = s->j;
  using T = typename real_of<C>::type;
  const T inv = sizeof(T) == 4 ? (T)s->inv_next32 : (T)s->inv_next;   // reciprocal in the vector precision
  C* Vj = V + (long long)j * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x) {
    const C v = cscale(w[e], inv);
    Vj[e] = v;
    u[e] = v;
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

// x += scale * z   (x FP64, z any precision)
template <class C>
__global__ void k_axpy_to64(double2* __restrict__ x, const C* __restrict__ z, long long n3, const double* __restrict__ sc,
                            int sidx) {
  const double a = sc ? sc[sidx] : 1.0;
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
  static cudaGraphExec_t& g(Krylov& K) { return K.g64; }
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
  static cudaGraphExec_t& g(Krylov& K) { return K.g128; }
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

static vie_status krylov_alloc(vie_plan_s* P, bool need64, bool need128) {
  if (!P->kry) P->kry.reset(new Krylov());
  Krylov& K = *P->kry;
  const long long n3 = 3LL * P->nx * P->ny * P->nz;
  const int R = P->opts.restart;
  K.restart = R;
  K.n3 = n3;
  K.ld = (n3 + 31) / 32 * 32;
  const long long ld = K.ld;
  if (!K.state.p) {
    VIE_TRY(K.state.alloc(sizeof(GmresDev)));
    // stream-ordered like the allocation (a legacy-stream memset would not be
    // ordered with the plan's non-blocking stream)
    VIE_CUDA(cudaMemsetAsync(K.state.p, 0, sizeof(GmresDev), P->st));
    VIE_TRY(K.partial.alloc(sizeof(double2) * NPART * PST));
    VIE_TRY(K.scal.alloc(sizeof(double) * 8));
    VIE_TRY(K.x128.alloc(sizeof(double2) * n3));
    VIE_TRY(K.r128.alloc(sizeof(double2) * n3));
    VIE_TRY(K.b128.alloc(sizeof(double2) * n3));
    VIE_TRY(K.t128.alloc(sizeof(double2) * n3));
    VIE_CUDA(cudaHostAlloc((void**)&K.hflag, sizeof(int) * 4, cudaHostAllocDefault));
    VIE_CUDA(cudaEventCreateWithFlags(&K.ev, cudaEventDisableTiming));
    VIE_CUDA(cudaStreamCreateWithFlags(&K.cap, cudaStreamNonBlocking));
  }
  if (need64 && !K.V64.p) {
    VIE_TRY(K.V64.alloc(sizeof(float2) * ld * (R + 1)));
    VIE_TRY(K.u64.alloc(sizeof(float2) * n3));
    VIE_TRY(K.z64.alloc(sizeof(float2) * n3));
    VIE_TRY(K.w64.alloc(sizeof(float2) * ld));
    VIE_TRY(K.d64.alloc(sizeof(float2) * n3));
    VIE_TRY(K.rhs64.alloc(sizeof(float2) * n3));
    VIE_TRY(K.r64.alloc(sizeof(float2) * n3));
  }
  if (need128 && !K.V128.p) {
    VIE_TRY(K.V128.alloc(sizeof(double2) * ld * (R + 1)));
    VIE_TRY(K.u128.alloc(sizeof(double2) * n3));
    VIE_TRY(K.z128.alloc(sizeof(double2) * n3));
    VIE_TRY(K.w128.alloc(sizeof(double2) * ld));
  }
  return VIE_OK;
}

// kernels in one captured Arnoldi step (for launch accounting)
static int step_kernels(vie_plan_s* P) {
  Krylov& K = *P->kry;
  return K.step_launches;
}

template <class C>
static size_t dot_smem() {
  return (size_t)(ST_CONS / 32) * (4 * (RMAX + 1) + 4) * sizeof(typename Acc<C>::T);
}

// enqueue one Arnoldi step (u holds u_j on entry and u_{j+1} on exit)
template <class C>
static vie_status enqueue_step(vie_plan_s* P) {
  Krylov& K = *P->kry;
  cudaStream_t st = P->st;
  GmresDev* s = K.state.as<GmresDev>();
  double2* part = K.partial.as<double2>();
  C* V = KB<C>::V(K);
  C* u = KB<C>::u(K);
  C* z = KB<C>::z(K);
  C* w = KB<C>::w(K);
  const long long n3 = K.n3;
  VIE_TRY(smem_optin(k_dot_partial<C>, dot_smem<C>()));
  VIE_TRY(op_Pinv<C>(P, u, z));
  VIE_TRY(op_A<C>(P, z, w));
  // delayed CGS2: one reduction (s, z and the Hessenberg bookkeeping in its
  // last block) and one update (q_j, w'' and ||w''|| in its last block)
  {
    Prof pf_(sizeof(C) == 8 ? "arnoldi_dot_c64" : "arnoldi_dot_c128", st);
    k_dot_partial<C><<<NPART, ST_THREADS, dot_smem<C>(), st>>>(V, K.ld, w, n3, s, part);
  }
  {
    Prof pf_(sizeof(C) == 8 ? "arnoldi_update_c64" : "arnoldi_update_c128", st);
    k_update<C><<<NPART, UPD_THREADS, 0, st>>>(V, K.ld, w, n3, s, part);
  }
  count_launch(2);
  { Prof pf_("arnoldi_scale", st); k_scale_next<C><<<grid_for(n3), 256, 0, st>>>(V, K.ld, w, u, n3, s); }
  count_launch(1);
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

// Run GMRES cycles on A x = rhs (precision C) from x = 0, accumulating the
// solution into x (C).  Stops when the true relative residual (rhs - A x,
// precision C) is <= tol, or after max_iter steps.  Returns the steps used
// through *iters and the last true relative residual through *relres.
template <class C>
static vie_status gmres(vie_plan_s* P, const C* rhs, C* x, C* rwork, double tol, int max_iter, int max_cycles,
                        int* iters, double* relres) {
  Krylov& K = *P->kry;
  cudaStream_t st = P->st;
  GmresDev* s = K.state.as<GmresDev>();
  double2* part = K.partial.as<double2>();
  const long long n3 = K.n3;
  C* V = KB<C>::V(K);
  C* u = KB<C>::u(K);
  C* z = KB<C>::z(K);
  C* w = KB<C>::w(K);
  double* scal = K.scal.as<double>();
  // ||rhs||
  k_norm_partial<C><<<NPART, RED_THREADS, 0, st>>>(rhs, n3, part);
  k_norm_final<<<1, 32, 0, st>>>(part, NPART, scal, 0);
  VIE_CUDA(cudaMemsetAsync(x, 0, sizeof(C) * n3, st));
  VIE_CUDA(cudaMemcpyAsync(rwork, rhs, sizeof(C) * n3, cudaMemcpyDeviceToDevice, st));
  count_launch(2);
  double hsc[2];
  VIE_CUDA(cudaMemcpyAsync(hsc, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  VIE_CUDA(cudaStreamSynchronize(st));
  const double bnorm = hsc[0];
  *iters = 0;
  *relres = 0;
  if (bnorm == 0.0) return VIE_OK;
  cudaGraphExec_t& gexec = KB<C>::g(K);
  int total = 0, cycles = 0;
  double rr = 1.0, rr_best = 1.0;   // x0 = 0 has the residual ||b||
  int stalls = 0;
  bool have_best = false;
  C* xb = nullptr;
  if (max_cycles > 1) {
    if (K.xbest.bytes < sizeof(C) * n3) VIE_TRY(K.xbest.alloc(sizeof(C) * n3));
    xb = K.xbest.as<C>();
  }
  while (total < max_iter) {
    // cycle start from the current residual rwork
    k_norm_partial<C><<<NPART, RED_THREADS, 0, st>>>(rwork, n3, part);
    k_cycle_init<<<1, 32, 0, st>>>(s, part, NPART, tol * bnorm, std::min(K.restart, max_iter - total));
    k_cycle_v0<C><<<grid_for(n3), 256, 0, st>>>(rwork, V, u, n3, s);
    count_launch(3);
    VIE_CHECK_LAUNCH();
    if (!gexec && !prof_enabled()) {
      // one Arnoldi step as a graph: its kernels read j and the stop flag
      // from device memory, so the same graph serves every step
      // capture on a private stream (the plan stream may be the legacy
      // default stream, which cannot be captured); the graph is launched on
      // the plan stream
      cudaGraph_t graph;
      VIE_CUDA(cudaStreamSynchronize(st));
      P->st = K.cap;
      cudaError_t cb = cudaStreamBeginCapture(K.cap, cudaStreamCaptureModeRelaxed);
      if (cb != cudaSuccess) { P->st = st; set_error("graph capture: %s", cudaGetErrorString(cb)); return VIE_ECUDA; }
      const long long before = launches_total();
      vie_status es = enqueue_step<C>(P);
      K.step_launches = (int)(launches_total() - before);
      count_launch(-K.step_launches);
      cudaError_t ce = cudaStreamEndCapture(K.cap, &graph);
      P->st = st;
      if (es < 0) return es;
      if (ce != cudaSuccess) { set_error("graph capture: %s", cudaGetErrorString(ce)); return VIE_ECUDA; }
      VIE_CUDA(cudaGraphInstantiate(&gexec, graph, 0));
      cudaGraphDestroy(graph);
    }
    // run steps in chunks, polling the stop flag
    int done = 0, steps_cycle = 0;
    // restart columns take restart + 1 steps: the last reduction finalises the last column
    const int cyc = std::min(K.restart, max_iter - total) + 1;
    while (!done && steps_cycle < cyc) {
      const int chunk = std::min(4, cyc - steps_cycle);
      if (prof_enabled()) {
        for (int c = 0; c < chunk; ++c) VIE_TRY(enqueue_step<C>(P));
      } else {
        for (int c = 0; c < chunk; ++c) VIE_CUDA(cudaGraphLaunch(gexec, st));
        count_launch(chunk * step_kernels(P));
      }
      steps_cycle += chunk;
      VIE_CUDA(cudaMemcpyAsync(K.hflag, &s->done, sizeof(int), cudaMemcpyDeviceToHost, st));
      VIE_CUDA(cudaMemcpyAsync(K.hflag + 1, &s->iters, sizeof(int), cudaMemcpyDeviceToHost, st));
      VIE_CUDA(cudaStreamSynchronize(st));
      done = K.hflag[0];
    }
    int hk = 0;
    VIE_CUDA(cudaMemcpyAsync(&hk, &s->k, sizeof(int), cudaMemcpyDeviceToHost, st));
    // x += P^-1 (V y)
    {
      const size_t smem = sizeof(double2) * (size_t)K.restart * (K.restart + 1) / 2;
      VIE_TRY(smem_optin(k_solve_y, smem));
      k_solve_y<<<1, SOLVE_THREADS, smem, st>>>(s);
    }
    k_combine<C><<<grid_for(n3), 256, 0, st>>>(V, K.ld, u, n3, s);
    count_launch(2);
    VIE_TRY(op_Pinv<C>(P, u, z));
    VIE_TRY(axpy_same<C>(x, z, n3, st));
    if (++cycles >= max_cycles) {
      // the caller evaluates the residual itself (in higher precision)
      VIE_CUDA(cudaStreamSynchronize(st));
      total += hk;
      rr = -1.0;
      break;
    }
    // true residual rwork = rhs - A x
    VIE_TRY(op_A<C>(P, x, w));
    VIE_TRY(sub_same<C>(rhs, w, rwork, n3, st));
    k_norm_partial<C><<<NPART, RED_THREADS, 0, st>>>(rwork, n3, part);
    k_norm_final<<<1, 32, 0, st>>>(part, NPART, scal, 1);
    count_launch(2);
    VIE_CUDA(cudaMemcpyAsync(hsc + 1, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    VIE_CUDA(cudaStreamSynchronize(st));
    VIE_CHECK_LAUNCH();
    total += hk;
    rr = hsc[1] / bnorm;
    if (rr <= tol || hk == 0) break;
    // a cycle cannot raise the true residual in exact arithmetic (y = 0 is
    // feasible), but on an ill-conditioned operator the basis can lose
    // orthogonality and it does; the next cycle still starts from the new
    // residual (a different Krylov space), and the best iterate is kept
    if (rr < rr_best) {
      VIE_CUDA(cudaMemcpyAsync(xb, x, sizeof(C) * n3, cudaMemcpyDeviceToDevice, st));
      have_best = true;
    }
    // restarted GMRES may converge slowly, but three cycles in a row that
    // do not improve the best residual by 1% mean stagnation (or the
    // rounding floor of this precision): stop and report the residual
    if (rr > 0.99 * rr_best) {
      if (++stalls >= 3) break;
    } else {
      stalls = 0;
    }
    rr_best = std::min(rr, rr_best);
  }
  if (rr > rr_best) {
    // end on the best iterate (x0 = 0 when no cycle went below ||b||)
    if (have_best) VIE_CUDA(cudaMemcpyAsync(x, xb, sizeof(C) * n3, cudaMemcpyDeviceToDevice, st));
    else VIE_CUDA(cudaMemsetAsync(x, 0, sizeof(C) * n3, st));
    VIE_TRY(op_A<C>(P, x, w));
    VIE_TRY(sub_same<C>(rhs, w, rwork, n3, st));
    rr = rr_best;
  }
  *iters = total;
  *relres = rr;
  return VIE_OK;
}


void reset_graphs(vie_plan_s* P) {
  if (!P->kry) return;
  if (P->kry->g64) { cudaGraphExecDestroy(P->kry->g64); P->kry->g64 = nullptr; }
  if (P->kry->g128) { cudaGraphExecDestroy(P->kry->g128); P->kry->g128 = nullptr; }
}

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

// (I - M N) w = M e_inc
vie_status solve(vie_plan_s* P, const double2* e_inc, double2* w_out, vie_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!P->has_eps) { set_error("vie_solve: permittivity not set"); return VIE_ESTATE; }
  const bool mixed = P->opts.precision == VIE_MIXED;
  VIE_TRY(krylov_alloc(P, mixed, !mixed));
  Krylov& K = *P->kry;
  cudaStream_t st = P->st;
  const long long n3 = K.n3;
  const long long N = n3 / 3;
  double2* b = K.b128.as<double2>();
  double2* x = K.x128.as<double2>();
  double2* r = K.r128.as<double2>();
  double2* t = K.t128.as<double2>();
  k_rhs<<<grid_for(n3), 256, 0, st>>>(P->M128.as<double2>(), e_inc, b, N);
  count_launch();
  VIE_CHECK_LAUNCH();
  double bnorm = 0;
  VIE_TRY(norm128(P, b, 2, &bnorm));
  if (!std::isfinite(bnorm)) {
    set_error("vie_solve: non-finite right-hand side (check the permittivity and incident field)");
    return VIE_EINVAL;
  }
  if (!P->prec_built) VIE_TRY(precond_build(P));
  GmresDev* sdev = K.state.as<GmresDev>();
  VIE_CUDA(cudaMemsetAsync(&sdev->reorths, 0, sizeof(int), st));
  int inner = 0, outer = 0;
  double relres = 0;
  const double tol = P->opts.tol;
  if (bnorm == 0.0) {
    VIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * n3, st));
  } else if (!mixed) {
    int it = 0;
    double rr = 0;
    VIE_TRY(gmres<double2>(P, b, x, r, tol, P->opts.max_iter, 1 << 30, &it, &rr));
    inner = it;
    outer = 1;
  } else {
    // GMRES-IR: each refinement step runs one complex-FP32 GMRES cycle on
    // A d = r / ||r|| (stopped early once its Arnoldi residual estimate
    // reaches eta), then x += ||r|| d and r = b - A x in FP64.  Restarts thus
    // happen in FP64 and the FP32 rounding floor of the inner residual never
    // limits the outer accuracy.
    VIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * n3, st));
    VIE_CUDA(cudaMemcpyAsync(r, b, sizeof(double2) * n3, cudaMemcpyDeviceToDevice, st));
    double rn = bnorm;
    VIE_TRY(norm128(P, r, 3, &rn));   // scal[3] = ||r||, read by the narrowing and the update
    double rn_prev = 2.0 * bnorm;
    int stalls = 0;
    while (outer < P->opts.max_refine && inner < P->opts.max_iter) {
      if (rn <= tol * bnorm) break;
      const double eta = std::max(P->opts.inner_tol, 0.5 * tol * bnorm / rn);
      k_narrow_scaled<<<grid_for(n3), 256, 0, st>>>(r, K.rhs64.as<float2>(), n3, K.scal.as<double>(), 3);
      count_launch();
      int it = 0;
      double rr = 0;
      VIE_TRY(gmres<float2>(P, K.rhs64.as<float2>(), K.d64.as<float2>(), K.r64.as<float2>(), eta,
                            std::min(P->opts.restart, P->opts.max_iter - inner), 1, &it, &rr));
      inner += it;
      k_axpy_to64<float2><<<grid_for(n3), 256, 0, st>>>(x, K.d64.as<float2>(), n3, K.scal.as<double>(), 3);
      count_launch();
      VIE_TRY(op_A<double2>(P, x, t));
      k_sub<<<grid_for(n3), 256, 0, st>>>(b, t, r, n3);
      count_launch();
      VIE_CHECK_LAUNCH();
      ++outer;
      VIE_TRY(norm128(P, r, 3, &rn));
      if (!std::isfinite(rn)) {
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
      if (it == 0) break;
      // a step that does not reduce the FP64 residual by 10% (twice in a row)
      // means the inner solve has nothing left to give
      if (rn > 0.9 * rn_prev) { if (++stalls >= 2) break; } else stalls = 0;
      rn_prev = rn;
    }
  }
  // final FP64 residual
  VIE_TRY(op_A<double2>(P, x, t));
  k_sub<<<grid_for(n3), 256, 0, st>>>(b, t, r, n3);
  count_launch();
  VIE_CHECK_LAUNCH();
  double rn = 0;
  VIE_TRY(norm128(P, r, 4, &rn));
  relres = bnorm > 0 ? rn / bnorm : 0.0;
  VIE_CUDA(cudaMemcpyAsync(w_out, x, sizeof(double2) * n3, cudaMemcpyDeviceToDevice, st));
  int herr = 0, hreorth = 0;
  VIE_CUDA(cudaMemcpyAsync(&herr, P->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  VIE_CUDA(cudaMemcpyAsync(&hreorth, &sdev->reorths, sizeof(int), cudaMemcpyDeviceToHost, st));
  VIE_CUDA(cudaStreamSynchronize(st));
  if (herr) {
    cudaMemsetAsync(P->dev_err.p, 0, sizeof(int), st);
    set_error("vie_solve: a bounded wait in a kernel ran out (code %d); results invalid", herr);
    return VIE_ETIMEOUT;
  }
  const float ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) {
    info->iters_inner = inner;
    info->iters_outer = outer;
    info->relres = relres;
    info->precond_bytes = P->precond_bytes;
    info->kept_fraction = P->kept_fraction;
    info->t_setup_ms = P->t_setup_ms;
    info->t_solve_ms = ms;
    info->precond_blocks = P->precond_blocks;
    info->precond_discarded = P->precond_discarded;
    info->reorth_passes = hreorth;
  }
  return relres <= tol ? VIE_OK : VIE_ENOCONV;
}

}  // namespace vie
