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

struct GmresDev {
  double2 H[(RMAX + 1) * RMAX];   // column j at H[j*(RMAX+1) + i], after rotations
  double cs[RMAX];
  double2 sn[RMAX];
  double2 g[RMAX + 1];
  double2 y[RMAX];
  double2 hc[RMAX + 1];           // coefficients of the current projection step
  double2 hsum[RMAX + 1];         // accumulated column (both CGS passes)
  double beta;                    // norm of the cycle's starting residual
  double tol_abs;                 // stop when |g_{j+1}| <= tol_abs
  double hnext;                   // h_{j+1,j}
  double resest;                  // |g_{j+1}|
  int j;                          // current column
  int k;                          // columns in the finished cycle
  int done;                       // 1: cycle finished (converged, full, or breakdown)
  int restart;
  int iters;                      // total Arnoldi steps of this state
  int reorth;                     // 1: second Gram-Schmidt pass needed (DGKS test)
  int reorths;                    // second passes taken
  int arrive_dot;                 // arrival counters of the fused grid reductions
  int arrive_upd;
  int pad[3];
  double wnorm0;                  // ||A z|| before orthogonalisation
};

struct Krylov {
  int restart = 0;
  long long n3 = 0;
  DevBuf V64, V128;               // (restart + 1) * n3 basis
  DevBuf u64, u128, z64, z128, w64, w128;
  DevBuf partial;                 // double2 [NPART][RMAX + 1]
  DevBuf state;                   // GmresDev
  DevBuf x128, r128, b128, d64, rhs64, r64, t128;
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
vie_plan_s::~vie_plan_s() = default;

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
    const double2 p = __ldcg(partial + (long long)b * (RMAX + 1) + i);
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

// Hessenberg column, rotations, residual estimate, stop test.  Run by one
// whole block: the column and the previous rotations are staged in shared
// memory, then one thread applies the rotations in sequence.
__device__ void givens_step(GmresDev* __restrict__ s, double nn) {
  __shared__ double2 col[RMAX + 1];
  __shared__ double csv[RMAX];
  __shared__ double2 snv[RMAX];
  const int j = s->j;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = s->hsum[i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) { csv[i] = s->cs[i]; snv[i] = s->sn[i]; }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double hn = sqrt(nn);
    col[j + 1] = make_double2(hn, 0);
    for (int i = 0; i < j; ++i) {
      const double2 a = col[i], b = col[i + 1];
      const double c = csv[i];
      const double2 sn = snv[i];
      // [c s; -conj(s) c] [a; b]
      col[i] = make_double2(c * a.x + (sn.x * b.x - sn.y * b.y), c * a.y + (sn.x * b.y + sn.y * b.x));
      col[i + 1] = make_double2(-(sn.x * a.x + sn.y * a.y) + c * b.x, -(sn.x * a.y - sn.y * a.x) + c * b.y);
    }
    const double2 a = col[j];
    const double b = hn;   // real, >= 0
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
    s->cs[j] = c;
    s->sn[j] = sn;
    col[j] = make_double2(c * a.x + sn.x * b, c * a.y + sn.y * b);
    col[j + 1] = make_double2(0, 0);
    const double2 gj = s->g[j];
    // g_{j+1} = -conj(s) g_j ; g_j = c g_j
    const double2 g1 = make_double2(-(sn.x * gj.x + sn.y * gj.y), -(sn.x * gj.y - sn.y * gj.x));
    s->g[j + 1] = g1;
    s->g[j] = make_double2(c * gj.x, c * gj.y);
    const double res = sqrt(g1.x * g1.x + g1.y * g1.y);
    s->resest = res;
    s->hnext = hn;
    s->iters += 1;
    s->k = j + 1;
    if (res <= s->tol_abs || j + 1 >= s->restart || hn == 0.0) s->done = 1;
    else s->j = j + 1;
  }
  __syncthreads();
  double2* H = s->H + (long long)j * (RMAX + 1);
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) H[i] = col[i];
}

// Sum of 16 values over a warp as a reduce-scatter butterfly (16 shuffles
// instead of 5 per value): returns, in every lane, the warp sum of value
// (lane >> 1) & 15.
template <class T>
__device__ __forceinline__ T warp_reduce16(const T (&v)[16], int lane) {
  T a8[8], a4[4], a2[2];
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
#pragma unroll
  for (int k = 0; k < 8; ++k) a8[k] = (b4 ? v[8 + k] : v[k]) + __shfl_xor_sync(0xffffffffu, b4 ? v[k] : v[8 + k], 16);
#pragma unroll
  for (int k = 0; k < 4; ++k) a4[k] = (b3 ? a8[4 + k] : a8[k]) + __shfl_xor_sync(0xffffffffu, b3 ? a8[k] : a8[4 + k], 8);
#pragma unroll
  for (int k = 0; k < 2; ++k) a2[k] = (b2 ? a4[2 + k] : a4[k]) + __shfl_xor_sync(0xffffffffu, b2 ? a4[k] : a4[2 + k], 4);
  T a1 = (b1 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, b1 ? a2[0] : a2[1], 2);
  a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
  return a1;
}

// partial[b][i] = sum over this block's chunk of conj(V_i) w, i = 0..j.
// Each thread accumulates DOT_T = 8 columns at once, so one pass over its
// elements serves 8 dot products; the 16 real sums are reduced over the warp
// by a butterfly and over the block by 16 warps at once (one barrier per
// group: the warp sums alternate between two shared buffers).
constexpr int DOT_T = 8;
template <class C>
__global__ void __launch_bounds__(RED_THREADS) k_dot_partial(const C* __restrict__ V, const C* __restrict__ w,
                                                             long long n3, GmresDev* __restrict__ s,
                                                             double2* __restrict__ partial, int pass) {
  // intra-block sums stay in the accumulator precision: FP64 issues at a small
  // fraction of the FP32 rate on this part, so only the per-block partial is
  // widened (once per coefficient)
  using T = typename Acc<C>::T;
  __shared__ T ws[2][RED_THREADS / 32][2 * DOT_T];
  __shared__ T wn[RED_THREADS / 32];
  if (s->done || (pass == 1 && !s->reorth)) return;
  const int j = s->j;
  const long long chunk = (n3 + gridDim.x - 1) / gridDim.x;
  const long long c0 = blockIdx.x * chunk, c1 = min(n3, c0 + chunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* pb = reinterpret_cast<double*>(partial + (long long)blockIdx.x * (RMAX + 1));
  T nn = 0;   // ||w||^2 over the chunk (pass 0), gathered with the first group
  int buf = 0;
  for (int i0 = 0; i0 <= j; i0 += DOT_T, buf ^= 1) {
    T a[2 * DOT_T];
#pragma unroll
    for (int t = 0; t < 2 * DOT_T; ++t) a[t] = 0;
    const int nt = min(DOT_T, j + 1 - i0);
    const bool with_norm = pass == 0 && i0 == 0;
    for (long long e = c0 + threadIdx.x; e < c1; e += blockDim.x) {
      const C x = w[e];
      if (with_norm) nn += x.x * x.x + x.y * x.y;
#pragma unroll
      for (int t = 0; t < DOT_T; ++t) {
        if (t < nt) {
          const C v = V[(long long)(i0 + t) * n3 + e];
          a[2 * t] += v.x * x.x + v.y * x.y;
          a[2 * t + 1] += v.x * x.y - v.y * x.x;
        }
      }
    }
    const T r = warp_reduce16<T>(a, lane);
    if ((lane & 1) == 0) ws[buf][warp][lane >> 1] = r;
    __syncthreads();
    if (warp < 2 * DOT_T) {   // warp q sums value q over the block's warps
      T x = ws[buf][lane][warp];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0 && (warp >> 1) < nt) pb[2 * (i0 + (warp >> 1)) + (warp & 1)] = (double)x;
    }
  }
  if (pass == 0) {   // ||w||^2 before orthogonalisation, slot RMAX
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    if (lane == 0) wn[warp] = nn;
    __syncthreads();
    if (warp == 0) {
      T x = wn[lane];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) partial[(long long)blockIdx.x * (RMAX + 1) + RMAX] = make_double2((double)x, 0.0);
    }
  }
  // the last block to finish reduces the partials: h (pass 0 sets, pass 1
  // adds) and, in pass 0, ||w|| before orthogonalisation
  GmresDev* sm = const_cast<GmresDev*>(s);
  if (!last_block(&sm->arrive_dot)) return;
  const int nw = blockDim.x >> 5;
  for (int i = warp; i <= j; i += nw) {
    const double2 t = warp_sum_partials_cg(partial, gridDim.x, i);
    if (lane == 0) {
      sm->hc[i] = t;
      if (pass == 0) sm->hsum[i] = t;
      else { sm->hsum[i].x += t.x; sm->hsum[i].y += t.y; }
    }
  }
  if (pass == 0 && warp == nw - 1) {
    const double t = warp_sum_partials_cg(partial, gridDim.x, RMAX).x;
    if (lane == 0) sm->wnorm0 = sqrt(t);
  }
}

// sum of partial[b][i] over b by one warp (fixed order: lane-strided sums,
// then a butterfly)
__device__ __forceinline__ double2 warp_sum_partials(const double2* __restrict__ partial, int nparts, int i) {
  const int lane = threadIdx.x & 31;
  double2 t = make_double2(0, 0);
  for (int b = lane; b < nparts; b += 32) {
    const double2 p = partial[(long long)b * (RMAX + 1) + i];
    t.x += p.x;
    t.y += p.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
    t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
  }
  return t;
}

// w -= sum_i hc[i] V_i ; optionally partial[b][0] = ||w||^2 over the chunk
template <class C>
__global__ void __launch_bounds__(RED_THREADS) k_update(const C* __restrict__ V, C* __restrict__ w, long long n3,
                                                        GmresDev* __restrict__ s, double2* __restrict__ partial,
                                                        int pass) {
  __shared__ double2 sh[32];
  __shared__ C hcs[RMAX + 1];
  if (s->done || (pass == 1 && !s->reorth)) return;
  const int want_norm = 1;
  const int j = s->j;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) hcs[i] = cconv<C>(s->hc[i]);
  __syncthreads();
  const long long chunk = (n3 + gridDim.x - 1) / gridDim.x;
  const long long c0 = blockIdx.x * chunk, c1 = min(n3, c0 + chunk);
  using T = typename Acc<C>::T;
  T nrm = 0;
  for (long long e = c0 + threadIdx.x; e < c1; e += blockDim.x) {
    C x = w[e];
    int i = 0;
    for (; i + 7 <= j; i += 8) {
      C v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) v[t] = V[(long long)(i + t) * n3 + e];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const C h = hcs[i + t];
        x.x -= h.x * v[t].x - h.y * v[t].y;
        x.y -= h.x * v[t].y + h.y * v[t].x;
      }
    }
    for (; i <= j; ++i) {
      const C v = V[(long long)i * n3 + e];
      const C h = hcs[i];
      x.x -= h.x * v.x - h.y * v.y;
      x.y -= h.x * v.y + h.y * v.x;
    }
    w[e] = x;
    nrm += x.x * x.x + x.y * x.y;
  }
  if (want_norm) {
    __shared__ T shn[32];
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) shn[warp] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
      T t = 0;
      for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += shn[w2];
      partial[(long long)blockIdx.x * (RMAX + 1)] = make_double2((double)t, 0.0);
    }
  }
  // the last block: ||w|| over the grid, then (pass 0) the DGKS test, and the
  // Givens step once no second Gram-Schmidt pass follows
  GmresDev* sm = const_cast<GmresDev*>(s);
  if (!last_block(&sm->arrive_upd)) return;
  __shared__ double nn_s;
  if ((threadIdx.x >> 5) == 0) {
    const double nn = warp_sum_partials_cg(partial, gridDim.x, 0).x;
    if (threadIdx.x == 0) nn_s = nn;
  }
  __syncthreads();
  const double nn = nn_s;
  bool final_pass = true;
  if (pass == 0) {
    // re-orthogonalise only if the projection removed more than 1 - 1/sqrt(2) of ||w||
    const int r = sqrt(nn) < 0.70710678118654752 * sm->wnorm0 ? 1 : 0;
    __syncthreads();
    if (threadIdx.x == 0) { sm->reorth = r; sm->reorths += r; }
    final_pass = (r == 0);
  }
  if (final_pass) givens_step(sm, nn);
}

// V_{j} = w / h (j already advanced) and u = V_j
template <class C>
__global__ void k_scale_next(C* __restrict__ V, const C* __restrict__ w, C* __restrict__ u, long long n3,
                             const GmresDev* __restrict__ s) {
  if (s->done) return;
  const int j = s->j;
  using T = typename real_of<C>::type;
  const T inv = (T)1 / (T)s->hnext;   // reciprocal in the vector precision
  C* Vj = V + (long long)j * n3;
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
  const long long chunk = (n3 + gridDim.x - 1) / gridDim.x;
  const long long c0 = blockIdx.x * chunk, c1 = min(n3, c0 + chunk);
  double nrm = 0;   // FP64 per thread: called once per cycle
  for (long long e = c0 + threadIdx.x; e < c1; e += blockDim.x) nrm += (double)r[e].x * r[e].x + (double)r[e].y * r[e].y;
  const double2 t = block_sum2(make_double2(nrm, 0), sh);
  if (threadIdx.x == 0) partial[(long long)blockIdx.x * (RMAX + 1)] = t;
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
__global__ void k_solve_y(GmresDev* __restrict__ s) {
  if (threadIdx.x != 0) return;
  const int k = s->k;
  for (int i = k - 1; i >= 0; --i) {
    double2 t = s->g[i];
    for (int l = i + 1; l < k; ++l) {
      const double2 h = s->H[(long long)l * (RMAX + 1) + i];
      const double2 y = s->y[l];
      t.x -= h.x * y.x - h.y * y.y;
      t.y -= h.x * y.y + h.y * y.x;
    }
    const double2 d = s->H[(long long)i * (RMAX + 1) + i];
    const double2 id = cinv(d);
    s->y[i] = cmul(t, id);
  }
}

// u = sum_{i<k} y_i V_i
template <class C>
__global__ void k_combine(const C* __restrict__ V, C* __restrict__ u, long long n3, const GmresDev* __restrict__ s) {
  __shared__ C ys[RMAX];
  const int k = s->k;
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = cconv<C>(s->y[i]);
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x) {
    C acc = czero<C>();
    for (int i = 0; i < k; ++i) cfma(acc, ys[i], V[(long long)i * n3 + e]);
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
  if (!K.state.p) {
    VIE_TRY(K.state.alloc(sizeof(GmresDev)));
    VIE_CUDA(cudaMemset(K.state.p, 0, sizeof(GmresDev)));
    VIE_TRY(K.partial.alloc(sizeof(double2) * NPART * (RMAX + 1)));
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
    VIE_TRY(K.V64.alloc(sizeof(float2) * n3 * (R + 1)));
    VIE_TRY(K.u64.alloc(sizeof(float2) * n3));
    VIE_TRY(K.z64.alloc(sizeof(float2) * n3));
    VIE_TRY(K.w64.alloc(sizeof(float2) * n3));
    VIE_TRY(K.d64.alloc(sizeof(float2) * n3));
    VIE_TRY(K.rhs64.alloc(sizeof(float2) * n3));
    VIE_TRY(K.r64.alloc(sizeof(float2) * n3));
  }
  if (need128 && !K.V128.p) {
    VIE_TRY(K.V128.alloc(sizeof(double2) * n3 * (R + 1)));
    VIE_TRY(K.u128.alloc(sizeof(double2) * n3));
    VIE_TRY(K.z128.alloc(sizeof(double2) * n3));
    VIE_TRY(K.w128.alloc(sizeof(double2) * n3));
  }
  return VIE_OK;
}

// kernels in one captured Arnoldi step (for launch accounting)
static int step_kernels(vie_plan_s* P) {
  Krylov& K = *P->kry;
  return K.step_launches;
}

// enqueue one Arnoldi step (u holds v_j on entry and v_{j+1} on exit)
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
  VIE_TRY(op_Pinv<C>(P, u, z));
  VIE_TRY(op_A<C>(P, z, w));
  // CGS2 with the DGKS test: dot (+ grid reduction of h in its last block),
  // update (+ ||w||, DGKS test and, on the final pass, the Givens step in its
  // last block); the second pass exits at once when not needed
  for (int pass = 0; pass < 2; ++pass) {
    { Prof pf_(sizeof(C) == 8 ? "arnoldi_dot_c64" : "arnoldi_dot_c128", st); k_dot_partial<C><<<NPART, RED_THREADS, 0, st>>>(V, w, n3, s, part, pass); }
    { Prof pf_(sizeof(C) == 8 ? "arnoldi_update_c64" : "arnoldi_update_c128", st); k_update<C><<<NPART, RED_THREADS, 0, st>>>(V, w, n3, s, part, pass); }
    count_launch(2);
  }
  { Prof pf_("arnoldi_scale", st); k_scale_next<C><<<grid_for(n3), 256, 0, st>>>(V, w, u, n3, s); }
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
  double rr = 1.0, rr_prev = 2.0;
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
    const int cyc = std::min(K.restart, max_iter - total);
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
    k_solve_y<<<1, 32, 0, st>>>(s);
    k_combine<C><<<grid_for(n3), 256, 0, st>>>(V, u, n3, s);
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
    // restarted cycles that no longer halve the true residual have hit the
    // rounding floor of this precision
    if (rr > 0.5 * rr_prev) break;
    rr_prev = rr;
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
      if (!std::isfinite(rn)) { set_error("vie_solve: refinement diverged (non-finite residual)"); return VIE_ECUDA; }
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
    set_error("vie_solve: a tensor-core wait ran out (results invalid)");
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
