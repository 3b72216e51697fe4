// Block-diagonal 1-level circulant preconditioner (Sec. 4, Sec. 5.1.1,
// Sec. 5.2, Sec. 5.3).
//
// Per box (nx_b x ny_b x nz_b voxels, m = 3 ny_b nz_b unknowns per x-slab,
// rows ordered [alpha][z][y]):
//  1. homogenise M over the box (Sec. 5.2: mode, x-mean, or real x-mean);
//  2. for each generator pair and transverse offset, the Chan vector of the
//     x-Toeplitz line (Eq. Chan) and its DFT lambda_f (C = F^-1 Lambda F);
//  3. proxy v_f (Eqs. proxy1-proxy2) and the kept set K = {f : v^_f > tau};
//  4. D_f = I - M~ (I + Lambda_f) (Eq. Di) for the stored frequencies;
//  5. FP64 LU with partial pivoting of every stored block, then the explicit
//     inverse (complex FP32 for the mixed path, FP64 for the FP64 path);
//  6. apply: z = F^-1 P^T diag(D_f^-1) P F r (the C_B^-1 display of Sec. 4).
// Only f <= n/2 carry blocks: the x-parity of the generators gives
// D_{n-f} = S D_f S, S = diag(-1 on x-component rows, +1 otherwise), so f and
// n - f share one block read.  Frequencies outside K use the central block
// D_{ceil(n/2)} (1-based) through one multi-right-hand-side product.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <chrono>

#include "greens.cuh"
#include "internal.h"
#include "umma.cuh"
#include "prof.h"

namespace vie {


__device__ __forceinline__ int pair_code(int a, int b) {
  if (a > b) { int t = a; a = b; b = t; }
  // xx0 xy1 xz2 yy3 yz4 zz5
  return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

struct BoxDims {
  int x0, y0, z0, n, ny, nz, m;
  int gnx, gny, gnz;   // full grid
};

// ---------------------------------------------------------------------------
// 1. homogenisation
// ---------------------------------------------------------------------------
__global__ void k_hom_mean(const double2* __restrict__ M, double2* __restrict__ Mt, BoxDims b, int real_only) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b.ny * b.nz) return;
  const int yb = t % b.ny, zb = t / b.ny;
  const double2* row = M + ((long long)(b.z0 + zb) * b.gny + (b.y0 + yb)) * b.gnx + b.x0;
  double sr = 0, si = 0;
  for (int x = 0; x < b.n; ++x) { sr += row[x].x; si += row[x].y; }
  sr /= b.n;
  si /= b.n;
  Mt[t] = make_double2(sr, real_only ? 0.0 : si);
}

// Plane mean for a 2-level box (M~ invariant in x and y): one block per
// z-plane, a fixed-order tree sum; the value is replicated over y so that
// M~ keeps the [nz][ny] layout of the 1-level boxes.
__global__ void __launch_bounds__(256) k_hom_plane(const double2* __restrict__ M, double2* __restrict__ Mt, BoxDims b,
                                                   int real_only) {
  __shared__ double sr[256], si[256];
  const int zb = blockIdx.x;
  double ar = 0, ai = 0;
  const int e_n = b.n * b.ny;
  for (int e = threadIdx.x; e < e_n; e += blockDim.x) {
    const int x = e % b.n, yb = e / b.n;
    const double2 v = M[((long long)(b.z0 + zb) * b.gny + (b.y0 + yb)) * b.gnx + b.x0 + x];
    ar += v.x;
    ai += v.y;
  }
  sr[threadIdx.x] = ar;
  si[threadIdx.x] = ai;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) { sr[threadIdx.x] += sr[threadIdx.x + s]; si[threadIdx.x] += si[threadIdx.x + s]; }
    __syncthreads();
  }
  const double2 mv = make_double2(sr[0] / e_n, real_only ? 0.0 : si[0] / e_n);
  for (int yb = threadIdx.x; yb < b.ny; yb += blockDim.x) Mt[zb * b.ny + yb] = mv;
}

// Mode of all box entries: one block keeps a table of distinct values and
// counts.  Ties go to the smallest |value|, then the smallest (re, im).
constexpr int MODE_MAXV = 512;
__global__ void __launch_bounds__(1024) k_hom_mode(const double2* __restrict__ M, double2* __restrict__ Mt, BoxDims b,
                                                   int* __restrict__ err) {
  __shared__ double2 vals[MODE_MAXV];
  __shared__ int counts[MODE_MAXV];
  __shared__ double2 chunk[1024];
  __shared__ int found[1024];
  __shared__ int nv;
  __shared__ int overflow;
  if (threadIdx.x == 0) { nv = 0; overflow = 0; }
  for (int i = threadIdx.x; i < MODE_MAXV; i += blockDim.x) counts[i] = 0;
  __syncthreads();
  const long long total = (long long)b.n * b.ny * b.nz;
  for (long long base = 0; base < total; base += blockDim.x) {
    const long long e = base + threadIdx.x;
    const int nloc = (int)min((long long)blockDim.x, total - base);
    double2 v = make_double2(0, 0);
    int idx = -1;
    if (e < total) {
      const int x = (int)(e % b.n);
      const long long r = e / b.n;
      const int yb = (int)(r % b.ny), zb = (int)(r / b.ny);
      v = M[((long long)(b.z0 + zb) * b.gny + (b.y0 + yb)) * b.gnx + b.x0 + x];
      const int cur = nv;
      for (int j = 0; j < cur; ++j)
        if (vals[j].x == v.x && vals[j].y == v.y) { idx = j; break; }
      if (idx >= 0) atomicAdd(&counts[idx], 1);
      chunk[threadIdx.x] = v;
      found[threadIdx.x] = idx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int t = 0; t < nloc; ++t) {
        if (found[t] >= 0) continue;
        const double2 w = chunk[t];
        int j = 0;
        for (; j < nv; ++j)
          if (vals[j].x == w.x && vals[j].y == w.y) break;
        if (j == nv) {
          if (nv >= MODE_MAXV) { overflow = 1; continue; }
          vals[nv] = w;
          counts[nv] = 0;
          ++nv;
        }
        counts[j] += 1;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int best = 0;
    for (int j = 1; j < nv; ++j) {
      const double aj = vals[j].x * vals[j].x + vals[j].y * vals[j].y;
      const double ab = vals[best].x * vals[best].x + vals[best].y * vals[best].y;
      bool better = counts[j] > counts[best];
      if (counts[j] == counts[best]) {
        if (aj < ab) better = true;
        else if (aj == ab && (vals[j].x < vals[best].x || (vals[j].x == vals[best].x && vals[j].y < vals[best].y)))
          better = true;
      }
      if (better) best = j;
    }
    const double2 mv = nv ? vals[best] : make_double2(0, 0);
    for (int t = 0; t < b.ny * b.nz; ++t) Mt[t] = mv;
    if (overflow) *err = 1;
  }
}

// ---------------------------------------------------------------------------
// 2. Chan coefficients of every x-Toeplitz line (Eq. Chan):
//    c_k = ((n - k) t_k + k t_{k-n}) / n,  t_i = G^c(i, dy, dz)
// lines ordered (c, dz + nz - 1, dy + ny - 1); output [line][k]
// ---------------------------------------------------------------------------
__global__ void k_chan_coeffs(double2* __restrict__ out, BoxDims b, double h, double kb, double2 self) {
  const int ndy = 2 * b.ny - 1, ndz = 2 * b.nz - 1;
  const long long nl = 6LL * ndz * ndy;
  const long long total = nl * b.n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(idx % b.n);
    const long long line = idx / b.n;
    const int dyi = (int)(line % ndy);
    const long long r = line / ndy;
    const int dzi = (int)(r % ndz);
    const int c = (int)(r / ndz);
    const int dy = dyi - (b.ny - 1), dz = dzi - (b.nz - 1);
    const double2 tk = gen_entry(c, k, dy, dz, h, kb, self);
    double2 v;
    if (k == 0) {
      v = tk;
    } else {
      const double2 tm = gen_entry(c, k - b.n, dy, dz, h, kb, self);
      const double wn = (double)(b.n - k) / b.n, wk = (double)k / b.n;
      v = make_double2(wn * tk.x + wk * tm.x, wn * tk.y + wk * tm.y);
    }
    out[idx] = v;
  }
}

// ---------------------------------------------------------------------------
// 3. proxy and selection (one block).  lam is frequency-major [f][line].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_select(const double2* __restrict__ lam, const double2* __restrict__ Mt,
                                                 BoxDims b, double tau, double* __restrict__ vhat,
                                                 int* __restrict__ fmap, int* __restrict__ fsgn,
                                                 int* __restrict__ disc, int* __restrict__ blkf,
                                                 int* __restrict__ counts) {
  const int n = b.n;
  const int ndy = 2 * b.ny - 1, ndz = 2 * b.nz - 1;
  const int nl = 6 * ndz * ndy;
  const int cstar = ((b.ny + 1) / 2) * ((b.nz + 1) / 2) - 1;
  int line;
  bool diag = false;
  if (cstar == 0) {
    line = (0 * ndz + (b.nz - 1)) * ndy + (b.ny - 1);
    diag = true;
  } else {
    const int zq = (cstar % (b.ny * b.nz)) / b.ny, yq = cstar % b.ny;
    line = (0 * ndz + (-zq + b.nz - 1)) * ndy + (-yq + b.ny - 1);
  }
  __shared__ double red[1024];
  double mx = 0.0;
  for (int f = threadIdx.x; f < n; f += blockDim.x) {
    double2 v = lam[(long long)f * nl + line];
    if (diag) {
      const double2 m0 = Mt[0];
      // 1 - M0 (1 + lambda)
      const double ar = 1.0 + v.x, ai = v.y;
      v = make_double2(1.0 - (m0.x * ar - m0.y * ai), -(m0.x * ai + m0.y * ar));
    }
    const double a = sqrt(v.x * v.x + v.y * v.y);
    vhat[f] = a;
    mx = fmax(mx, a);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  const double vmax = red[0];
  __syncthreads();
  for (int f = threadIdx.x; f < n; f += blockDim.x) vhat[f] = vmax > 0 ? vhat[f] / vmax : 1.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int half = n / 2;
    const int rep = (n + 1) / 2 - 1;
    int nb = 0;
    // slots for kept f <= n/2 (kept decided at the folded frequency)
    for (int f = 0; f <= half; ++f) {
      const bool keep = tau <= 0.0 || vhat[f] > tau;
      if (keep) { blkf[nb] = f; fmap[f] = nb; ++nb; } else fmap[f] = -1;
    }
    const int nks = nb;
    int rep_slot = fmap[rep];
    if (rep_slot < 0) { blkf[nb] = rep; rep_slot = nb; ++nb; }
    int nd = 0, nk = 0;
    for (int f = 0; f < n; ++f) {
      const int fo = f <= half ? f : n - f;
      const int s = fmap[fo];
      if (f > half) fmap[f] = s;
      fsgn[f] = (f > half) ? 1 : 0;
      if (s < 0) disc[nd++] = f; else ++nk;
    }
    counts[0] = nb;
    counts[1] = nk;
    counts[2] = nd;
    counts[3] = rep_slot;
    counts[4] = nks;
  }
}

// ---------------------------------------------------------------------------
// 4. block assembly D_f[p][q] = delta - M~_p (delta + lambda_f^{pq}), column-major
// ---------------------------------------------------------------------------
__global__ void k_block_assemble(double2* __restrict__ D, const double2* __restrict__ lam,
                                 const double2* __restrict__ Mt, const int* __restrict__ blkf, BoxDims b, int nblk) {
  const int m = b.m;
  const int ndy = 2 * b.ny - 1, ndz = 2 * b.nz - 1;
  const int nl = 6 * ndz * ndy;
  const int yz = b.ny * b.nz;
  const long long total = (long long)nblk * m * m;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(idx % m);
    const long long r = idx / m;
    const int q = (int)(r % m);
    const int s = (int)(r / m);
    const int f = blkf[s];
    const int ap = p / yz, zp = (p % yz) / b.ny, yp = p % b.ny;
    const int aq = q / yz, zq = (q % yz) / b.ny, yq = q % b.ny;
    const int c = pair_code(ap, aq);
    const int line = (c * ndz + (zp - zq + b.nz - 1)) * ndy + (yp - yq + b.ny - 1);
    const double2 l = lam[(long long)f * nl + line];
    const double2 mp = Mt[zp * b.ny + yp];
    const double dl = (p == q) ? 1.0 : 0.0;
    const double ar = dl + l.x, ai = l.y;
    D[idx] = make_double2(dl - (mp.x * ar - mp.y * ai), -(mp.x * ai + mp.y * ar));
  }
}

// ---------------------------------------------------------------------------
// 5a. batched LU with partial pivoting (column-major, right-looking with
//     panels of NB columns), in complex FP64 for the FP64 preconditioner and
//     in complex FP32 for the complex-FP32 one.  Each panel step is two
//     launches over all matrices: the panel (pivoting, row swaps,
//     U12 = L11^-1 A12; one block per matrix), then the trailing update
//     A22 -= L21 U12 as 32x32 tiles of every matrix, so that the work fills
//     every SM whatever the batch size.
// ---------------------------------------------------------------------------
constexpr int LU_NB = 16;
constexpr int LU_TILE = 32;

template <class C>
__device__ __forceinline__ typename real_of<C>::type cabs1(C a) { return fabs(a.x) + fabs(a.y); }

template <class C>
__global__ void __launch_bounds__(512) k_lu_panel(C* __restrict__ Aall, int* __restrict__ pivall, int m, int k0,
                                                  int* __restrict__ info) {
  using R = typename real_of<C>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* P = reinterpret_cast<C*>(smem_raw);     // panel: NB columns x (m - k0) rows
  __shared__ R rv[32];
  __shared__ int ri[32];
  __shared__ int piv_s;
  C* A = Aall + (long long)blockIdx.x * m * m;
  int* piv = pivall + (long long)blockIdx.x * m;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int nb = min(LU_NB, m - k0);
  const int rows = m - k0;
  for (int e = tid; e < nb * rows; e += nt) {
    const int j = e / rows, i = e - j * rows;
    P[j * rows + i] = A[(long long)(k0 + j) * m + k0 + i];
  }
  __syncthreads();
  for (int kk = 0; kk < nb; ++kk) {
    const int k = k0 + kk;
    C* col = P + kk * rows;
    // pivot search over rows k..m-1 (first maximum of |re| + |im|); the
    // candidate starts at the diagonal row so that the index stays valid
    // even if every entry compares false (NaN)
    R best = -1;
    int bi = kk;
    for (int i = kk + tid; i < rows; i += nt) {
      const R v = cabs1(col[i]);
      if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const R ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      R b0 = rv[0];
      int i0 = ri[0];
      for (int w = 1; w < nw; ++w)
        if (rv[w] > b0 || (rv[w] == b0 && ri[w] < i0)) { b0 = rv[w]; i0 = ri[w]; }
      if (i0 < kk || i0 >= rows) i0 = kk;
      piv_s = i0;
      piv[k] = k0 + i0;
      if (!(b0 > 0)) atomicExch(info, 1);   // zero or non-finite pivot
    }
    __syncthreads();
    const int pi = piv_s;
    if (pi != kk) {   // swap rows kk and pi inside the panel
      for (int j = tid; j < nb; j += nt) {
        const C t = P[j * rows + kk];
        P[j * rows + kk] = P[j * rows + pi];
        P[j * rows + pi] = t;
      }
    }
    __syncthreads();
    const C pv = col[kk];
    C ipv = czero<C>();
    if (pv.x != 0 || pv.y != 0) {
      const R d = R(1) / (pv.x * pv.x + pv.y * pv.y);
      ipv = cmake<C>(pv.x * d, -pv.y * d);
    }
    for (int i = kk + 1 + tid; i < rows; i += nt) col[i] = cmul(col[i], ipv);
    __syncthreads();
    // rank-1 update of the remaining panel columns
    const int rem = nb - kk - 1;
    for (int e = tid; e < rem * (rows - kk - 1); e += nt) {
      const int jj = kk + 1 + e / (rows - kk - 1);
      const int i = kk + 1 + e % (rows - kk - 1);
      C a = P[jj * rows + i];
      const C l = col[i], u = P[jj * rows + kk];
      a.x -= l.x * u.x - l.y * u.y;
      a.y -= l.x * u.y + l.y * u.x;
      P[jj * rows + i] = a;
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * rows; e += nt) {
    const int j = e / rows, i = e - j * rows;
    A[(long long)(k0 + j) * m + k0 + i] = P[j * rows + i];
  }
  // the panel's row swaps on every other column (left: the final L; right:
  // the columns still to be factored), then U12 = L11^{-1} A12
  for (int j = tid; j < m; j += nt) {
    if (j >= k0 && j < k0 + nb) continue;
    C* cj = A + (long long)j * m;
    for (int kk = 0; kk < nb; ++kk) {
      const int k = k0 + kk, p = piv[k];
      if (p != k) { const C t = cj[k]; cj[k] = cj[p]; cj[p] = t; }
    }
    if (j >= k0 + nb) {
      C u[LU_NB];
#pragma unroll
      for (int t = 0; t < LU_NB; ++t) u[t] = t < nb ? cj[k0 + t] : czero<C>();
#pragma unroll
      for (int t = 0; t < LU_NB; ++t) {
        if (t >= nb) break;
#pragma unroll
        for (int i = t + 1; i < LU_NB; ++i) {
          if (i >= nb) break;
          const C l = P[t * rows + i];
          u[i].x -= l.x * u[t].x - l.y * u[t].y;
          u[i].y -= l.x * u[t].y + l.y * u[t].x;
        }
      }
#pragma unroll
      for (int t = 0; t < LU_NB; ++t) if (t < nb) cj[k0 + t] = u[t];
    }
  }
}

// A22 -= L21 U12 on one 32x32 tile of one matrix.  Thread (tx, ty) owns
// rows tx, tx + 16 and columns ty, ty + 16 of the tile.  Complex FP64 takes
// three real products per complex product (T1 = Lr Ur, T2 = Li Ui,
// T3 = (Lr + Li)(Ur + Ui); re -= T1 - T2, im -= T3 - T1 - T2): FP64 issues
// slowly on this part, and this saves a quarter of the multiply-adds.
// Complex FP32 keeps the four products (no cancellation in T3 - T1 - T2).
template <class C>
__global__ void __launch_bounds__(256) k_lu_update(C* __restrict__ Aall, int m, int k0, int nb) {
  using R = typename real_of<C>::type;
  constexpr bool k3m = sizeof(R) == 8;
  __shared__ R Lr[LU_NB][LU_TILE], Li[LU_NB][LU_TILE], Ls[k3m ? LU_NB : 1][LU_TILE];
  __shared__ R Ur[LU_NB][LU_TILE], Ui[LU_NB][LU_TILE], Us[k3m ? LU_NB : 1][LU_TILE];
  const int r0 = k0 + nb;                    // first row / column of A22
  const int r22 = m - r0;
  const int nti = (r22 + LU_TILE - 1) / LU_TILE;
  const int i0 = r0 + (blockIdx.x % nti) * LU_TILE, j0 = r0 + (blockIdx.x / nti) * LU_TILE;
  C* A = Aall + (long long)blockIdx.y * m * m;
  const int tid = threadIdx.x;
  for (int e = tid; e < LU_NB * LU_TILE; e += blockDim.x) {
    const int t = e / LU_TILE, q = e % LU_TILE;
    C l = czero<C>(), u = czero<C>();
    if (t < nb && i0 + q < m) l = A[(long long)(k0 + t) * m + i0 + q];   // L21[i][t], column k0 + t
    if (t < nb && j0 + q < m) u = A[(long long)(j0 + q) * m + k0 + t];   // U12[t][j], row k0 + t
    Lr[t][q] = l.x; Li[t][q] = l.y;
    Ur[t][q] = u.x; Ui[t][q] = u.y;
    if constexpr (k3m) { Ls[t][q] = l.x + l.y; Us[t][q] = u.x + u.y; }
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  R t1[2][2] = {}, t2[2][2] = {}, t3[2][2] = {};
  for (int t = 0; t < nb; ++t) {
    R lr[2], li[2], ur[2], ui[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      lr[a] = Lr[t][tx + 16 * a]; li[a] = Li[t][tx + 16 * a];
      ur[a] = Ur[t][ty + 16 * a]; ui[a] = Ui[t][ty + 16 * a];
    }
    if constexpr (k3m) {
      R ls[2], us[2];
#pragma unroll
      for (int a = 0; a < 2; ++a) { ls[a] = Ls[t][tx + 16 * a]; us[a] = Us[t][ty + 16 * a]; }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          t1[a][b] = fma(lr[a], ur[b], t1[a][b]);
          t2[a][b] = fma(li[a], ui[b], t2[a][b]);
          t3[a][b] = fma(ls[a], us[b], t3[a][b]);
        }
    } else {
      // t1 = re(L U), t3 = im(L U)
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          t1[a][b] = fma(lr[a], ur[b], t1[a][b]);
          t1[a][b] = fma(-li[a], ui[b], t1[a][b]);
          t3[a][b] = fma(lr[a], ui[b], t3[a][b]);
          t3[a][b] = fma(li[a], ur[b], t3[a][b]);
        }
    }
  }
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const int j = j0 + ty + 16 * b;
    if (j >= m) continue;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int i = i0 + tx + 16 * a;
      if (i >= m) continue;
      C v = A[(long long)j * m + i];
      if constexpr (k3m) {
        v.x -= t1[a][b] - t2[a][b];
        v.y -= t3[a][b] - t1[a][b] - t2[a][b];
      } else {
        v.x -= t1[a][b];
        v.y -= t3[a][b];
      }
      A[(long long)j * m + i] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// 5b. explicit inverse from the LU factors: solve L U X = P I for a chunk of
//     CB columns; X written row-major in precision C.
// ---------------------------------------------------------------------------
// blocks (or their FP64 LU factors) rounded to complex FP32
__global__ void k_lu_narrow(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

// Columns j0..j0+cb-1 of D^{-1} = U^{-1} L^{-1} P: the pivoted identity
// columns in shared memory, forward substitution with the unit lower L, back
// substitution with U.  Column k of the factor is staged in shared memory one
// step ahead (the load of step k+1 overlaps the update of step k), the
// inverted diagonal is formed once up front, and the back substitution's
// scaling is folded into each thread's update, so every step has one barrier.
template <class C>
__global__ void __launch_bounds__(256) k_block_inv(const C* __restrict__ LUall, const int* __restrict__ pivall,
                                                   C* __restrict__ invall, int m, int CB) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Y = reinterpret_cast<C*>(smem_raw);   // [m][CB]
  C* col0 = Y + (size_t)m * CB;            // two staged columns
  C* col1 = col0 + m;
  C* dinv = col1 + m;                      // [m] 1 / U[k][k]
  using T = typename real_of<C>::type;
  const C* LU = LUall + (long long)blockIdx.x * m * m;
  const int* piv = pivall + (long long)blockIdx.x * m;
  C* inv = invall + (long long)blockIdx.x * m * m;
  const int j0 = blockIdx.y * CB;
  const int cb = min(CB, m - j0);
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < m * CB; e += nt) {
    const int i = e / CB, c = e - i * CB;
    Y[e] = (c < cb && i == j0 + c) ? cmake<C>(1, 0) : czero<C>();
  }
  for (int k = tid; k < m; k += nt) {
    const C u = LU[(long long)k * m + k];
    const T q = (T)1 / (u.x * u.x + u.y * u.y);
    dinv[k] = cmake<C>(u.x * q, -u.y * q);
  }
  if (m > 1)
    for (int i = 1 + tid; i < m; i += nt) col0[i] = LU[i];   // column 0 of L
  __syncthreads();
  // P applied to the identity columns: the row swaps in order
  if (tid < cb) {
    for (int k = 0; k < m; ++k) {
      const int p = piv[k];
      if (p != k) { const C t = Y[k * CB + tid]; Y[k * CB + tid] = Y[p * CB + tid]; Y[p * CB + tid] = t; }
    }
  }
  __syncthreads();
  // forward substitution with unit lower L
  for (int k = 0; k < m - 1; ++k) {
    C* cur = (k & 1) ? col1 : col0;
    C* nxt = (k & 1) ? col0 : col1;
    if (k + 1 < m - 1)
      for (int i = k + 2 + tid; i < m; i += nt) nxt[i] = LU[(long long)(k + 1) * m + i];
    const int cnt = (m - k - 1) * cb;
    for (int e = tid; e < cnt; e += nt) {
      const int i = k + 1 + e / cb, c = e % cb;
      const C lc = cur[i];
      C y = Y[i * CB + c];
      const C yk = Y[k * CB + c];
      y.x -= lc.x * yk.x - lc.y * yk.y;
      y.y -= lc.x * yk.y + lc.y * yk.x;
      Y[i * CB + c] = y;
    }
    __syncthreads();
  }
  // back substitution with U: row k of the result is Y[k] / U[k][k], written
  // out directly; the rows above subtract U[i][k] times it
  {
    C* cur = col0;
    for (int i = tid; i < m - 1; i += nt) cur[i] = LU[(long long)(m - 1) * m + i];
  }
  __syncthreads();
  for (int k = m - 1; k >= 0; --k) {
    const int par = (m - 1 - k) & 1;
    C* cur = par ? col1 : col0;
    C* nxt = par ? col0 : col1;
    if (k > 0)
      for (int i = tid; i < k - 1; i += nt) nxt[i] = LU[(long long)(k - 1) * m + i];
    const C dk = dinv[k];
    if (tid < cb) inv[(long long)k * m + j0 + tid] = cmul(Y[k * CB + tid], dk);
    const int cnt = k * cb;
    for (int e = tid; e < cnt; e += nt) {
      const int i = e / cb, c = e % cb;
      const C uc = cur[i];
      const C yk = cmul(Y[k * CB + c], dk);
      C y = Y[i * CB + c];
      y.x -= uc.x * yk.x - uc.y * yk.y;
      y.y -= uc.x * yk.y + uc.y * yk.x;
      Y[i * CB + c] = y;
    }
    __syncthreads();
  }
}

// 8-byte global -> shared copy that does not hold the issuing thread
// (cp.async; completion by commit groups)
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// all but the most recent group of this thread complete
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Register-blocked variant for m <= 8 RPG (complex FP32): 256 threads = 8
// row groups (one per warp) x 32 right-hand-side columns; thread (g, c) keeps
// rows [g RPG, (g + 1) RPG) of column c in registers.  Per step the owner of
// row k publishes it through shared memory (one barrier), and every thread
// updates its own rows with the staged factor column, so the update touches
// shared memory once per multiply-add (the factor) instead of four times.
// The factor columns stream through three shared buffers, copied two steps
// ahead with cp.async, so no step waits on a global load.
template <int RPG>
__global__ void __launch_bounds__(256) k_block_inv_rb(const float2* __restrict__ LUall, const int* __restrict__ pivall,
                                                      float2* __restrict__ invall, int m) {
  __shared__ __align__(16) float2 col[3][8 * RPG];
  __shared__ float2 rowk[2][32];
  __shared__ float2 dinv[8 * RPG];
  __shared__ int pv[8 * RPG];
  const float2* LU = LUall + (long long)blockIdx.x * m * m;
  const int* piv = pivall + (long long)blockIdx.x * m;
  float2* inv = invall + (long long)blockIdx.x * m * m;
  const int j0 = blockIdx.y * 32;
  const int tid = threadIdx.x, c = tid & 31, g = tid >> 5;
  const int r0 = g * RPG;
  // L column k below the diagonal (rows k + 1 .. m - 1) into buffer k % 3
  auto fetch_l = [&](int k) {
    if (k < m - 1)
      for (int i = k + 1 + tid; i < m; i += 256) cp_async8(&col[k % 3][i], LU + (long long)k * m + i);
    cp_async_commit();
  };
  // U column k above the diagonal (rows 0 .. k - 1) into buffer (m - 1 - k) % 3
  auto fetch_u = [&](int k) {
    if (k > 0)
      for (int i = tid; i < k; i += 256) cp_async8(&col[(m - 1 - k) % 3][i], LU + (long long)k * m + i);
    cp_async_commit();
  };
  fetch_l(0);
  fetch_l(1);
  for (int k = tid; k < m; k += 256) {
    const float2 u = LU[(long long)k * m + k];
    const float q = 1.f / (u.x * u.x + u.y * u.y);
    dinv[k] = make_float2(u.x * q, -u.y * q);
    pv[k] = piv[k];
  }
  __syncthreads();
  // P e_{j0 + c}: apply the row swaps in order to the index of the unit entry
  int one = j0 + c;
  for (int k = 0; k < m; ++k) {
    const int p = pv[k];
    if (one == k) one = p;
    else if (one == p) one = k;
  }
  float2 y[RPG];
#pragma unroll
  for (int q = 0; q < RPG; ++q) y[q] = make_float2((j0 + c < m && r0 + q == one) ? 1.f : 0.f, 0.f);
  // forward substitution with unit lower L
  if (r0 <= 0 && 0 < r0 + RPG) rowk[0][c] = y[0];
  cp_async_wait1();   // column 0
  __syncthreads();
  for (int k = 0; k < m - 1; ++k) {
    const int b = k & 1;
    fetch_l(k + 2);
    const float2* lk = col[k % 3];
    const float2 yk = rowk[b][c];
    if (r0 + RPG > k + 1) {   // warp-uniform: this row group still has rows below k
#pragma unroll
      for (int q = 0; q < RPG; ++q) {
        const int i = r0 + q;
        if (i > k && i < m) {
          const float2 l = lk[i];
          y[q].x -= l.x * yk.x - l.y * yk.y;
          y[q].y -= l.x * yk.y + l.y * yk.x;
        }
      }
    }
    // the owner of row k + 1 publishes it for the next step
    if (r0 <= k + 1 && k + 1 < r0 + RPG) {
#pragma unroll
      for (int q = 0; q < RPG; ++q)
        if (r0 + q == k + 1) rowk[b ^ 1][c] = y[q];
    }
    cp_async_wait1();   // column k + 1
    __syncthreads();
  }
  // back substitution with U: row k of the result is y_k / U[k][k]
  cp_async_wait0();
  __syncthreads();     // every buffer free
  fetch_u(m - 1);
  fetch_u(m - 2);
  if (r0 <= m - 1 && m - 1 < r0 + RPG) {
#pragma unroll
    for (int q = 0; q < RPG; ++q)
      if (r0 + q == m - 1) rowk[0][c] = y[q];
  }
  cp_async_wait1();   // column m - 1
  __syncthreads();
  for (int k = m - 1; k >= 0; --k) {
    const int b = (m - 1 - k) & 1;
    fetch_u(k - 2);
    const float2* uk = col[(m - 1 - k) % 3];
    const float2 yk = cmul(rowk[b][c], dinv[k]);
    if (g == 0 && j0 + c < m) inv[(long long)k * m + j0 + c] = yk;
    if (r0 < k) {
#pragma unroll
      for (int q = 0; q < RPG; ++q) {
        const int i = r0 + q;
        if (i < k) {
          const float2 u = uk[i];
          y[q].x -= u.x * yk.x - u.y * yk.y;
          y[q].y -= u.x * yk.y + u.y * yk.x;
        }
      }
    }
    if (k > 0 && r0 <= k - 1 && k - 1 < r0 + RPG) {
#pragma unroll
      for (int q = 0; q < RPG; ++q)
        if (r0 + q == k - 1) rowk[b ^ 1][c] = y[q];
    }
    cp_async_wait1();   // column k - 1
    __syncthreads();
  }
  cp_async_wait0();
}

// ---------------------------------------------------------------------------
// 6. apply kernels
// ---------------------------------------------------------------------------
// Kept blocks: warp per row, the block's rows shared by f and n - f.
template <class C>
__global__ void __launch_bounds__(256) k_block_gemv(const C* __restrict__ inv, const int* __restrict__ blkf,
                                                    const C* __restrict__ R, C* __restrict__ Z, int m, int n,
                                                    int ny_nz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* r = reinterpret_cast<C*>(smem_raw);   // [2][m]
  const int s = blockIdx.x;
  const int f = blkf[s];
  const int f2 = (n - f) % n;
  const bool pair = (f2 != f);
  const C* D = inv + (long long)s * m * m;
  const int rows_per = (m + gridDim.y - 1) / gridDim.y;
  const int r0 = blockIdx.y * rows_per, r1 = min(m, r0 + rows_per);
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    r[j] = R[(long long)j * n + f];
    if (pair) {
      C v = R[(long long)j * n + f2];
      if (j < ny_nz) { v.x = -v.x; v.y = -v.y; }
      r[m + j] = v;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = r0 + warp; i < r1; i += nw) {
    const C* row = D + (long long)i * m;
    C a1 = czero<C>(), a2 = czero<C>();
    for (int j = lane; j < m; j += 32) {
      // streamed once per application: evict-first, so that the blocks do
      // not push the Krylov basis out of L2
      const C d = __ldcs(row + j);
      cfma(a1, d, r[j]);
      if (pair) cfma(a2, d, r[m + j]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a1.x += __shfl_xor_sync(0xffffffffu, a1.x, o);
      a1.y += __shfl_xor_sync(0xffffffffu, a1.y, o);
      a2.x += __shfl_xor_sync(0xffffffffu, a2.x, o);
      a2.y += __shfl_xor_sync(0xffffffffu, a2.y, o);
    }
    if (lane == 0) {
      Z[(long long)i * n + f] = a1;
      if (pair) {
        if (i < ny_nz) { a2.x = -a2.x; a2.y = -a2.y; }
        Z[(long long)i * n + f2] = a2;
      }
    }
  }
}

// Discarded frequencies: Z[f] = D_rep^{-1} R[f], one multi-right-hand-side
// product.  Register-tiled: a block of 256 threads computes GB_F frequencies
// x GB_I rows, each thread a 2 x 4 complex micro-tile; K advances GB_K
// columns at a time through shared memory, the next tile prefetched into
// registers while the current one is consumed.
constexpr int GB_F = 32, GB_I = 64, GB_K = 16;
template <class C>
__global__ void __launch_bounds__(256) k_rep_gemm(const C* __restrict__ Drep, const int* __restrict__ disc, int ndisc,
                                                  const C* __restrict__ R, C* __restrict__ Z, int m, int n) {
  __shared__ C Rs[GB_K][GB_F];
  __shared__ C Ds[GB_K][GB_I];
  __shared__ int fidx[GB_F];
  const int f0 = blockIdx.x * GB_F, i0 = blockIdx.y * GB_I;
  const int tid = threadIdx.x;
  const int tf = tid % 16, ti = tid / 16;   // 16 x 16 threads: 2 frequencies x 4 rows each
  if (tid < GB_F) fidx[tid] = (f0 + tid < ndisc) ? disc[f0 + tid] : -1;
  __syncthreads();
  // global -> register staging: R tile 32x16 (2 per thread), D tile 64x16 (4 per thread)
  C rr[2], dr[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      // consecutive threads walk consecutive frequencies of one row p
      const int e = tid + u * 256, a = e % GB_F, b = e / GB_F;
      const int f = fidx[a];
      rr[u] = (f >= 0 && k0 + b < m) ? R[(long long)(k0 + b) * n + f] : czero<C>();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + u * 256, a = e / GB_K, b = e % GB_K;
      dr[u] = (i0 + a < m && k0 + b < m) ? Drep[(long long)(i0 + a) * m + k0 + b] : czero<C>();
    }
  };
  C acc[2][4];
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = czero<C>();
  fetch(0);
  for (int k0 = 0; k0 < m; k0 += GB_K) {
#pragma unroll
    for (int u = 0; u < 2; ++u) { const int e = tid + u * 256; Rs[e / GB_F][e % GB_F] = rr[u]; }
#pragma unroll
    for (int u = 0; u < 4; ++u) { const int e = tid + u * 256; Ds[e % GB_K][e / GB_K] = dr[u]; }
    __syncthreads();
    if (k0 + GB_K < m) fetch(k0 + GB_K);
#pragma unroll
    for (int k = 0; k < GB_K; ++k) {
      C a[2], b[4];
#pragma unroll
      for (int p = 0; p < 2; ++p) a[p] = Rs[k][tf * 2 + p];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Ds[k][ti * 4 + q];
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) cfma(acc[p][q], b[q], a[p]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int f = fidx[tf * 2 + p];
    if (f < 0) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + ti * 4 + q;
      if (i < m) Z[(long long)i * n + f] = acc[p][q];
    }
  }
}

// Representative-block product on the tensor cores (tcgen05, kind::tf32,
// accumulator in TMEM), complex FP32 through a real formulation with the
// real and imaginary parts of each source row p interleaved along K:
//   C[t][2i + c] = sum_k A[t][k] B[2i + c][k],   k = 2p + c' < 2m,
//   A[t][2p] = Re R[p][f_t],  A[t][2p+1] = Im R[p][f_t],
//   B[2i][2p] = Re D[i][p],   B[2i][2p+1] = -Im D[i][p],
//   B[2i+1][2p] = Im D[i][p], B[2i+1][2p+1] = Re D[i][p],
// so C's columns are the interleaved real and imaginary parts of Z[i][f_t].
// Each fp32 operand is split into tf32 hi + lo and the product accumulates
// hi*hi + hi*lo + lo*hi (FP32-level accuracy).
//
// Both operands are packed in global memory in the order the MMA reads them
// from shared memory (K-major core matrices, chunks of TC_KC along K, hi then
// lo), so every K-chunk of a tile is one contiguous bulk copy: B once per
// build, A by a gather kernel per apply.  The GEMM is a TC_STAGES-deep ring:
// one thread issues the bulk copies, one issues the MMAs, and the commit of a
// chunk's MMAs frees its stage.
// The N tile (TN = 64 or 32 columns of C, i.e. 32 or 16 rows of D) is chosen
// per shape by the autotuner: the smaller tile runs twice the CTAs.
constexpr int TC_M = 128, TC_KC = 32, TC_STAGES = 4;
constexpr int TC_ACHUNK = 2 * TC_M * TC_KC;   // floats per packed A chunk (hi + lo)
__host__ __device__ constexpr int tc_bchunk(int tn) { return 2 * tn * TC_KC; }   // floats per packed B chunk
__host__ __device__ constexpr int tc_stage_bytes(int tn) { return (TC_ACHUNK + tc_bchunk(tn)) * 4; }
constexpr size_t tc_smem(int tn) { return (size_t)TC_STAGES * tc_stage_bytes(tn); }

// (row, k) of slot q of a K-major core-matrix chunk with TC_KC columns
__device__ __forceinline__ void tc_slot(int q, int& row, int& k) {
  row = (q >> 8) * 8 + ((q >> 2) & 7);
  k = ((q >> 5) & 7) * 4 + (q & 3);
}

// B operand of one representative block, packed [N tile][chunk][hi | lo]
template <int TN>
__global__ void k_bpack(const float2* __restrict__ D, float* __restrict__ Bp, int m) {
  constexpr int TC_BCHUNK = tc_bchunk(TN);
  const int nchunks = 2 * m / TC_KC;
  const long long total = (long long)(2 * m / TN) * nchunks * (TN * TC_KC);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e % (TN * TC_KC));
    const int ct = (int)(e / (TN * TC_KC));
    const int nt = ct / nchunks, c = ct - nt * nchunks;
    int row, k;
    tc_slot(q, row, k);
    const int nrow = nt * TN + row, kg = c * TC_KC + k;
    const float2 d = D[(long long)(nrow >> 1) * m + (kg >> 1)];
    const int co = nrow & 1, ci = kg & 1;
    const float v = co == 0 ? (ci == 0 ? d.x : -d.y) : (ci == 0 ? d.y : d.x);
    float hi, lo;
    umma::split_tf32(v, hi, lo);
    Bp[(long long)ct * TC_BCHUNK + q] = hi;
    Bp[(long long)ct * TC_BCHUNK + TN * TC_KC + q] = lo;
  }
}

// A operand: the discarded frequencies' columns of R (line-major [p][f]),
// packed [M tile][chunk][hi | lo]; each thread takes one (re, im) pair
__global__ void k_apack(const float2* __restrict__ R, const int* __restrict__ disc, int ndisc, int m, int n,
                        float* __restrict__ Ap) {
  const int nchunks = 2 * m / TC_KC;
  const long long total = (long long)((ndisc + TC_M - 1) / TC_M) * nchunks * (TC_M * TC_KC / 2);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int q = 2 * (int)(e % (TC_M * TC_KC / 2));
    const int ct = (int)(e / (TC_M * TC_KC / 2));
    const int mt = ct / nchunks, c = ct - mt * nchunks;
    int row, k;
    tc_slot(q, row, k);
    const int t = mt * TC_M + row;
    const int p = (c * TC_KC + k) >> 1;
    const float2 v = t < ndisc ? R[(long long)p * n + disc[t]] : make_float2(0.f, 0.f);
    float2 hi, lo;
    umma::split_tf32(v.x, hi.x, lo.x);
    umma::split_tf32(v.y, hi.y, lo.y);
    *(float2*)(Ap + (long long)ct * TC_ACHUNK + q) = hi;
    *(float2*)(Ap + (long long)ct * TC_ACHUNK + TC_M * TC_KC + q) = lo;
  }
}

template <int TC_N>
__global__ void __launch_bounds__(128) k_rep_gemm_tc(const float* __restrict__ Ap, const float* __restrict__ Bp,
                                                     const int* __restrict__ disc, int ndisc,
                                                     float2* __restrict__ Z, int m, int n, int* __restrict__ err) {
  constexpr int TC_BCHUNK = tc_bchunk(TC_N);
  constexpr int TC_STAGE_BYTES = tc_stage_bytes(TC_N);
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], done;
  __shared__ uint32_t tslot;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, nt = blockIdx.y;
  const int nchunks = 2 * m / TC_KC;
  const unsigned long long kLimitNs = 1000000000ull;   // 1 s per wait
  if (warp == 2) umma::tmem_alloc(&tslot, TC_N);
  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) { umma::mbar_init(&full[s], 1); umma::mbar_init(&empty[s], 1); }
    umma::mbar_init(&done, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tslot;

  if (tid == 0) {
    // producer: chunk c into stage c % TC_STAGES once the MMAs of chunk c - TC_STAGES are done
    const float* a = Ap + (long long)mt * nchunks * TC_ACHUNK;
    const float* b = Bp + (long long)nt * nchunks * TC_BCHUNK;
    int issued = 0;
    for (int c = 0; c < nchunks; ++c) {
      const int s = c % TC_STAGES;
      if (c >= TC_STAGES && !umma::mbar_wait_ns(&empty[s], ((c / TC_STAGES) - 1) & 1, kLimitNs)) {
        atomicExch(&failed, 1);
        break;
      }
      unsigned char* st = smem + (size_t)s * TC_STAGE_BYTES;
      umma::mbar_arrive_expect_tx(&full[s], TC_STAGE_BYTES);
      umma::bulk_g2s(st, a + (long long)c * TC_ACHUNK, TC_ACHUNK * 4, &full[s]);
      umma::bulk_g2s(st + TC_ACHUNK * 4, b + (long long)c * TC_BCHUNK, TC_BCHUNK * 4, &full[s]);
      issued = c + 1;
    }
    // every copy issued must land before the block may exit
    for (int c = (issued > TC_STAGES ? issued - TC_STAGES : 0); c < issued; ++c)
      umma::mbar_wait_ns(&full[c % TC_STAGES], (c / TC_STAGES) & 1, kLimitNs);
  } else if (tid == 32) {
    // MMA issuer
    const uint32_t idesc = umma::idesc_tf32(TC_M, TC_N);
    const uint32_t lbo = 128, sbo = (TC_KC / 4) * 128;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int s = c % TC_STAGES;
      if (!umma::mbar_wait_ns(&full[s], (c / TC_STAGES) & 1, kLimitNs)) { ok = false; break; }
      umma::fence_after_sync();
      const uint32_t base = umma::smem_u32(smem + (size_t)s * TC_STAGE_BYTES);
      const uint32_t ah = base, al = base + TC_M * TC_KC * 4;
      const uint32_t bh = base + TC_ACHUNK * 4, bl = bh + TC_N * TC_KC * 4;
#pragma unroll
      for (int ks = 0; ks < TC_KC / 8; ++ks) {
        const uint32_t o = ks * 256;
        umma::mma_tf32(tmem, umma::smem_desc(ah + o, lbo, sbo), umma::smem_desc(bh + o, lbo, sbo), idesc,
                       (c | ks) ? 1u : 0u);
        umma::mma_tf32(tmem, umma::smem_desc(ah + o, lbo, sbo), umma::smem_desc(bl + o, lbo, sbo), idesc, 1u);
        umma::mma_tf32(tmem, umma::smem_desc(al + o, lbo, sbo), umma::smem_desc(bh + o, lbo, sbo), idesc, 1u);
      }
      umma::commit(&empty[s]);
    }
    if (!ok) atomicExch(&failed, 1);
    umma::commit(&done);   // tracks every MMA issued above
  }
  __syncwarp();
  const bool ok = umma::mbar_wait_ns(&done, 0, kLimitNs);
  __syncthreads();
  if (!ok || failed) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    umma::fence_after_sync();
    const int t = mt * TC_M + 32 * warp + lane;
    const int f = t < ndisc ? disc[t] : -1;
#pragma unroll
    for (int col0 = 0; col0 < TC_N; col0 += 16) {
      float v[16];
      umma::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + col0, v);
      if (f >= 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int io = (nt * TC_N + col0) / 2 + q;
          Z[(long long)io * n + f] = make_float2(v[2 * q], v[2 * q + 1]);
        }
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 2) umma::tmem_dealloc(tmem, TC_N);
}

// the representative block's B operand packed for N tile tn (64 or 32)
static vie_status rep_pack(vie_plan_s* P, BoxPrec& B, int tn) {
  const int m = B.m;
  const long long nch = 2LL * m / TC_KC;
  VIE_TRY(B.bpack.alloc(sizeof(float) * (size_t)(2 * m / tn) * nch * tc_bchunk(tn)));
  const float2* rep = B.inv64.as<float2>() + (size_t)B.rep * m * m;
  Prof pf_("bpack", P->st);
  if (tn == 64) k_bpack<64><<<152 * 4, 256, 0, P->st>>>(rep, B.bpack.as<float>(), m);
  else k_bpack<32><<<152 * 4, 256, 0, P->st>>>(rep, B.bpack.as<float>(), m);
  count_launch();
  VIE_CHECK_LAUNCH();
  B.tc_n = tn;
  return VIE_OK;
}

// the discarded frequencies' product on the tensor cores with the packed N tile
static vie_status launch_rep_tc(vie_plan_s* P, BoxPrec& B, float2* zh, cudaStream_t st) {
  const int m = B.m;
  Prof pf_("rep_gemm_tc", st);
  dim3 grid(ceil_div(B.ndisc, TC_M), (2 * m) / B.tc_n);
  if (B.tc_n == 64) {
    VIE_TRY(smem_optin(k_rep_gemm_tc<64>, tc_smem(64)));
    k_rep_gemm_tc<64><<<grid, 128, tc_smem(64), st>>>(B.apack.as<float>(), B.bpack.as<float>(), B.disc.as<int>(),
                                                      B.ndisc, zh, m, B.n, P->dev_err.as<int>());
  } else {
    VIE_TRY(smem_optin(k_rep_gemm_tc<32>, tc_smem(32)));
    k_rep_gemm_tc<32><<<grid, 128, tc_smem(32), st>>>(B.apack.as<float>(), B.bpack.as<float>(), B.disc.as<int>(),
                                                      B.ndisc, zh, m, B.n, P->dev_err.as<int>());
  }
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

// autotuner: N tile of the tensor-core product (64 or 32; the MMAs of every
// output element run the same K chunks in the same order either way), timed
// on the box's own operands, cached per shape
static vie_status tune_rep_tc(vie_plan_s* P, BoxPrec& B) {
  if (!autotune_enabled() || (2 * B.m) % 64 != 0) return VIE_OK;
  const TuneKey key{4, 0, B.m, B.ndisc, B.n};
  int choice;
  std::string rep;
  if (!tune_cache_get(key, &choice, &rep)) {
    VIE_CUDA(cudaMemsetAsync(B.apack.p, 0, B.apack.bytes, P->st));
    char buf[160];
    snprintf(buf, sizeof(buf), "rep_gemm_tc m=%d discarded=%d n=%d:", B.m, B.ndisc, B.n);
    rep = buf;
    int best = 0;
    float tbest = 0;
    for (int tn : {64, 32}) {
      VIE_TRY(rep_pack(P, B, tn));
      float ms = 0;
      VIE_TRY(time_ms(P->st, 3, [&] { return launch_rep_tc(P, B, B.zhat64.as<float2>(), P->st); }, &ms));
      snprintf(buf, sizeof(buf), " N tile %d %.4f ms;", tn, ms);
      rep += buf;
      if (best == 0 || ms < tbest) { best = tn; tbest = ms; }
    }
    snprintf(buf, sizeof(buf), " chosen %d\n", best);
    rep += buf;
    choice = best;
    tune_cache_put(key, choice, rep);
  }
  if (B.tc_n != choice) VIE_TRY(rep_pack(P, B, choice));
  P->tuning += rep;
  return VIE_OK;
}

// force the N tile of every box's tensor-core product (test hook)
vie_status precond_set_rep_tile(vie_plan_s* P, int tn) {
  for (auto& Bp : P->bp) {
    BoxPrec& B = *Bp;
    if (!B.bpack.p) continue;
    if ((2 * B.m) % tn != 0) { set_error("vie_plan_set_tuning: 2m is not a multiple of the N tile"); return VIE_EINVAL; }
    VIE_TRY(rep_pack(P, B, tn));
  }
  VIE_CUDA(cudaStreamSynchronize(P->st));
  return VIE_OK;
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
static BoxDims dims_of(const vie_plan_s* P, const vie_box& b) {
  BoxDims d;
  d.x0 = b.x0; d.y0 = b.y0; d.z0 = b.z0; d.n = b.nx; d.ny = b.ny; d.nz = b.nz;
  d.m = 3 * b.ny * b.nz;
  d.gnx = P->nx; d.gny = P->ny; d.gnz = P->nz;
  return d;
}

void precond_free(vie_plan_s* P) {
  P->bp.clear();
  P->prec_built = false;
  P->precond_bytes = 0;
  P->precond_blocks = 0;
  P->precond_discarded = 0;
}

// Homogenised M~ of a box as [nz][ny] (Sec. 5.2): mode over the box, or the
// (real) mean along x (1-level) or over each z-plane (2-level, plane = true).
vie_status box_homogenise(vie_plan_s* P, const vie_box& b, DevBuf& Mt, bool plane) {
  const BoxDims bd = dims_of(P, b);
  cudaStream_t st = P->st;
  VIE_TRY(Mt.alloc(sizeof(double2) * bd.ny * bd.nz));
  DevBuf err;
  VIE_TRY(err.alloc(sizeof(int)));
  VIE_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
  const int real_only = P->opts.homog == VIE_HOM_REALMEAN ? 1 : 0;
  if (P->opts.homog == VIE_HOM_MODE) {
    k_hom_mode<<<1, 1024, 0, st>>>(P->M128.as<double2>(), Mt.as<double2>(), bd, err.as<int>());
  } else if (plane) {
    k_hom_plane<<<bd.nz, 256, 0, st>>>(P->M128.as<double2>(), Mt.as<double2>(), bd, real_only);
  } else {
    const int t = bd.ny * bd.nz;
    k_hom_mean<<<ceil_div(t, 128), 128, 0, st>>>(P->M128.as<double2>(), Mt.as<double2>(), bd, real_only);
  }
  count_launch();
  VIE_CHECK_LAUNCH();
  int herr = 0;
  VIE_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  VIE_CUDA(cudaStreamSynchronize(st));
  if (herr) { set_error("mode homogenisation: more than %d distinct values in a box", MODE_MAXV); return VIE_EINVAL; }
  return VIE_OK;
}

// batched LU of nblk column-major m x m blocks in place (panel + trailing
// update per 16 columns)
template <class C>
static vie_status lu_factor(vie_plan_s* P, C* A, int* piv, int* info, int m, int nblk) {
  cudaStream_t st = P->st;
  const size_t smem = sizeof(C) * (size_t)LU_NB * m;
  VIE_TRY(smem_optin(k_lu_panel<C>, smem));
  const bool c64 = sizeof(C) == 8;
  for (int k0 = 0; k0 < m; k0 += LU_NB) {
    const int nb = std::min(LU_NB, m - k0);
    {
      Prof pf_(c64 ? "lu_panel_c64" : "lu_panel", st);
      k_lu_panel<C><<<nblk, 512, smem, st>>>(A, piv, m, k0, info);
      count_launch();
    }
    const int r22 = m - k0 - nb;
    if (r22 > 0) {
      const int nti = ceil_div(r22, LU_TILE);
      Prof pf_(c64 ? "lu_update_c64" : "lu_update", st);
      k_lu_update<C><<<dim3(nti * nti, nblk), 256, 0, st>>>(A, m, k0, nb);
      count_launch();
    }
    VIE_CHECK_LAUNCH();
  }
  return VIE_OK;
}

// LU with partial pivoting of nblk column-major m x m blocks (FP64, in
// place in LU), then the explicit inverses, row-major: complex FP64
// (want128) from the FP64 factors, complex FP32 (want64) from the complex-FP32
// LU of the blocks rounded to FP32 (or from the FP64 factors rounded to FP32
// when both are wanted).  The complex-FP32 inverse carries FP32 rounding
// either way; factoring in FP32 runs at the FP32 rate, which on this part is
// about 58 times the FP64 rate.  VIE_EINVAL if a block is singular.
vie_status factor_invert_blocks(vie_plan_s* P, DevBuf& LU, int m, int nblk, bool want64, DevBuf* inv64, bool want128,
                                DevBuf* inv128) {
  cudaStream_t st = P->st;
  const size_t mm = (size_t)m * m;
  DevBuf piv, info, LU32;
  VIE_TRY(piv.alloc(sizeof(int) * (size_t)m * nblk));
  VIE_TRY(info.alloc(sizeof(int)));
  VIE_CUDA(cudaMemsetAsync(info.p, 0, sizeof(int), st));
  if (want128) VIE_TRY(lu_factor<double2>(P, LU.as<double2>(), piv.as<int>(), info.as<int>(), m, nblk));
  if (want64) {
    VIE_TRY(LU32.alloc(sizeof(float2) * mm * nblk));
    const long long tot = (long long)mm * nblk;
    k_lu_narrow<<<(int)std::min<long long>((tot + 255) / 256, 152LL * 16), 256, 0, st>>>(LU.as<double2>(),
                                                                                        LU32.as<float2>(), tot);
    count_launch();
    VIE_CHECK_LAUNCH();
    if (!want128) VIE_TRY(lu_factor<float2>(P, LU32.as<float2>(), piv.as<int>(), info.as<int>(), m, nblk));
  }
  // column chunk of the inverse: m x (CB + 3) elements of shared memory
  auto chunk = [&](size_t esz) { return (int)std::max<size_t>(1, std::min<size_t>(32, (200 * 1024) / (esz * m) - 3)); };
  if (want64) {
    const int CB = chunk(sizeof(float2));
    dim3 gi(nblk, ceil_div(m, CB));
    VIE_TRY(inv64->alloc(sizeof(float2) * mm * nblk));
    if (m <= 8 * 72) {
      // register-blocked: 8 row groups x 32 columns per CTA
      dim3 gr(nblk, ceil_div(m, 32));
      Prof pf_("block_inv_c64", st);
      if (m <= 8 * 16) k_block_inv_rb<16><<<gr, 256, 0, st>>>(LU32.as<float2>(), piv.as<int>(), inv64->as<float2>(), m);
      else if (m <= 8 * 32) k_block_inv_rb<32><<<gr, 256, 0, st>>>(LU32.as<float2>(), piv.as<int>(), inv64->as<float2>(), m);
      else if (m <= 8 * 48) k_block_inv_rb<48><<<gr, 256, 0, st>>>(LU32.as<float2>(), piv.as<int>(), inv64->as<float2>(), m);
      else k_block_inv_rb<72><<<gr, 256, 0, st>>>(LU32.as<float2>(), piv.as<int>(), inv64->as<float2>(), m);
    } else {
      const size_t smem = sizeof(float2) * (size_t)m * (CB + 3);
      VIE_TRY(smem_optin(k_block_inv<float2>, smem));
      Prof pf_("block_inv_c64", st);
      k_block_inv<float2><<<gi, 256, smem, st>>>(LU32.as<float2>(), piv.as<int>(), inv64->as<float2>(), m, CB);
    }
    count_launch();
    VIE_CHECK_LAUNCH();
  }
  if (want128) {
    const int CB = chunk(sizeof(double2));
    dim3 gi(nblk, ceil_div(m, CB));
    VIE_TRY(inv128->alloc(sizeof(double2) * mm * nblk));
    const size_t smem = sizeof(double2) * (size_t)m * (CB + 3);
    VIE_TRY(smem_optin(k_block_inv<double2>, smem));
    { Prof pf_("block_inv_c128", st);
      k_block_inv<double2><<<gi, 256, smem, st>>>(LU.as<double2>(), piv.as<int>(), inv128->as<double2>(), m, CB); }
    count_launch();
    VIE_CHECK_LAUNCH();
  }
  int hinfo = 0;
  VIE_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  VIE_CUDA(cudaStreamSynchronize(st));
  if (hinfo) { set_error("preconditioner: singular block D_f"); return VIE_EINVAL; }
  return VIE_OK;
}

// the kept-block product of a 1-level box with `split` CTAs per block (0: the
// default rule, enough CTAs for about four per SM)
template <class C>
static vie_status launch_block_gemv(BoxPrec& B, const C* inv, const C* rh, C* zh, int split, cudaStream_t st) {
  const int m = B.m;
  const size_t smem = sizeof(C) * 2 * m;
  if (split <= 0) split = std::max(1, std::min(8, (4 * 152 + B.nhalf - 1) / B.nhalf));
  Prof pf_(sizeof(C) == 8 ? "block_gemv_c64" : "block_gemv_c128", st);
  dim3 grid(B.nhalf, split);
  k_block_gemv<C><<<grid, 256, smem, st>>>(inv, B.blkf.as<int>(), rh, zh, m, B.n, B.b.ny * B.b.nz);
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

// autotuner: CTAs per block of the kept-block product (every split computes
// each output row with one warp in the same order, so results do not depend
// on the choice); timed on the box's own blocks, cached per shape
template <class C>
static vie_status tune_gemv(vie_plan_s* P, BoxPrec& B, int pi) {
  if (B.nhalf <= 0 || !autotune_enabled()) return VIE_OK;
  const TuneKey key{1, pi, B.m, B.nhalf, B.n};
  int choice;
  std::string rep;
  if (!tune_cache_get(key, &choice, &rep)) {
    C* inv = (C*)(pi == 0 ? B.inv64.p : B.inv128.p);
    C* rh = (C*)(pi == 0 ? B.rhat64.p : B.rhat128.p);
    C* zh = (C*)(pi == 0 ? B.zhat64.p : B.zhat128.p);
    VIE_CUDA(cudaMemsetAsync(rh, 0, sizeof(C) * (size_t)B.n * B.m, P->st));
    char buf[160];
    snprintf(buf, sizeof(buf), "block_gemv_%s m=%d blocks=%d n=%d:", pi == 0 ? "c64" : "c128", B.m, B.nhalf, B.n);
    rep = buf;
    int best = 0;
    float tbest = 0;
    for (int split : {1, 2, 4, 8}) {
      if (split > 1 && B.m / split < 16) break;
      float ms = 0;
      VIE_TRY(time_ms(P->st, 3, [&] { return launch_block_gemv<C>(B, inv, rh, zh, split, P->st); }, &ms));
      snprintf(buf, sizeof(buf), " split %d %.4f ms;", split, ms);
      rep += buf;
      if (best == 0 || ms < tbest) { best = split; tbest = ms; }
    }
    snprintf(buf, sizeof(buf), " chosen %d\n", best);
    rep += buf;
    choice = best;
    tune_cache_put(key, choice, rep);
  }
  B.gemv_split[pi] = choice;
  P->tuning += rep;
  return VIE_OK;
}

static vie_status build_box(vie_plan_s* P, BoxPrec& B, bool want64, bool want128) {
  const BoxDims bd = dims_of(P, B.b);
  cudaStream_t st = P->st;
  const int n = bd.n, m = bd.m;
  B.n = n; B.m = m;
  B.rep = (n + 1) / 2 - 1;
  VIE_TRY(fft_get(n, &B.fx));
  // 1. homogenise
  VIE_TRY(box_homogenise(P, B.b, B.Mt, false));
  // 2. Chan coefficients and eigenvalues (frequency-major)
  const int ndy = 2 * bd.ny - 1, ndz = 2 * bd.nz - 1;
  const int nl = 6 * ndz * ndy;
  DevBuf coef;
  VIE_TRY(coef.alloc(sizeof(double2) * (size_t)nl * n));
  VIE_TRY(B.lam.alloc(sizeof(double2) * (size_t)nl * n));
  const double2 self = self_term_value(P->h, P->kb);
  {
    const long long total = (long long)nl * n;
    const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    Prof pf_("chan_coeffs", st);
    k_chan_coeffs<<<grid, 256, 0, st>>>(coef.as<double2>(), bd, P->h, P->kb, self);
    count_launch();
    VIE_CHECK_LAUNCH();
  }
  {
    DevBuf tmp;
    const size_t ts = fft_scratch_elems<double2>(*B.fx, nl);
    if (ts) VIE_TRY(tmp.alloc(sizeof(double2) * ts));
    LineDesc ld = lines_flat(n, n, nl, n, 1, 1, nl);   // out: [f][line]
    VIE_TRY(fft_lines<double2>(coef.as<double2>(), B.lam.as<double2>(), ld, *B.fx, -1, 1.0, tmp.as<double2>(), st));
    VIE_CUDA(cudaStreamSynchronize(st));
  }
  coef.release();
  // 3. proxy and selection
  VIE_TRY(B.vhat.alloc(sizeof(double) * n));
  VIE_TRY(B.fmap.alloc(sizeof(int) * n));
  VIE_TRY(B.fsgn.alloc(sizeof(int) * n));
  VIE_TRY(B.disc.alloc(sizeof(int) * n));
  VIE_TRY(B.blkf.alloc(sizeof(int) * (n / 2 + 2)));
  DevBuf cnt;
  VIE_TRY(cnt.alloc(sizeof(int) * 8));
  k_select<<<1, 1024, 0, st>>>(B.lam.as<double2>(), B.Mt.as<double2>(), bd, P->opts.reduce_tol, B.vhat.as<double>(),
                               B.fmap.as<int>(), B.fsgn.as<int>(), B.disc.as<int>(), B.blkf.as<int>(), cnt.as<int>());
  count_launch();
  VIE_CHECK_LAUNCH();
  int hc[8] = {0};
  VIE_CUDA(cudaMemcpyAsync(hc, cnt.p, sizeof(int) * 8, cudaMemcpyDeviceToHost, st));
  VIE_CUDA(cudaStreamSynchronize(st));
  B.nblk = hc[0];
  B.nkept = hc[1];
  B.ndisc = hc[2];
  B.rep = hc[3];     // now the representative's slot
  B.nhalf = hc[4];   // number of kept slots (they come first)
  // 4. assemble the stored blocks (FP64, column-major)
  DevBuf LU;
  const size_t mm = (size_t)m * m;
  VIE_TRY(LU.alloc(sizeof(double2) * mm * B.nblk));
  {
    const long long total = (long long)mm * B.nblk;
    const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
    Prof pf_("block_assemble", st);
    k_block_assemble<<<grid, 256, 0, st>>>(LU.as<double2>(), B.lam.as<double2>(), B.Mt.as<double2>(),
                                           B.blkf.as<int>(), bd, B.nblk);
    count_launch();
    VIE_CHECK_LAUNCH();
  }
  // 5. FP64 LU, then the inverse(s)
  VIE_TRY(factor_invert_blocks(P, LU, m, B.nblk, want64, &B.inv64, want128, &B.inv128));
  if (want64) {
    VIE_TRY(B.rhat64.alloc(sizeof(float2) * (size_t)n * m));
    VIE_TRY(B.zhat64.alloc(sizeof(float2) * (size_t)n * m));
    // tensor-core operands of the representative-block product (tf32 hi/lo split)
    if ((2 * m) % 32 == 0 && B.ndisc > 0) {
      const long long nch = 2LL * m / TC_KC;
      VIE_TRY(B.apack.alloc(sizeof(float) * (size_t)ceil_div(B.ndisc, TC_M) * nch * TC_ACHUNK));
      VIE_TRY(rep_pack(P, B, (2 * m) % 64 == 0 ? 64 : 32));
    }
    const size_t ts = fft_scratch_elems<float2>(*B.fx, m);
    if (ts) VIE_TRY(B.tmp64.alloc(sizeof(float2) * ts));
  }
  if (want128) {
    VIE_TRY(B.rhat128.alloc(sizeof(double2) * (size_t)n * m));
    VIE_TRY(B.zhat128.alloc(sizeof(double2) * (size_t)n * m));
    const size_t ts = fft_scratch_elems<double2>(*B.fx, m);
    if (ts) VIE_TRY(B.tmp128.alloc(sizeof(double2) * ts));
  }
  if (want64) VIE_TRY(tune_gemv<float2>(P, B, 0));
  if (want128) VIE_TRY(tune_gemv<double2>(P, B, 1));
  if (want64 && B.bpack.p) VIE_TRY(tune_rep_tc(P, B));
  return VIE_OK;
}

vie_status precond_build(vie_plan_s* P) {
  reset_graphs(P);   // captured Arnoldi steps point at the old blocks
  P->tuning = P->tuning.substr(0, P->tuning_matvec);
  if (!P->side) {
    VIE_CUDA(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking));
    VIE_CUDA(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
    VIE_CUDA(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
  }
  precond_free(P);
  if (P->opts.precond == VIE_PREC_NONE) { P->prec_built = true; P->kept_fraction = 0; return VIE_OK; }
  const auto t0 = std::chrono::steady_clock::now();
  const bool want64 = P->opts.precision == VIE_MIXED;
  const bool want128 = P->opts.precision == VIE_FP64;
  long long kept = 0, total = 0, nblk = 0, ndisc = 0;
  size_t bytes = 0;
  for (const vie_box& b : P->boxes) {
    std::unique_ptr<BoxPrec> B(new BoxPrec());
    B->b = b;
    if (b.levels == 2) VIE_TRY(build_box2(P, *B, want64, want128));
    else VIE_TRY(build_box(P, *B, want64, want128));
    kept += B->nkept;
    total += B->n;
    bytes += B->inv64.bytes + B->inv128.bytes + B->bpack.bytes + B->apack.bytes;
    nblk += B->nblk;
    ndisc += B->ndisc;
    P->bp.push_back(std::move(B));
  }
  P->precond_bytes = bytes;
  P->precond_blocks = nblk;
  P->precond_discarded = ndisc;
  P->kept_fraction = total ? (double)kept / total : 0;
  P->prec_built = true;
  P->t_setup_ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return VIE_OK;
}

// The complex-FP64 inverses of a preconditioner built for the mixed solve
// (its blocks are rebuilt in the same order, so the selection and the
// complex-FP32 inverses stay as they are): used when a mixed solve falls
// back to FP64 GMRES.
vie_status precond_add_fp64(vie_plan_s* P) {
  if (!P->prec_built) { set_error("preconditioner not built"); return VIE_ESTATE; }
  size_t bytes = 0;
  for (auto& Bp : P->bp) {
    BoxPrec& B = *Bp;
    if (!B.inv128.p) {
      if (B.b.levels == 2) VIE_TRY(build_box2(P, B, false, true));
      else VIE_TRY(build_box(P, B, false, true));
    }
    bytes += B.inv64.bytes + B.inv128.bytes + B.bpack.bytes + B.apack.bytes;
  }
  P->precond_bytes = bytes;
  return VIE_OK;
}

template <class C> struct BoxBufs;
template <> struct BoxBufs<float2> {
  static float2* inv(BoxPrec& B) { return B.inv64.as<float2>(); }
  static float2* rh(BoxPrec& B) { return B.rhat64.as<float2>(); }
  static float2* zh(BoxPrec& B) { return B.zhat64.as<float2>(); }
  static float2* tmp(BoxPrec& B) { return B.tmp64.as<float2>(); }
};
template <> struct BoxBufs<double2> {
  static double2* inv(BoxPrec& B) { return B.inv128.as<double2>(); }
  static double2* rh(BoxPrec& B) { return B.rhat128.as<double2>(); }
  static double2* zh(BoxPrec& B) { return B.zhat128.as<double2>(); }
  static double2* tmp(BoxPrec& B) { return B.tmp128.as<double2>(); }
};

template <class C>
vie_status precond_apply(vie_plan_s* P, const C* r, C* z, cudaStream_t st) {
  const long long N = (long long)P->nx * P->ny * P->nz;
  if (!P->prec_built) { set_error("preconditioner not built"); return VIE_ESTATE; }
  const bool whole = P->bp.size() == 1 && P->boxes[0].nx == P->nx && P->boxes[0].ny == P->ny &&
                     P->boxes[0].nz == P->nz;
  if (P->opts.precond == VIE_PREC_NONE || !whole) {
    VIE_CUDA(cudaMemcpyAsync(z, r, sizeof(C) * 3 * N, cudaMemcpyDeviceToDevice, st));
    if (P->opts.precond == VIE_PREC_NONE) return VIE_OK;
  }
  for (auto& Bp : P->bp) {
    BoxPrec& B = *Bp;
    C* inv = BoxBufs<C>::inv(B);
    if (!inv) { set_error("preconditioner not built for this precision"); return VIE_ESTATE; }
    const int n = B.n, m = B.m, nyb = B.b.ny, nzb = B.b.nz;
    C* rh = BoxBufs<C>::rh(B);
    C* zh = BoxBufs<C>::zh(B);
    if (B.levels == 2) {
      VIE_TRY(apply_box2<C>(P, B, r, z, inv, rh, zh, BoxBufs<C>::tmp(B), st));
      continue;
    }
    // gather + x-FFT: line p = (alpha, zb, yb) -> R[p][f] (line-major)
    LineDesc ld{n, n, m, nyb, nzb,
                (long long)P->nx, (long long)P->ny * P->nx, N, 1,
                (long long)n, (long long)nyb * n, (long long)nyb * nzb * n, 1};
    const long long base = ((long long)B.b.z0 * P->ny + B.b.y0) * P->nx + B.b.x0;
    VIE_TRY(fft_lines<C>(r + base, rh, ld, *B.fx, -1, 1.0, BoxBufs<C>::tmp(B), st));
    // kept blocks (S1 pairs) on the plan stream and, for complex FP32 with a
    // packed representative block, the discarded frequencies on the tensor
    // cores on a second stream: the two write disjoint frequencies of zh and
    // overlap (HBM-bound GEMV beside the tensor-core product)
    const bool tc = B.ndisc > 0 && sizeof(C) == 8 && B.bpack.p;
    if (tc) {
      VIE_CUDA(cudaEventRecord(P->ev_fork, st));
      VIE_CUDA(cudaStreamWaitEvent(P->side, P->ev_fork, 0));
      cudaStream_t s2 = P->side;
      {
        Prof pf_("rep_apack", s2);
        k_apack<<<152 * 4, 256, 0, s2>>>((const float2*)rh, B.disc.as<int>(), B.ndisc, m, n, B.apack.as<float>());
        count_launch();
        VIE_CHECK_LAUNCH();
      }
      VIE_TRY(launch_rep_tc(P, B, (float2*)zh, s2));
    }
    if (B.nhalf > 0) VIE_TRY(launch_block_gemv<C>(B, inv, rh, zh, B.gemv_split[sizeof(C) == 16], st));
    if (tc) {
      VIE_CUDA(cudaEventRecord(P->ev_join, P->side));
      VIE_CUDA(cudaStreamWaitEvent(st, P->ev_join, 0));
    } else if (B.ndisc > 0) {
      Prof pf_(sizeof(C) == 8 ? "rep_gemm_c64" : "rep_gemm_c128", st);
      dim3 grid(ceil_div(B.ndisc, GB_F), ceil_div(m, GB_I));
      k_rep_gemm<C><<<grid, 256, 0, st>>>(inv + (size_t)B.rep * m * m, B.disc.as<int>(), B.ndisc, rh, zh, m, n);
      count_launch();
      VIE_CHECK_LAUNCH();
    }
    // inverse x-FFT + scatter
    LineDesc lo{n, n, m, nyb, nzb,
                (long long)n, (long long)nyb * n, (long long)nyb * nzb * n, 1,
                (long long)P->nx, (long long)P->ny * P->nx, N, 1};
    VIE_TRY(fft_lines<C>(zh, z + base, lo, *B.fx, +1, 1.0 / n, BoxBufs<C>::tmp(B), st));
  }
  return VIE_OK;
}

template vie_status precond_apply<float2>(vie_plan_s*, const float2*, float2*, cudaStream_t);
template vie_status precond_apply<double2>(vie_plan_s*, const double2*, double2*, cudaStream_t);

}  // namespace vie
