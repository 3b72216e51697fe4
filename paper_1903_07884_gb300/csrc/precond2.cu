// Chan-Olkin 2-level circulant preconditioner of one box (Sec. 4, the
// paragraph after the C_B^-1 display; the disk box of Sec. 5.3.1).
//
// The 1-level blocks D_f of a box are Toeplitz-block along y once M~ is also
// y-invariant (homogenised over each z-plane).  The second level replaces each
// y-Toeplitz block by its Chan circulant and diagonalises it with the y-DFT,
// which leaves one dense block of m2 = 3 nz_b rows (ordered [alpha][z]) per
// frequency pair (f, g):
//   D_{f,g}[(a,z),(b,z')] = delta - M~_z (delta + lambda_{f,g}^{ab}(z - z')).
// Applying the Chan step along x and then along y to the generator entries
// gives the coefficient array of every (pair, dz) plane directly,
//   c(kx, ky) = sum_{u,v in {0,1}} wx_u(kx) wy_v(ky) G(kx - u n, ky - v ny, dz),
//   wx_0 = (n - kx)/n, wx_1 = kx/n (kx > 0), and likewise along y,
// and lambda_{f,g} is its 2-D DFT.  The generators' parities in x and y give
//   D_{n-f,g} = Sx D_{f,g} Sx,  D_{f,ny-g} = Sy D_{f,g} Sy,
// (S = -1 on the x- resp. y-component rows), so only f <= n/2, g <= ny/2 are
// factored; a quarter of the blocks.
//
// Storage: each stored block is assembled as its transpose in the column-major
// layout of the batched LU, so the row-major inverse that the LU produces is
// D_{f,g}^{-1} in column-major order: one warp applies a block with a lane per
// row and every column a coalesced load.
#include <math.h>

#include <algorithm>

#include "greens.cuh"
#include "internal.h"
#include "prof.h"

namespace vie {

namespace {

__device__ __forceinline__ int pair_code2(int a, int b) {
  if (a > b) { int t = a; a = b; b = t; }
  return a == 0 ? b : (a == 1 ? 2 + b : 5);   // xx0 xy1 xz2 yy3 yz4 zz5
}

// 2-level Chan coefficients, planes (c, dz + nz - 1), each [ky][kx]
__global__ void k_chan2_coeffs(double2* __restrict__ out, int n, int ny, int nz, double h, double kb, double2 self) {
  const int ndz = 2 * nz - 1;
  const long long plane = (long long)n * ny;
  const long long total = 6LL * ndz * plane;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(idx % n);
    const long long r = idx / n;
    const int ky = (int)(r % ny);
    const long long line = r / ny;
    const int dz = (int)(line % ndz) - (nz - 1);
    const int c = (int)(line / ndz);
    double ar = 0, ai = 0;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 1 && kx == 0) continue;
      const double wx = u == 0 ? (double)(n - kx) / n : (double)kx / n;
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        if (v == 1 && ky == 0) continue;
        const double wy = v == 0 ? (double)(ny - ky) / ny : (double)ky / ny;
        const double2 t = gen_entry(c, kx - u * n, ky - v * ny, dz, h, kb, self);
        ar += wx * wy * t.x;
        ai += wx * wy * t.y;
      }
    }
    out[idx] = make_double2(ar, ai);
  }
}

// Stored blocks s = gs * nfs + fs (f = fs <= n/2, g = gs <= ny/2), each written
// as D^T column-major: element (p, q) of D_{f,g} at s m2^2 + p m2 + q.
__global__ void k_block_assemble2(double2* __restrict__ D, const double2* __restrict__ lam2,
                                  const double2* __restrict__ Mt, int n, int ny, int nz, int nfs, int nblk) {
  const int m2 = 3 * nz, ndz = 2 * nz - 1;
  const long long plane = (long long)n * ny;
  const long long total = (long long)nblk * m2 * m2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(idx % m2);
    const long long r = idx / m2;
    const int p = (int)(r % m2);
    const int s = (int)(r / m2);
    const int f = s % nfs, g = s / nfs;
    const int ap = p / nz, zp = p % nz, aq = q / nz, zq = q % nz;
    const int line = pair_code2(ap, aq) * ndz + (zp - zq + nz - 1);
    const double2 l = lam2[line * plane + (long long)g * n + f];
    const double2 mp = Mt[zp * ny];
    const double dl = (p == q) ? 1.0 : 0.0;
    const double ar = dl + l.x, ai = l.y;
    D[idx] = make_double2(dl - (mp.x * ar - mp.y * ai), -(mp.x * ai + mp.y * ar));
  }
}

// One warp per stored block (8 per CTA, consecutive f of one g so that the
// strided spectrum reads of neighbouring warps share sectors).  The block
// serves up to four frequency pairs: (f, g), (n-f, g) with Sx, (f, ny-g) with
// Sy and (n-f, ny-g) with Sx Sy.  R, Z: [m2][ny][n] spectra; invT: column-major
// D^{-1} per block.  Lane i owns rows i, i + 32, ... (RPL rows).
constexpr int G2_WARPS = 8;
constexpr int G2_JB = 8;
template <class C, int RPL>
__global__ void __launch_bounds__(G2_WARPS * 32) k_block_gemv2(const C* __restrict__ invT, const C* __restrict__ R,
                                                              C* __restrict__ Z, int n, int ny, int nz, int nfs,
                                                              int nblk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m2 = 3 * nz;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  C* rv = reinterpret_cast<C*>(smem_raw) + (size_t)warp * 4 * m2;   // [4][m2]
  const int s = blockIdx.x * G2_WARPS + warp;
  if (s >= nblk) return;
  const int f = s % nfs, g = s / nfs;
  const int f2 = (n - f) % n, g2 = (ny - g) % ny;
  const bool hx = f2 != f, hy = g2 != g;
  const long long plane = (long long)n * ny;
  const long long o0 = (long long)g * n + f, o1 = (long long)g * n + f2;
  const long long o2 = (long long)g2 * n + f, o3 = (long long)g2 * n + f2;
  for (int j = lane; j < m2; j += 32) {
    const int a = j / nz;
    const C* src = R + (long long)j * plane;
    rv[j] = src[o0];
    if (hx) { C v = src[o1]; if (a == 0) { v.x = -v.x; v.y = -v.y; } rv[m2 + j] = v; }
    if (hy) { C v = src[o2]; if (a == 1) { v.x = -v.x; v.y = -v.y; } rv[2 * m2 + j] = v; }
    if (hx && hy) { C v = src[o3]; if (a <= 1) { v.x = -v.x; v.y = -v.y; } rv[3 * m2 + j] = v; }
  }
  __syncwarp();
  C acc[RPL][4];
#pragma unroll
  for (int u = 0; u < RPL; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = czero<C>();
  const C* D = invT + (long long)s * m2 * m2;
  // G2_JB columns per batch: all their loads are issued before the first
  // product, so a warp keeps G2_JB * RPL loads in flight instead of one
  for (int j0 = 0; j0 < m2; j0 += G2_JB) {
    C dv[G2_JB][RPL];
#pragma unroll
    for (int jj = 0; jj < G2_JB; ++jj) {
      const int j = j0 + jj;
#pragma unroll
      for (int u = 0; u < RPL; ++u) {
        const int i = lane + 32 * u;
        dv[jj][u] = (j < m2 && i < m2) ? D[(long long)j * m2 + i] : czero<C>();
      }
    }
#pragma unroll
    for (int jj = 0; jj < G2_JB; ++jj) {
      const int j = j0 + jj;
      if (j >= m2) break;
      const C r0 = rv[j];
      const C r1 = hx ? rv[m2 + j] : czero<C>();
      const C r2 = hy ? rv[2 * m2 + j] : czero<C>();
      const C r3 = (hx && hy) ? rv[3 * m2 + j] : czero<C>();
#pragma unroll
      for (int u = 0; u < RPL; ++u) {
        cfma(acc[u][0], dv[jj][u], r0);
        cfma(acc[u][1], dv[jj][u], r1);
        cfma(acc[u][2], dv[jj][u], r2);
        cfma(acc[u][3], dv[jj][u], r3);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    const int i = lane + 32 * u;
    if (i >= m2) continue;
    const int a = i / nz;
    C* dst = Z + (long long)i * plane;
    dst[o0] = acc[u][0];
    if (hx) { C v = acc[u][1]; if (a == 0) { v.x = -v.x; v.y = -v.y; } dst[o1] = v; }
    if (hy) { C v = acc[u][2]; if (a == 1) { v.x = -v.x; v.y = -v.y; } dst[o2] = v; }
    if (hx && hy) { C v = acc[u][3]; if (a <= 1) { v.x = -v.x; v.y = -v.y; } dst[o3] = v; }
  }
}

}  // namespace

vie_status build_box2(vie_plan_s* P, BoxPrec& B, bool want64, bool want128) {
  cudaStream_t st = P->st;
  const int n = B.b.nx, ny = B.b.ny, nz = B.b.nz;
  const int m2 = 3 * nz;
  B.levels = 2;
  B.n = n;
  B.m = 3 * ny * nz;
  B.m2 = m2;
  B.nfs = n / 2 + 1;
  B.ngs = ny / 2 + 1;
  B.nblk = B.nfs * B.ngs;
  B.nhalf = B.nblk;
  B.nkept = n;        // every x-frequency keeps its own blocks
  B.ndisc = 0;
  VIE_TRY(fft_get(n, &B.fx));
  VIE_TRY(fft_get(ny, &B.fy));
  // 1. plane-homogenised M~
  VIE_TRY(box_homogenise(P, B.b, B.Mt, true));
  // 2. 2-level Chan coefficients, then the 2-D DFT of every (pair, dz) plane
  const int ndz = 2 * nz - 1;
  const int nl2 = 6 * ndz;
  const size_t nel = (size_t)nl2 * ny * n;
  DevBuf coef, lam2;
  VIE_TRY(coef.alloc(sizeof(double2) * nel));
  VIE_TRY(lam2.alloc(sizeof(double2) * nel));
  {
    const double2 self = self_term_value(P->h, P->kb);
    const int grid = (int)std::min<long long>(((long long)nel + 255) / 256, 152LL * 16);
    Prof pf_("chan2_coeffs", st);
    k_chan2_coeffs<<<grid, 256, 0, st>>>(coef.as<double2>(), n, ny, nz, P->h, P->kb, self);
    count_launch();
    VIE_CHECK_LAUNCH();
  }
  {
    DevBuf tmp;
    const size_t ts = std::max(fft_scratch_elems<double2>(*B.fx, nl2 * ny), fft_scratch_elems<double2>(*B.fy, nl2 * n));
    if (ts) VIE_TRY(tmp.alloc(sizeof(double2) * ts));
    // x: contiguous lines of n points
    LineDesc dx = lines_flat(n, n, nl2 * ny, n, 1, n, 1);
    VIE_TRY(fft_lines<double2>(coef.as<double2>(), lam2.as<double2>(), dx, *B.fx, -1, 1.0, tmp.as<double2>(), st));
    // y: lines of ny points at stride n, line (kx, plane)
    LineDesc dy{ny, ny, nl2 * n, n, nl2, 1, (long long)ny * n, 0, n, 1, (long long)ny * n, 0, n};
    VIE_TRY(fft_lines<double2>(lam2.as<double2>(), coef.as<double2>(), dy, *B.fy, -1, 1.0, tmp.as<double2>(), st));
    VIE_CUDA(cudaStreamSynchronize(st));
  }
  lam2.release();   // the eigenvalues are now in coef
  // 3. assemble the stored blocks (transposed), LU, inverse
  DevBuf LU;
  const size_t mm = (size_t)m2 * m2;
  VIE_TRY(LU.alloc(sizeof(double2) * mm * B.nblk));
  {
    const long long total = (long long)mm * B.nblk;
    const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 32);
    Prof pf_("block_assemble2", st);
    k_block_assemble2<<<grid, 256, 0, st>>>(LU.as<double2>(), coef.as<double2>(), B.Mt.as<double2>(), n, ny, nz, B.nfs,
                                            B.nblk);
    count_launch();
    VIE_CHECK_LAUNCH();
  }
  coef.release();
  VIE_TRY(factor_invert_blocks(P, LU, m2, B.nblk, want64, &B.inv64, want128, &B.inv128));
  // spectra and transform scratch of the apply: x-lines (m lines) and y-lines (m2 n lines)
  const size_t vec = (size_t)n * B.m;
  if (want64) {
    VIE_TRY(B.rhat64.alloc(sizeof(float2) * vec));
    VIE_TRY(B.zhat64.alloc(sizeof(float2) * vec));
    const size_t ts = std::max(fft_scratch_elems<float2>(*B.fx, B.m), fft_scratch_elems<float2>(*B.fy, m2 * n));
    if (ts) VIE_TRY(B.tmp64.alloc(sizeof(float2) * ts));
  }
  if (want128) {
    VIE_TRY(B.rhat128.alloc(sizeof(double2) * vec));
    VIE_TRY(B.zhat128.alloc(sizeof(double2) * vec));
    const size_t ts = std::max(fft_scratch_elems<double2>(*B.fx, B.m), fft_scratch_elems<double2>(*B.fy, m2 * n));
    if (ts) VIE_TRY(B.tmp128.alloc(sizeof(double2) * ts));
  }
  return VIE_OK;
}

// z_box = C_B2^{-1} r_box: gather + x-FFT, y-FFT, per-(f, g) block products,
// inverse y-FFT, inverse x-FFT + scatter.  rh, zh: [m2][ny][n] spectra.
template <class C>
vie_status apply_box2(vie_plan_s* P, BoxPrec& B, const C* r, C* z, C* inv, C* rh, C* zh, C* tmp, cudaStream_t st) {
  const long long N = (long long)P->nx * P->ny * P->nz;
  const int n = B.n, m = B.m, nyb = B.b.ny, nzb = B.b.nz, m2 = B.m2;
  const long long base = ((long long)B.b.z0 * P->ny + B.b.y0) * P->nx + B.b.x0;
  LineDesc ld{n, n, m, nyb, nzb,
              (long long)P->nx, (long long)P->ny * P->nx, N, 1,
              (long long)n, (long long)nyb * n, (long long)nyb * nzb * n, 1};
  VIE_TRY(fft_lines<C>(r + base, rh, ld, *B.fx, -1, 1.0, tmp, st));
  LineDesc dy{nyb, nyb, m2 * n, n, m2, 1, (long long)nyb * n, 0, n, 1, (long long)nyb * n, 0, n};
  VIE_TRY(fft_lines<C>(rh, zh, dy, *B.fy, -1, 1.0, tmp, st));
  {
    const size_t smem = sizeof(C) * 4 * m2 * G2_WARPS;
    const int grid = ceil_div(B.nblk, G2_WARPS);
    Prof pf_(sizeof(C) == 8 ? "block_gemv2_c64" : "block_gemv2_c128", st);
    if (m2 <= 32) k_block_gemv2<C, 1><<<grid, G2_WARPS * 32, smem, st>>>(inv, zh, rh, n, nyb, nzb, B.nfs, B.nblk);
    else if (m2 <= 64) k_block_gemv2<C, 2><<<grid, G2_WARPS * 32, smem, st>>>(inv, zh, rh, n, nyb, nzb, B.nfs, B.nblk);
    else k_block_gemv2<C, 3><<<grid, G2_WARPS * 32, smem, st>>>(inv, zh, rh, n, nyb, nzb, B.nfs, B.nblk);
    count_launch();
    VIE_CHECK_LAUNCH();
  }
  VIE_TRY(fft_lines<C>(rh, zh, dy, *B.fy, +1, 1.0 / nyb, tmp, st));
  LineDesc lo{n, n, m, nyb, nzb,
              (long long)n, (long long)nyb * n, (long long)nyb * nzb * n, 1,
              (long long)P->nx, (long long)P->ny * P->nx, N, 1};
  return fft_lines<C>(zh, z + base, lo, *B.fx, +1, 1.0 / n, tmp, st);
}

template vie_status apply_box2<float2>(vie_plan_s*, BoxPrec&, const float2*, float2*, float2*, float2*, float2*,
                                       float2*, cudaStream_t);
template vie_status apply_box2<double2>(vie_plan_s*, BoxPrec&, const double2*, double2*, double2*, double2*, double2*,
                                        double2*, cudaStream_t);

}  // namespace vie
