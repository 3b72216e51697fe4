// y = A x = x - M (x + G x) through the circulant embedding of the 3-level
// Toeplitz blocks of G (Sec. 1: O(n log n) FFT product; Sec. 2 Eq. sys_mat).
//
// Three passes per matvec, every transform in shared memory:
//   A  (yz forward)  per component b and group of XG consecutive x: zero-pad
//      the ny x nz slabs to Py x Pz, 2-D FFT, write T[b][kz][ky][x].
//   B  (x pass)      per (ky, kz): the three x-lines of length nx, zero-padded
//      to L, forward FFT, 3x3 symmetric tensor product with the generator
//      spectra, inverse FFT, keep x < nx, write back to T.
//   C  (yz inverse)  per component a and x group: inverse 2-D FFT, crop to
//      ny x nz, epilogue y = x - M (x + Gx).
// The generator spectra hold only the non-negative octant; the other octants
// follow from the parity of each component (sign flips).  The inverse
// normalisation 1/(L Py Pz) is folded into the stored spectra.
#pragma once

#include <algorithm>

#include <cooperative_groups.h>

#include "internal.h"
#include "prof.h"

namespace vie {

// parity sign of pair c under reversal of axis (0 x, 1 y, 2 z)
__device__ __forceinline__ float pair_parity(int c, int axis) {
  const int A[6] = {0, 0, 0, 1, 1, 2};
  const int B[6] = {0, 1, 2, 1, 2, 2};
  return ((A[c] == axis) != (B[c] == axis)) ? -1.f : 1.f;
}

template <class C>
__global__ void __launch_bounds__(256) k_mv_yz_fwd(const C* __restrict__ x, C* __restrict__ T, MvDims d,
                                                   FftPlanDev py, FftPlanDev pz, int XG) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int b = blockIdx.y;
  const int x0 = blockIdx.x * XG;
  const int xg = min(XG, d.nx - x0);
  const int SP = d.Py * d.Pz + 1;
  C* a = s;
  C* bb = s + (size_t)XG * SP;
  for (int e = threadIdx.x; e < 2 * XG * SP; e += blockDim.x) s[e] = czero<C>();
  __syncthreads();
  const long long plane = (long long)d.ny * d.nx;
  const C* xb = x + (long long)b * d.nz * plane;
  const int nin = xg * d.ny * d.nz;
  batched_copy<8>(
      nin,
      [&](int e) {
        const int xl = e % xg, r = e / xg;
        const int y = r % d.ny, z = r / d.ny;
        return xb[(long long)z * plane + (long long)y * d.nx + x0 + xl];
      },
      [&](int e, C v) {
        const int xl = e % xg, r = e / xg;
        const int y = r % d.ny, z = r / d.ny;
        a[xl * SP + z * d.Py + y] = v;
      });
  __syncthreads();
  // y lines (only the nz non-zero rows), then z lines (all Py columns); rows
  // z >= nz stay zero in both buffers
  C* r1 = fft_smem_pp(a, bb, py, SmemLines{xg * d.nz, d.nz, d.Py, SP, 1, 0}, -1);
  C* r2 = fft_smem_pp(r1, r1 == a ? bb : a, pz, SmemLines{xg * d.Py, d.Py, 1, SP, d.Py, 1}, -1);
  const int nout = xg * d.Py * d.Pz;
  C* Tb = T + (long long)b * d.Pz * d.Py * d.nx;
  for (int e = threadIdx.x; e < nout; e += blockDim.x) {
    const int xl = e % xg;
    const int r = e / xg;
    const int ky = r % d.Py, kz = r / d.Py;
    Tb[((long long)kz * d.Py + ky) * d.nx + x0 + xl] = r2[xl * SP + kz * d.Py + ky];
  }
}

// fetch G^{c}(kx, ky, kz) from the stored octant
template <class C>
__device__ __forceinline__ C spec_at(const C* __restrict__ spec, int c, int kx, int kyo, int kzo, float syz_c,
                                     const MvDims& d, long long Q) {
  const bool fx = kx > d.L / 2;
  const int kxo = fx ? d.L - kx : kx;
  C v = spec[(long long)c * Q + ((long long)kzo * d.Pyh + kyo) * d.Lh + kxo];
  float sg = syz_c;
  if (fx) sg *= pair_parity(c, 0);
  if (sg < 0) { v.x = -v.x; v.y = -v.y; }
  return v;
}

// the 3x3 tensor product on n spectrum points held at k = 0..n-1 of the
// lines, which are the x-frequencies kx = k0 + kstep k
template <class C>
__device__ __forceinline__ void tensor_mul(C* s0, C* s1, C* s2, int L, int ky, int kz, const C* __restrict__ spec,
                                           const MvDims& d, int kstep = 1, int k0 = 0) {
  const bool fy = ky > d.Py / 2, fz = kz > d.Pz / 2;
  const int kyo = fy ? d.Py - ky : ky;
  const int kzo = fz ? d.Pz - kz : kz;
  const long long Q = (long long)d.Lh * d.Pyh * d.Pzh;
  float syz[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    float sg = 1.f;
    if (fy) sg *= pair_parity(c, 1);
    if (fz) sg *= pair_parity(c, 2);
    syz[c] = sg;
  }
  for (int k = threadIdx.x; k < L; k += blockDim.x) {
    const int kx = k0 + kstep * k;
    const C X0 = s0[k], X1 = s1[k], X2 = s2[k];
    const C gxx = spec_at(spec, 0, kx, kyo, kzo, syz[0], d, Q);
    const C gxy = spec_at(spec, 1, kx, kyo, kzo, syz[1], d, Q);
    const C gxz = spec_at(spec, 2, kx, kyo, kzo, syz[2], d, Q);
    const C gyy = spec_at(spec, 3, kx, kyo, kzo, syz[3], d, Q);
    const C gyz = spec_at(spec, 4, kx, kyo, kzo, syz[4], d, Q);
    const C gzz = spec_at(spec, 5, kx, kyo, kzo, syz[5], d, Q);
    C y0 = cmul(gxx, X0), y1 = cmul(gxy, X0), y2 = cmul(gxz, X0);
    cfma(y0, gxy, X1); cfma(y1, gyy, X1); cfma(y2, gyz, X1);
    cfma(y0, gxz, X2); cfma(y1, gyz, X2); cfma(y2, gzz, X2);
    s0[k] = y0; s1[k] = y1; s2[k] = y2;
  }
}

// fused x pass: shared memory holds the three x-lines of one (ky, kz).
// MAXE == 0: ping-pong passes over two copies; MAXE > 0: in place (for the
// longest embeddings).
template <class C, int MAXE>
__global__ void __launch_bounds__(MAXE == 0 ? 512 : 1024) k_mv_x(C* __restrict__ T, const C* __restrict__ spec,
                                                                 MvDims d, FftPlanDev pl, int joint) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int kyz = blockIdx.x;
  const int ky = kyz % d.Py, kz = kyz / d.Py;
  const int L = d.L;
  const long long lstride = (long long)d.Pz * d.Py * d.nx;
  const long long loff = ((long long)kz * d.Py + ky) * d.nx;
  batched_copy<8>(
      3 * L,
      [&](int e) {
        const int b = e / L, i = e - b * L;
        return i < d.nx ? T[b * lstride + loff + i] : czero<C>();
      },
      [&](int e, C v) { s[e] = v; });
  __syncthreads();
  C* res = s;
  if constexpr (MAXE == 0) {
    const SmemLines Ls{3, 3, L, 0, 1, 0};
    C* r1 = fft_smem_pp(s, s + 3 * L, pl, Ls, -1);
    tensor_mul(r1, r1 + L, r1 + 2 * L, L, ky, kz, spec, d);
    __syncthreads();
    res = fft_smem_pp(r1, r1 == s ? s + 3 * L : s, pl, Ls, +1);
  } else {
    // one call site of the in-place transform keeps register use compact
    const SmemLines Ls = joint ? SmemLines{3, 3, L, 0, 1, 0} : SmemLines{1, 1, 0, 0, 1, 0};
    for (int step = 0; step < 2 * (joint ? 1 : 3); ++step) {
      const int dir = joint ? step : step / 3;
      const int b = joint ? 0 : step % 3;
      fft_smem<MAXE>(s + b * L, pl, Ls, dir == 0 ? -1 : +1);
      if (step == (joint ? 0 : 2)) {
        tensor_mul(s, s + L, s + 2 * L, L, ky, kz, spec, d);
        __syncthreads();
      }
    }
  }
  for (int e = threadIdx.x; e < 3 * d.nx; e += blockDim.x) {
    const int a = e / d.nx, i = e - a * d.nx;
    T[a * lstride + loff + i] = res[a * L + i];
  }
}

// ---------------------------------------------------------------------------
// Fused x pass split over a cluster of Q CTAs (complex FP32), for embeddings
// whose three lines do not fit one CTA's shared memory.  With Lq = L / Q,
// CTA r of the cluster of one (ky, kz) forms, by decimation in frequency,
//   a_r[n] = sum_j x[n + j Lq] W_L^{(n + j Lq) r}   (n < Lq; x = 0 from nx on),
// whose Lq-point transform is X[Q k + r]; it multiplies those frequencies by
// the generator spectra and transforms them back to z_r.  The outputs are
//   y[n] = sum_r W_L^{-n r} z_r[n mod Lq]   (n < nx),
// each CTA assembling a contiguous share of them from the Q CTAs' shared
// memory (distributed shared memory of the cluster).
// ---------------------------------------------------------------------------
template <int Q>
__global__ void __cluster_dims__(Q, 1, 1) __launch_bounds__(512)
    k_mv_xq(float2* __restrict__ T, const float2* __restrict__ spec, MvDims d, FftPlanDev pl,
            const float2* __restrict__ twL) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* s = reinterpret_cast<float2*>(smem_raw);
  const int r = (int)cl.block_rank();
  const int kyz = blockIdx.x / Q;
  const int ky = kyz % d.Py, kz = kyz / d.Py;
  const int L = d.L, Lq = L / Q;
  const long long lstride = (long long)d.Pz * d.Py * d.nx;
  const long long loff = ((long long)kz * d.Py + ky) * d.nx;
  for (int e = threadIdx.x; e < 3 * Lq; e += blockDim.x) {
    const int b = e / Lq, n = e - b * Lq;
    float2 a = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      const int i = n + j * Lq;
      if (i < d.nx) {
        const float2 v = T[b * lstride + loff + i];
        a = cadd(a, r == 0 ? v : cmul(v, twL[(i * r) % L]));
      }
    }
    s[e] = a;
  }
  __syncthreads();
  const SmemLines Ls{3, 3, Lq, 0, 1, 0};
  float2* r1 = fft_smem_pp(s, s + 3 * Lq, pl, Ls, -1);
  tensor_mul(r1, r1 + Lq, r1 + 2 * Lq, Lq, ky, kz, spec, d, Q, r);
  __syncthreads();
  float2* res = fft_smem_pp(r1, r1 == s ? s + 3 * Lq : s, pl, Ls, +1);
  // every CTA's z_r is complete (and visible to the cluster) past this point;
  // all of them read their inputs from T before it
  cl.sync();
  const float2* z[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) z[q] = cl.map_shared_rank(res, q);
  const int chunk = (d.nx + Q - 1) / Q;
  const int n0 = r * chunk, cnt = max(0, min(d.nx, n0 + chunk) - n0);
  for (int e = threadIdx.x; e < 3 * cnt; e += blockDim.x) {
    const int b = e / cnt, n = n0 + (e - b * cnt);
    const int nm = n % Lq;
    float2 y = z[0][b * Lq + nm];
#pragma unroll
    for (int q = 1; q < Q; ++q) {
      const float2 w = twL[(n * q) % L];
      y = cadd(y, cmul(z[q][b * Lq + nm], make_float2(w.x, -w.y)));
    }
    T[b * lstride + loff + n] = y;
  }
  // no CTA leaves (releasing its shared memory) while another still reads it
  cl.sync();
}

// ---------------------------------------------------------------------------
// Fused x pass for power-of-two embeddings L = R1 R2 R3 in complex FP32, all
// structure at compile time.  The forward transform is decimation in
// frequency: pass 1 (radix R1, stride L/R1, twiddles W_L^{b q}), pass 2 inside
// each of the R1 blocks (radix R2, twiddles W_{L/R1}^{b q}), pass 3 on R3
// contiguous points, which leaves X[q1 + R1 q2 + R1 R2 q3] at position
// q1 L/R1 + q2 R3 + q3.  The tensor product works on that digit-reversed order
// in registers, and the inverse is the mirror image (conjugate butterflies,
// conjugate twiddles applied before them, passes in reverse order), which
// returns natural order: no permutation anywhere.  A thread keeps the same
// positions of all three components, so the product needs no exchange; the
// first pass reads the zero-padded line straight from global memory and the
// last pass writes only the nx points kept.  Shared memory holds one copy
// of the three lines with one pad slot per 16 points, which makes every
// pass's accesses conflict-free.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int xpad(int i) { return i + (i >> 4); }

// W_16^j (DIR = -1) or its conjugate (DIR = +1), j compile-time after unrolling
template <int DIR>
__device__ __forceinline__ float2 w16(int j) {
  constexpr float c = 0.923879532511286756f, s = 0.382683432365089772f, h = 0.707106781186547524f;
  float2 w;
  switch (j & 15) {
    case 0: w = make_float2(1.f, 0.f); break;
    case 1: w = make_float2(c, -s); break;
    case 2: w = make_float2(h, -h); break;
    case 3: w = make_float2(s, -c); break;
    case 4: w = make_float2(0.f, -1.f); break;
    case 5: w = make_float2(-s, -c); break;
    case 6: w = make_float2(-h, -h); break;
    case 7: w = make_float2(-c, -s); break;
    case 8: w = make_float2(-1.f, 0.f); break;
    case 9: w = make_float2(-c, s); break;
    case 10: w = make_float2(-h, h); break;
    case 11: w = make_float2(-s, c); break;
    case 12: w = make_float2(0.f, 1.f); break;
    case 13: w = make_float2(s, c); break;
    case 14: w = make_float2(h, h); break;
    default: w = make_float2(c, s); break;
  }
  if (DIR > 0) w.y = -w.y;
  return w;
}

template <int N>
__host__ __device__ constexpr int bitrev_n(int i) {
  int r = 0;
  for (int b = 1; b < N; b <<= 1) { r = (r << 1) | (i & 1); i >>= 1; }
  return r;
}

// natural-order N-point transform (N = 2, 4, 8, 16) with the sign of DIR
template <int N, int DIR>
__device__ __forceinline__ void dft_pow2(float2 (&v)[N]) {
  float2 a[N];
#pragma unroll
  for (int i = 0; i < N; ++i) a[bitrev_n<N>(i)] = v[i];
#pragma unroll
  for (int m = 1; m < N; m <<= 1) {
#pragma unroll
    for (int k = 0; k < N; k += 2 * m) {
#pragma unroll
      for (int j = 0; j < m; ++j) {
        const float2 x = a[k + j];
        float2 b = a[k + j + m];
        if (j != 0) b = cmul(b, w16<DIR>(j * (8 / m)));   // W_{2m}^j = W_16^{8 j / m}
        a[k + j] = make_float2(x.x + b.x, x.y + b.y);
        a[k + j + m] = make_float2(x.x - b.x, x.y - b.y);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = a[i];
}

template <int R1, int R2, int R3>
__global__ void __launch_bounds__(R2 * R3, 512 / (R2 * R3)) k_mv_x16(float2* __restrict__ T, const float2* __restrict__ spec,
                                                    MvDims d, const float2* __restrict__ twL) {
  constexpr int L = R1 * R2 * R3, S1 = L / R1, S2 = S1 / R2, GPT = R1 / R3;
  constexpr int LP = L + L / 16;
  static_assert(R1 == R2 && R1 % R3 == 0 && S2 == R3, "pass structure");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);   // [3][LP]
  const int t = threadIdx.x;
  const int kyz = blockIdx.x;
  const int ky = kyz % d.Py, kz = kyz / d.Py;
  const long long lstride = (long long)d.Pz * d.Py * d.nx;
  const long long loff = ((long long)kz * d.Py + ky) * d.nx;
  // the passes other than the product take the components one at a time
  // (the twiddles of a pass stay in registers for all three)
  float2 w[R1];
  float2 v[R1];
  // forward pass 1: group b = t from global memory (zero beyond nx)
#pragma unroll
  for (int q = 1; q < R1; ++q) w[q] = twL[t * q];   // W_L^{b q}
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int i = t + S1 * r;
      v[r] = i < d.nx ? T[a * lstride + loff + i] : make_float2(0.f, 0.f);
    }
    dft_pow2<R1, -1>(v);
#pragma unroll
    for (int q = 1; q < R1; ++q) v[q] = cmul(v[q], w[q]);
#pragma unroll
    for (int q = 0; q < R1; ++q) sm[a * LP + xpad(t + S1 * q)] = v[q];
  }
  __syncthreads();
  // forward pass 2: block q1, offset b2
  const int b2 = t % S2, base2 = (t / S2) * S1;
#pragma unroll
  for (int q = 1; q < R2; ++q) w[q] = twL[b2 * q * R1];   // W_{L/R1}^{b q}
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int r = 0; r < R2; ++r) v[r] = sm[a * LP + xpad(base2 + b2 + S2 * r)];
    dft_pow2<R2, -1>(v);
#pragma unroll
    for (int q = 1; q < R2; ++q) v[q] = cmul(v[q], w[q]);
#pragma unroll
    for (int q = 0; q < R2; ++q) sm[a * LP + xpad(base2 + b2 + S2 * q)] = v[q];
  }
  __syncthreads();
  // pass 3, the tensor product and the inverse pass 3, on GPT groups of R3 contiguous points
  const bool fy = ky > d.Py / 2, fz = kz > d.Pz / 2;
  const int kyo = fy ? d.Py - ky : ky;
  const int kzo = fz ? d.Pz - kz : kz;
  const long long Q = (long long)d.Lh * d.Pyh * d.Pzh;
  float syz[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    float sg = 1.f;
    if (fy) sg *= pair_parity(c, 1);
    if (fz) sg *= pair_parity(c, 2);
    syz[c] = sg;
  }
#pragma unroll
  for (int g = 0; g < GPT; ++g) {
    const int sb = GPT * t + g;
    const int base3 = sb * R3;
    float2 u[3][R3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int r = 0; r < R3; ++r) u[a][r] = sm[a * LP + xpad(base3 + r)];
#pragma unroll
    for (int a = 0; a < 3; ++a) dft_pow2<R3, -1>(u[a]);
    const int q1 = sb / R2, q2 = sb - (sb / R2) * R2;
#pragma unroll
    for (int q3 = 0; q3 < R3; ++q3) {
      const int kx = q1 + R1 * q2 + R1 * R2 * q3;
      const float2 X0 = u[0][q3], X1 = u[1][q3], X2 = u[2][q3];
      const float2 gxx = spec_at(spec, 0, kx, kyo, kzo, syz[0], d, Q);
      const float2 gxy = spec_at(spec, 1, kx, kyo, kzo, syz[1], d, Q);
      const float2 gxz = spec_at(spec, 2, kx, kyo, kzo, syz[2], d, Q);
      const float2 gyy = spec_at(spec, 3, kx, kyo, kzo, syz[3], d, Q);
      const float2 gyz = spec_at(spec, 4, kx, kyo, kzo, syz[4], d, Q);
      const float2 gzz = spec_at(spec, 5, kx, kyo, kzo, syz[5], d, Q);
      float2 y0 = cmul(gxx, X0), y1 = cmul(gxy, X0), y2 = cmul(gxz, X0);
      cfma(y0, gxy, X1); cfma(y1, gyy, X1); cfma(y2, gyz, X1);
      cfma(y0, gxz, X2); cfma(y1, gyz, X2); cfma(y2, gzz, X2);
      u[0][q3] = y0; u[1][q3] = y1; u[2][q3] = y2;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) dft_pow2<R3, +1>(u[a]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int r = 0; r < R3; ++r) sm[a * LP + xpad(base3 + r)] = u[a][r];
  }
  __syncthreads();
  // inverse pass 2: conjugate twiddles, then conjugate butterflies
#pragma unroll
  for (int q = 1; q < R2; ++q) w[q].y = -w[q].y;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int q = 0; q < R2; ++q) v[q] = sm[a * LP + xpad(base2 + b2 + S2 * q)];
#pragma unroll
    for (int q = 1; q < R2; ++q) v[q] = cmul(v[q], w[q]);
    dft_pow2<R2, +1>(v);
#pragma unroll
    for (int r = 0; r < R2; ++r) sm[a * LP + xpad(base2 + b2 + S2 * r)] = v[r];
  }
  __syncthreads();
  // inverse pass 1, straight to global memory (the nx points kept)
#pragma unroll
  for (int q = 1; q < R1; ++q) {
    w[q] = twL[t * q];
    w[q].y = -w[q].y;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int q = 0; q < R1; ++q) v[q] = sm[a * LP + xpad(t + S1 * q)];
#pragma unroll
    for (int q = 1; q < R1; ++q) v[q] = cmul(v[q], w[q]);
    dft_pow2<R1, +1>(v);
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int i = t + S1 * r;
      if (i < d.nx) T[a * lstride + loff + i] = v[r];
    }
  }
}

// ---------------------------------------------------------------------------
// The same scheme with four passes, L = R1 R2 R3 R4 (R1 = R2, R3 and R4
// dividing R1), for the longer power-of-two embeddings: pass 1 radix R1 at
// stride L/R1 (twiddles W_L^{b q}), pass 2 radix R2 inside each block of L/R1
// (W_{L/R1}^{b q}), pass 3 radix R3 inside each block of L/(R1 R2)
// (W_{L/(R1 R2)}^{b q}), pass 4 on R4 contiguous points, which leaves
// X[q1 + R1 q2 + R1 R2 q3 + R1 R2 R3 q4] at position q1 L/R1 + q2 L/(R1 R2) +
// q3 R4 + q4; the tensor product works on that order and the inverse mirrors
// the forward passes.  A thread takes one pass-1 and one pass-2 butterfly,
// R1/R3 pass-3 butterflies and R1/R4 pass-4 groups, one component at a time
// except in the product, so its registers stay few with L/R1 threads.
// ---------------------------------------------------------------------------
template <int R1, int R2, int R3, int R4>
__global__ void __launch_bounds__(R1 * R2 * R3 * R4 / R1) k_mv_x4p(float2* __restrict__ T,
                                                                 const float2* __restrict__ spec, MvDims d,
                                                                 const float2* __restrict__ twL) {
  constexpr int L = R1 * R2 * R3 * R4, NT = L / R1;
  constexpr int S1 = L / R1, S2 = S1 / R2, S3 = S2 / R3;
  constexpr int G3 = R1 / R3, G4 = R1 / R4;
  constexpr int LP = L + L / 16;
  static_assert(R1 == R2 && R1 % R3 == 0 && R1 % R4 == 0 && S3 == R4, "pass structure");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);   // [3][LP]
  const int t = threadIdx.x;
  const int kyz = blockIdx.x;
  const int ky = kyz % d.Py, kz = kyz / d.Py;
  const long long lstride = (long long)d.Pz * d.Py * d.nx;
  const long long loff = ((long long)kz * d.Py + ky) * d.nx;
  float2 v[R1];
  // forward pass 1 from global memory (zero beyond nx); twiddles are read
  // again where a pass repeats, so that none stay live across the product
  {
  float2 w[R1];
#pragma unroll
  for (int q = 1; q < R1; ++q) w[q] = twL[t * q];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int i = t + S1 * r;
      v[r] = i < d.nx ? T[a * lstride + loff + i] : make_float2(0.f, 0.f);
    }
    dft_pow2<R1, -1>(v);
#pragma unroll
    for (int q = 1; q < R1; ++q) v[q] = cmul(v[q], w[q]);
#pragma unroll
    for (int q = 0; q < R1; ++q) sm[a * LP + xpad(t + S1 * q)] = v[q];
  }
  }
  __syncthreads();
  // forward pass 2: block q1 = t / S2, offset b2
  const int b2 = t % S2, base2 = (t / S2) * S1;
  {
  float2 w2[R2];
#pragma unroll
  for (int q = 1; q < R2; ++q) w2[q] = twL[b2 * q * R1];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int r = 0; r < R2; ++r) v[r] = sm[a * LP + xpad(base2 + b2 + S2 * r)];
    dft_pow2<R2, -1>(v);
#pragma unroll
    for (int q = 1; q < R2; ++q) v[q] = cmul(v[q], w2[q]);
#pragma unroll
    for (int q = 0; q < R2; ++q) sm[a * LP + xpad(base2 + b2 + S2 * q)] = v[q];
  }
  }
  __syncthreads();
  // forward pass 3: G3 butterflies per thread, block of S2 points, offset b3
#pragma unroll 1
  for (int g = 0; g < G3; ++g) {
    const int u3 = g * NT + t;                 // butterfly index < L / R3
    const int b3 = u3 % S3, base3 = (u3 / S3) * S2;
    float2 w3[R3];
#pragma unroll
    for (int q = 1; q < R3; ++q) w3[q] = twL[b3 * q * R1 * R2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2 x3[R3];
#pragma unroll
      for (int r = 0; r < R3; ++r) x3[r] = sm[a * LP + xpad(base3 + b3 + S3 * r)];
      dft_pow2<R3, -1>(x3);
#pragma unroll
      for (int q = 1; q < R3; ++q) x3[q] = cmul(x3[q], w3[q]);
#pragma unroll
      for (int q = 0; q < R3; ++q) sm[a * LP + xpad(base3 + b3 + S3 * q)] = x3[q];
    }
  }
  __syncthreads();
  // pass 4, the tensor product and the inverse pass 4 on G4 groups of R4 contiguous points
  const bool fy = ky > d.Py / 2, fz = kz > d.Pz / 2;
  const int kyo = fy ? d.Py - ky : ky;
  const int kzo = fz ? d.Pz - kz : kz;
  const long long Q = (long long)d.Lh * d.Pyh * d.Pzh;
  float syz[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    float sg = 1.f;
    if (fy) sg *= pair_parity(c, 1);
    if (fz) sg *= pair_parity(c, 2);
    syz[c] = sg;
  }
#pragma unroll 1
  for (int g = 0; g < G4; ++g) {
    const int sb = g * NT + t;                 // group index < L / R4
    const int base4 = sb * R4;
    float2 u[3][R4];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int r = 0; r < R4; ++r) u[a][r] = sm[a * LP + xpad(base4 + r)];
#pragma unroll
    for (int a = 0; a < 3; ++a) dft_pow2<R4, -1>(u[a]);
    // position base4 + q4 = q1 S1 + q2 S2 + q3 R4 + q4
    const int q1 = base4 / S1, q2 = (base4 % S1) / S2, q3 = (base4 % S2) / R4;
#pragma unroll
    for (int q4 = 0; q4 < R4; ++q4) {
      const int kx = q1 + R1 * q2 + R1 * R2 * q3 + R1 * R2 * R3 * q4;
      const float2 X0 = u[0][q4], X1 = u[1][q4], X2 = u[2][q4];
      const float2 gxx = spec_at(spec, 0, kx, kyo, kzo, syz[0], d, Q);
      const float2 gxy = spec_at(spec, 1, kx, kyo, kzo, syz[1], d, Q);
      const float2 gxz = spec_at(spec, 2, kx, kyo, kzo, syz[2], d, Q);
      const float2 gyy = spec_at(spec, 3, kx, kyo, kzo, syz[3], d, Q);
      const float2 gyz = spec_at(spec, 4, kx, kyo, kzo, syz[4], d, Q);
      const float2 gzz = spec_at(spec, 5, kx, kyo, kzo, syz[5], d, Q);
      float2 y0 = cmul(gxx, X0), y1 = cmul(gxy, X0), y2 = cmul(gxz, X0);
      cfma(y0, gxy, X1); cfma(y1, gyy, X1); cfma(y2, gyz, X1);
      cfma(y0, gxz, X2); cfma(y1, gyz, X2); cfma(y2, gzz, X2);
      u[0][q4] = y0; u[1][q4] = y1; u[2][q4] = y2;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) dft_pow2<R4, +1>(u[a]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int r = 0; r < R4; ++r) sm[a * LP + xpad(base4 + r)] = u[a][r];
  }
  __syncthreads();
  // inverse pass 3: conjugate twiddles, then conjugate butterflies
#pragma unroll 1
  for (int g = 0; g < G3; ++g) {
    const int u3 = g * NT + t;
    const int b3 = u3 % S3, base3 = (u3 / S3) * S2;
    float2 w3[R3];
#pragma unroll
    for (int q = 1; q < R3; ++q) {
      w3[q] = twL[b3 * q * R1 * R2];
      w3[q].y = -w3[q].y;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2 x3[R3];
#pragma unroll
      for (int q = 0; q < R3; ++q) x3[q] = sm[a * LP + xpad(base3 + b3 + S3 * q)];
#pragma unroll
      for (int q = 1; q < R3; ++q) x3[q] = cmul(x3[q], w3[q]);
      dft_pow2<R3, +1>(x3);
#pragma unroll
      for (int r = 0; r < R3; ++r) sm[a * LP + xpad(base3 + b3 + S3 * r)] = x3[r];
    }
  }
  __syncthreads();
  // inverse pass 2
  {
  float2 w2[R2];
#pragma unroll
  for (int q = 1; q < R2; ++q) {
    w2[q] = twL[b2 * q * R1];
    w2[q].y = -w2[q].y;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int q = 0; q < R2; ++q) v[q] = sm[a * LP + xpad(base2 + b2 + S2 * q)];
#pragma unroll
    for (int q = 1; q < R2; ++q) v[q] = cmul(v[q], w2[q]);
    dft_pow2<R2, +1>(v);
#pragma unroll
    for (int r = 0; r < R2; ++r) sm[a * LP + xpad(base2 + b2 + S2 * r)] = v[r];
  }
  }
  __syncthreads();
  // inverse pass 1, straight to global memory (the nx points kept)
  float2 w[R1];
#pragma unroll
  for (int q = 1; q < R1; ++q) {
    w[q] = twL[t * q];
    w[q].y = -w[q].y;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int q = 0; q < R1; ++q) v[q] = sm[a * LP + xpad(t + S1 * q)];
#pragma unroll
    for (int q = 1; q < R1; ++q) v[q] = cmul(v[q], w[q]);
    dft_pow2<R1, +1>(v);
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int i = t + S1 * r;
      if (i < d.nx) T[a * lstride + loff + i] = v[r];
    }
  }
}

// ---------------------------------------------------------------------------
// yz passes for power-of-two Py, Pz (<= 32) in complex FP32: one transform per
// thread in registers (radix-2 decimation in time), YZ_XG x-columns per CTA,
// one shared-memory exchange between the y and the z transforms.  Shared
// memory holds the y spectra of the nz non-zero z rows as [z][xl][ky] with a
// pitch of Py + 1, so both the row writes and the column reads are
// conflict-free; global accesses run along x (16 consecutive points).
// ---------------------------------------------------------------------------
// W_32^j (DIR = -1) or its conjugate (DIR = +1), j compile-time after unrolling
template <int DIR>
__device__ __forceinline__ float2 w32(int j) {
  // cos(pi k / 16), k = 0..8
  constexpr float Ct[9] = {1.f, 0.980785280403230449f, 0.923879532511286756f, 0.831469612302545237f,
                           0.707106781186547524f, 0.555570233019602225f, 0.382683432365089772f,
                           0.195090322016128268f, 0.f};
  int k = j & 31;
  float sg = 1.f;
  if (k >= 16) { k -= 16; sg = -1.f; }
  float c, s;   // cos, sin of pi k / 16
  if (k <= 8) { c = Ct[k]; s = Ct[8 - k]; }
  else { c = -Ct[16 - k]; s = Ct[k - 8]; }
  c *= sg;
  s *= sg;
  return make_float2(c, DIR < 0 ? -s : s);
}

// natural-order N-point transform (N = 2 .. 32) with the sign of DIR
template <int N, int DIR>
__device__ __forceinline__ void dft_p2(float2 (&v)[N]) {
  float2 a[N];
#pragma unroll
  for (int i = 0; i < N; ++i) a[bitrev_n<N>(i)] = v[i];
#pragma unroll
  for (int m = 1; m < N; m <<= 1) {
#pragma unroll
    for (int k = 0; k < N; k += 2 * m) {
#pragma unroll
      for (int j = 0; j < m; ++j) {
        const float2 x = a[k + j];
        float2 b = a[k + j + m];
        if (j != 0) b = cmul(b, w32<DIR>(j * (16 / m)));   // W_{2m}^j = W_32^{16 j / m}
        a[k + j] = make_float2(x.x + b.x, x.y + b.y);
        a[k + j + m] = make_float2(x.x - b.x, x.y - b.y);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = a[i];
}

// x-columns per CTA of the register yz passes: a template parameter, chosen
// per shape by the autotuner among 16, 8 and 4 (every choice transforms the
// same columns the same way)

template <int PY, int PZ, int YZ_XG>
__global__ void __launch_bounds__(128) k_mv_yz_fwd_r(const float2* __restrict__ x, float2* __restrict__ T, MvDims d) {
  constexpr int PITCH = PY + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* S = reinterpret_cast<float2*>(smem_raw);   // [nz][XG][PITCH]
  const int b = blockIdx.y, x0 = blockIdx.x * YZ_XG;
  const int xg = min(YZ_XG, d.nx - x0);
  const long long plane = (long long)d.ny * d.nx;
  const float2* xb = x + (long long)b * d.nz * plane;
  // y transforms of the rows z < nz (zero beyond ny)
  for (int ln = threadIdx.x; ln < d.nz * YZ_XG; ln += blockDim.x) {
    const int xl = ln % YZ_XG, z = ln / YZ_XG;
    float2 v[PY];
#pragma unroll
    for (int y = 0; y < PY; ++y)
      v[y] = (y < d.ny && xl < xg) ? xb[z * plane + (long long)y * d.nx + x0 + xl] : make_float2(0.f, 0.f);
    dft_p2<PY, -1>(v);
#pragma unroll
    for (int ky = 0; ky < PY; ++ky) S[(z * YZ_XG + xl) * PITCH + ky] = v[ky];
  }
  __syncthreads();
  // z transforms of the columns (xl, ky) (rows z >= nz are zero)
  float2* Tb = T + (long long)b * PZ * PY * d.nx;
  for (int ln = threadIdx.x; ln < YZ_XG * PY; ln += blockDim.x) {
    const int xl = ln % YZ_XG, ky = ln / YZ_XG;
    float2 v[PZ];
#pragma unroll
    for (int z = 0; z < PZ; ++z) v[z] = z < d.nz ? S[(z * YZ_XG + xl) * PITCH + ky] : make_float2(0.f, 0.f);
    dft_p2<PZ, -1>(v);
    if (xl < xg) {
#pragma unroll
      for (int kz = 0; kz < PZ; ++kz) Tb[((long long)kz * PY + ky) * d.nx + x0 + xl] = v[kz];
    }
  }
}

template <int PY, int PZ, int YZ_XG>
__global__ void __launch_bounds__(128) k_mv_yz_inv_r(const float2* __restrict__ T, const float2* __restrict__ x,
                                                     const float2* __restrict__ Mv, float2* __restrict__ y, MvDims d) {
  constexpr int PITCH = PY + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* S = reinterpret_cast<float2*>(smem_raw);   // [nz][XG][PITCH]
  const int a = blockIdx.y, x0 = blockIdx.x * YZ_XG;
  const int xg = min(YZ_XG, d.nx - x0);
  const float2* Ta = T + (long long)a * PZ * PY * d.nx;
  const long long plane = (long long)d.ny * d.nx;
  const long long off_a = (long long)a * d.nz * plane;
  // the epilogue's x and M of this thread's first output row, loaded before
  // the transforms so that their latency hides behind them
  float2 xp[PY / 2], mp[PY / 2];
  {
    const int ln = threadIdx.x;
    const int xl = ln % YZ_XG, z = ln / YZ_XG;
    const bool own = ln < d.nz * YZ_XG && xl < xg;
#pragma unroll
    for (int yy = 0; yy < PY / 2; ++yy) {
      xp[yy] = make_float2(0.f, 0.f);
      mp[yy] = make_float2(0.f, 0.f);
      if (own && yy < d.ny) {
        const long long vox = (long long)z * plane + (long long)yy * d.nx + x0 + xl;
        xp[yy] = x[off_a + vox];
        mp[yy] = Mv[vox];
      }
    }
  }
  // inverse z transforms of the columns (xl, ky); keep the rows z < nz
  for (int ln = threadIdx.x; ln < YZ_XG * PY; ln += blockDim.x) {
    const int xl = ln % YZ_XG, ky = ln / YZ_XG;
    float2 v[PZ];
#pragma unroll
    for (int kz = 0; kz < PZ; ++kz)
      v[kz] = xl < xg ? Ta[((long long)kz * PY + ky) * d.nx + x0 + xl] : make_float2(0.f, 0.f);
    dft_p2<PZ, +1>(v);
#pragma unroll
    for (int z = 0; z < PZ; ++z)
      if (z < d.nz) S[(z * YZ_XG + xl) * PITCH + ky] = v[z];
  }
  __syncthreads();
  // inverse y transforms of the rows z < nz, crop to ny, y = x - M (x + G x)
  for (int ln = threadIdx.x; ln < d.nz * YZ_XG; ln += blockDim.x) {
    const int xl = ln % YZ_XG, z = ln / YZ_XG;
    float2 v[PY];
#pragma unroll
    for (int ky = 0; ky < PY; ++ky) v[ky] = S[(z * YZ_XG + xl) * PITCH + ky];
    dft_p2<PY, +1>(v);
    if (xl < xg) {
      const bool first = ln == (int)threadIdx.x;
#pragma unroll
      for (int yy = 0; yy < PY / 2; ++yy) {
        if (yy < d.ny) {
          const long long vox = (long long)z * plane + (long long)yy * d.nx + x0 + xl;
          const float2 xv = first ? xp[yy] : x[off_a + vox];
          const float2 mv = first ? mp[yy] : Mv[vox];
          y[off_a + vox] = csub(xv, cmul(mv, cadd(xv, v[yy])));
        }
      }
    }
  }
}

// unfused x pass, step 2: tensor product on the full spectrum S[3][Pz][Py][L]
template <class C>
__global__ void k_mv_xmul(C* __restrict__ S, const C* __restrict__ spec, MvDims d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  (void)smem_raw;
  const int kyz = blockIdx.x;
  const int ky = kyz % d.Py, kz = kyz / d.Py;
  const long long lstride = (long long)d.Pz * d.Py * d.L;
  C* s0 = S + ((long long)kz * d.Py + ky) * d.L;
  tensor_mul(s0, s0 + lstride, s0 + 2 * lstride, d.L, ky, kz, spec, d);
}

template <class C>
__global__ void __launch_bounds__(256) k_mv_yz_inv(const C* __restrict__ T, const C* __restrict__ x,
                                                   const C* __restrict__ Mv, C* __restrict__ y, MvDims d,
                                                   FftPlanDev py, FftPlanDev pz, int XG) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int a = blockIdx.y;
  const int x0 = blockIdx.x * XG;
  const int xg = min(XG, d.nx - x0);
  const int SP = d.Py * d.Pz + 1;
  C* ba = s;
  C* bb = s + (size_t)XG * SP;
  const C* Ta = T + (long long)a * d.Pz * d.Py * d.nx;
  const int nin = xg * d.Py * d.Pz;
  batched_copy<8>(
      nin,
      [&](int e) {
        const int xl = e % xg, r = e / xg;
        const int ky = r % d.Py, kz = r / d.Py;
        return Ta[((long long)kz * d.Py + ky) * d.nx + x0 + xl];
      },
      [&](int e, C v) {
        const int xl = e % xg, r = e / xg;
        const int ky = r % d.Py, kz = r / d.Py;
        ba[xl * SP + kz * d.Py + ky] = v;
      });
  __syncthreads();
  // z lines (all Py columns), then y lines (only the nz rows kept)
  C* r1 = fft_smem_pp(ba, bb, pz, SmemLines{xg * d.Py, d.Py, 1, SP, d.Py, 1}, +1);
  C* r2 = fft_smem_pp(r1, r1 == ba ? bb : ba, py, SmemLines{xg * d.nz, d.nz, d.Py, SP, 1, 0}, +1);
  const long long plane = (long long)d.ny * d.nx;
  const long long off_a = (long long)a * d.nz * plane;
  const int nout = xg * d.ny * d.nz;
  struct XM { C x, m; };
  auto voxel = [&](int e, int& xl, int& yy, int& z) {
    xl = e % xg;
    const int r = e / xg;
    yy = r % d.ny;
    z = r / d.ny;
    return (long long)z * plane + (long long)yy * d.nx + x0 + xl;
  };
  batched_copy<4>(
      nout,
      [&](int e) {
        int xl, yy, z;
        const long long v = voxel(e, xl, yy, z);
        return XM{x[off_a + v], Mv[v]};
      },
      [&](int e, XM q) {
        int xl, yy, z;
        const long long v = voxel(e, xl, yy, z);
        const C g = r2[xl * SP + z * d.Py + yy];
        // y = x - M (x + Gx)
        y[off_a + v] = csub(q.x, cmul(q.m, cadd(q.x, g)));
      });
}

// epilogue of the split yz path: y holds G x on entry, y = x - M (x + G x)
template <class C>
__global__ void k_mv_epilogue(const C* __restrict__ x, const C* __restrict__ Mv, C* __restrict__ y, int nvox) {
  const long long n3 = 3LL * nvox;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x) {
    const C q = x[i];
    y[i] = csub(q, cmul(Mv[i % nvox], cadd(q, y[i])));
  }
}

static inline int pick_xg(const MvDims& d, size_t csize) {
  const size_t slab = (size_t)(d.Py * d.Pz + 1) * csize;
  int xg = 32;
  // two tile copies within about 64 KB: several blocks per SM and at least
  // two blocks per SM over the grid for the usual sizes
  while (xg > 1 && 2 * (size_t)xg * slab > 64 * 1024) xg /= 2;
  if (xg > d.nx) xg = std::max(1, d.nx);
  return xg;
}

template <class C> static FftPlanDev planof(const FftLen& f);
template <> inline FftPlanDev planof<double2>(const FftLen& f) { return f.pn64; }
template <> inline FftPlanDev planof<float2>(const FftLen& f) { return f.pn32; }

static inline int threads_for(long long E, int& maxe, int cap_per) {
  int threads = 128;
  while (threads < 1024 && E > (long long)cap_per * threads) threads *= 2;
  const long long per = (E + threads - 1) / threads;
  maxe = per <= 8 ? 8 : per <= 16 ? 16 : 32;
  return threads;
}

template <class K>
static vie_status set_smem(K kern, size_t smem) {
  return smem_optin(kern, smem);
}

#define VIE_DISPATCH_MAXE(ME, CALL)                                             \
  switch (ME) {                                                                 \
    case 8: CALL(8); break;                                                     \
    case 16: CALL(16); break;                                                   \
    default: set_error("matvec: tile too large for one block"); return VIE_EINVAL; \
  }

// Register yz pass (forward: x -> T; inverse: T -> y with the epilogue) for
// cross-section variant yzr (1: Py 32 x Pz 16, 2: 16 x 8) and xg x-columns per
// CTA (16, 8 or 4).
static inline vie_status yz_r_launch(const MvDims& d, int yzr, int xg, bool fwd, const float2* x, float2* T,
                                     const float2* Ti, const float2* Mv, float2* y, cudaStream_t st,
                                     const float2* xi = nullptr) {
  const int py = yzr == 1 ? 32 : 16;
  const size_t smem = (size_t)d.nz * xg * (py + 1) * sizeof(float2);
  const dim3 g(ceil_div(d.nx, xg), 3);
#define VIE_YZ(PY, PZ, XG)                                                                          \
  if (fwd) k_mv_yz_fwd_r<PY, PZ, XG><<<g, 128, smem, st>>>(x, T, d);                                \
  else k_mv_yz_inv_r<PY, PZ, XG><<<g, 128, smem, st>>>(Ti, xi, Mv, y, d);
  {
    Prof pf_(fwd ? "mv_yz_fwd_c64" : "mv_yz_inv_c64", st);
    if (yzr == 1) {
      if (xg == 16) { VIE_YZ(32, 16, 16) } else if (xg == 8) { VIE_YZ(32, 16, 8) } else { VIE_YZ(32, 16, 4) }
    } else {
      if (xg == 16) { VIE_YZ(16, 8, 16) } else if (xg == 8) { VIE_YZ(16, 8, 8) } else { VIE_YZ(16, 8, 4) }
    }
  }
#undef VIE_YZ
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

// register yz variant of a cross-section (0: none)
static inline int yz_variant(const MvDims& d) {
  return (d.Py == 32 && d.Pz == 16) ? 1 : (d.Py == 16 && d.Pz == 8) ? 2 : 0;
}

// The x pass alone (pass B of the matvec) in one of its variants: T holds
// the yz-transformed field on entry and the inverse x-transformed product on
// exit.  The autotuner times the variants with this entry.
// the cluster-split x pass with Q = 2, 4 or 8 CTAs per line triple
// (variants 5, 6, 7; Q = P->xq, the smallest that fits, by default)
static vie_status xpass_split(vie_plan_s* P, int Q, const float2* spec, float2* T, cudaStream_t st) {
  const MvDims& d = P->d;
  const int qi = Q == 2 ? 0 : Q == 4 ? 1 : 2;
  if (Q < P->xq || Q > 8 || d.L % Q || !P->fLq[qi]) { set_error("matvec: no %d-CTA split for L = %d", Q, d.L); return VIE_EINVAL; }
  const int Lq = d.L / Q;
  const size_t smem = 2 * 3 * (size_t)Lq * sizeof(float2);
  const FftPlanDev pl = planof<float2>(*P->fLq[qi]);
  const float2* tw = P->twL64.as<float2>();
  Prof pf_("mv_x_c64", st);
  if (Q == 2) {
    VIE_TRY(set_smem(k_mv_xq<2>, smem));
    k_mv_xq<2><<<d.Py * d.Pz * 2, 512, smem, st>>>(T, spec, d, pl, tw);
  } else if (Q == 4) {
    VIE_TRY(set_smem(k_mv_xq<4>, smem));
    k_mv_xq<4><<<d.Py * d.Pz * 4, 512, smem, st>>>(T, spec, d, pl, tw);
  } else {
    VIE_TRY(set_smem(k_mv_xq<8>, smem));
    k_mv_xq<8><<<d.Py * d.Pz * 8, 512, smem, st>>>(T, spec, d, pl, tw);
  }
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

template <class C>
vie_status xpass(vie_plan_s* P, const C* spec, C* T, C* S, int variant, cudaStream_t st) {
  const MvDims& d = P->d;
  const int cap = 16;
  if constexpr (sizeof(C) == 8) {
    if (P->xq > 1 && (variant >= 5 || variant < 0 || !P->fused_x64))
      return xpass_split(P, variant >= 5 ? 1 << (variant - 4) : P->xq, (const float2*)spec, (float2*)T, st);
  }
  const FftPlanDev plan_of = planof<C>(*P->fL);
  const bool fused = sizeof(C) == 16 ? P->fused_x128 : P->fused_x64;
  if (fused) {
    const size_t tile = (size_t)3 * d.L * sizeof(C);
    // variant 0 (or -1, untuned): the compile-time radix-16 kernel where one
    // exists; k >= 1: the generic Stockham kernel with radix order k - 1
    // variant 4: the four-pass compile-time kernel (L = 4096 or 8192), also the
    // default for L = 8192, which has no three-pass kernel
    const bool fp = sizeof(C) == 8 && ((d.L == 4096 && variant == 4) || (d.L == 8192 && (variant == 4 || variant < 0)));
    const bool ct = sizeof(C) == 8 && (d.L == 2048 || d.L == 4096) && variant <= 0;
    const FftPlanDev pl = (variant >= 1 && variant <= 3) ? P->xord[sizeof(C) == 8 ? 0 : 1][variant - 1] : plan_of;
    if (fp && d.L == 4096) {
      constexpr int L = 4096;
      const size_t smem = 3 * (size_t)(L + L / 16) * sizeof(float2);
      Prof pf_("mv_x_c64", st);
      VIE_TRY(set_smem(k_mv_x4p<16, 16, 4, 4>, smem));
      k_mv_x4p<16, 16, 4, 4><<<d.Py * d.Pz, L / 16, smem, st>>>((float2*)T, (const float2*)spec, d,
                                                                (const float2*)pl.tw);
    } else if (fp && d.L == 8192) {
      constexpr int L = 8192;
      const size_t smem = 3 * (size_t)(L + L / 16) * sizeof(float2);
      Prof pf_("mv_x_c64", st);
      VIE_TRY(set_smem(k_mv_x4p<16, 16, 8, 4>, smem));
      k_mv_x4p<16, 16, 8, 4><<<d.Py * d.Pz, L / 16, smem, st>>>((float2*)T, (const float2*)spec, d,
                                                                (const float2*)pl.tw);
    } else if (ct && d.L == 2048) {
      // compile-time radix structure 16 x 16 x 8 (complex FP32)
      constexpr int L = 2048;
      const size_t smem = 3 * (size_t)(L + L / 16) * sizeof(float2);
      Prof pf_("mv_x_c64", st);
      VIE_TRY(set_smem(k_mv_x16<16, 16, 8>, smem));
      k_mv_x16<16, 16, 8><<<d.Py * d.Pz, 128, smem, st>>>((float2*)T, (const float2*)spec, d, (const float2*)pl.tw);
    } else if (ct && d.L == 4096) {
      // 16 x 16 x 16, 256 threads, two blocks per SM
      constexpr int L = 4096;
      const size_t smem = 3 * (size_t)(L + L / 16) * sizeof(float2);
      Prof pf_("mv_x_c64", st);
      VIE_TRY(set_smem(k_mv_x16<16, 16, 16>, smem));
      k_mv_x16<16, 16, 16><<<d.Py * d.Pz, 256, smem, st>>>((float2*)T, (const float2*)spec, d, (const float2*)pl.tw);
    } else if (2 * tile <= 200 * 1024) {
      auto k = k_mv_x<C, 0>;
      VIE_TRY(set_smem(k, 2 * tile));
      Prof pf_(sizeof(C) == 8 ? "mv_x_c64" : "mv_x_c128", st);
      k<<<d.Py * d.Pz, 512, 2 * tile, st>>>(T, spec, d, pl, 1);
    } else {
      int meB;
      int joint = 1;
      int thB = threads_for(3LL * d.L, meB, cap);
      if ((long long)meB * thB < 3LL * d.L || meB > cap) {
        joint = 0;
        thB = threads_for((long long)d.L, meB, cap);
      }
      if ((long long)meB * thB < (joint ? 3LL : 1LL) * d.L) { set_error("matvec: x line too long"); return VIE_EINVAL; }
#define CALL_B(ME)                                                         \
  {                                                                        \
    auto k = k_mv_x<C, ME>;                                                \
    VIE_TRY(set_smem(k, tile));                                            \
    Prof pf_(sizeof(C) == 8 ? "mv_x_c64" : "mv_x_c128", st);               \
    k<<<d.Py * d.Pz, thB, tile, st>>>(T, spec, d, pl, joint);              \
  }
      VIE_DISPATCH_MAXE(meB, CALL_B)
#undef CALL_B
    }
    count_launch();
    VIE_CHECK_LAUNCH();
  } else {
    // forward x-FFT of every padded line into S, tensor product, inverse into T
    const int nl = 3 * d.Py * d.Pz;
    LineDesc lf = lines_flat(d.nx, d.L, nl, d.nx, 1, d.L, 1);
    if (!S) { set_error("matvec: missing x-spectrum scratch"); return VIE_EINVAL; }
    C* X = (C*)(sizeof(C) == 16 ? P->X128.p : P->X64.p);   // split scratch for over-long lines
    VIE_TRY(fft_lines<C>(T, S, lf, *P->fL, -1, 1.0, X, st));
    { Prof pf_(sizeof(C) == 8 ? "mv_xmul_c64" : "mv_xmul_c128", st); k_mv_xmul<C><<<d.Py * d.Pz, 256, 0, st>>>(S, spec, d); }
    count_launch();
    VIE_CHECK_LAUNCH();
    LineDesc li = lines_flat(d.L, d.nx, nl, d.L, 1, d.nx, 1);
    VIE_TRY(fft_lines<C>(S, T, li, *P->fL, +1, 1.0, X, st));
  }
  return VIE_OK;
}

template <class C>
vie_status matvec(vie_plan_s* P, const C* x, C* y, const C* Mv, const C* spec, C* T, C* S, cudaStream_t st) {
  const MvDims& d = P->d;
  const int cap = 16;
  // pass A
  // x-columns per CTA of the generic yz passes: the autotuner's choice
  // (complex FP32), else the rule of pick_xg
  const int XG = (sizeof(C) == 8 && P->yzxg_gen > 0) ? std::min(P->yzxg_gen, std::max(1, d.nx)) : pick_xg(d, sizeof(C));
  const size_t smemA = 2 * (size_t)XG * (d.Py * d.Pz + 1) * sizeof(C);
  dim3 gA(ceil_div(d.nx, XG), 3);
  const FftPlanDev py = planof<C>(*P->fPy), pz = planof<C>(*P->fPz), pl = planof<C>(*P->fL);
  // register transforms for the power-of-two cross-sections that have an instantiation
  const int yzr = sizeof(C) == 8 ? yz_variant(d) : 0;
  const int yzxg = P->yzxg > 0 ? P->yzxg : 16;
  C* U = (C*)(sizeof(C) == 16 ? P->U128.p : P->U64.p);
  const long long pyx = (long long)d.Py * d.nx;
  if (P->yz_split) {
    // y-lines of every (b, z) row (stride nx), padded to Py, into U; then
    // z-lines of every (b, ky, x) (stride Py nx), padded to Pz, into T
    LineDesc dy{d.ny, d.Py, 3 * d.nz * d.nx, d.nx, 3 * d.nz, 1, (long long)d.ny * d.nx, 0, d.nx,
                1, pyx, 0, d.nx};
    VIE_TRY(fft_lines<C>(x, U, dy, *P->fPy, -1, 1.0, nullptr, st));
    LineDesc dz{d.nz, d.Pz, (int)(3 * pyx), (int)pyx, 3, 1, d.nz * pyx, 0, pyx, 1, d.Pz * pyx, 0, pyx};
    VIE_TRY(fft_lines<C>(U, T, dz, *P->fPz, -1, 1.0, nullptr, st));
  } else if (yzr) {
    VIE_TRY(yz_r_launch(d, yzr, yzxg, true, (const float2*)x, (float2*)T, nullptr, nullptr, nullptr, st));
  } else {
    auto k = k_mv_yz_fwd<C>;
    VIE_TRY(set_smem(k, smemA));
    Prof pf_(sizeof(C) == 8 ? "mv_yz_fwd_c64" : "mv_yz_fwd_c128", st);
    k<<<gA, 256, smemA, st>>>(x, T, d, py, pz, XG);
  }
  if (!P->yz_split) count_launch();
  VIE_CHECK_LAUNCH();
  // pass B
  VIE_TRY(xpass<C>(P, spec, T, S, P->xvar[sizeof(C) == 8 ? 0 : 1], st));
  // pass C
  if (P->yz_split) {
    // inverse z-lines (keep z < nz) into U, inverse y-lines (keep y < ny) into
    // y, then the epilogue; 1/(L Py Pz) is in the spectra
    LineDesc iz{d.Pz, d.nz, (int)(3 * pyx), (int)pyx, 3, 1, d.Pz * pyx, 0, pyx, 1, d.nz * pyx, 0, pyx};
    VIE_TRY(fft_lines<C>(T, U, iz, *P->fPz, +1, 1.0, nullptr, st));
    LineDesc iy{d.Py, d.ny, 3 * d.nz * d.nx, d.nx, 3 * d.nz, 1, pyx, 0, d.nx, 1, (long long)d.ny * d.nx, 0, d.nx};
    VIE_TRY(fft_lines<C>(U, y, iy, *P->fPy, +1, 1.0, nullptr, st));
    const int nvox = d.nx * d.ny * d.nz;
    Prof pf_(sizeof(C) == 8 ? "mv_epilogue_c64" : "mv_epilogue_c128", st);
    k_mv_epilogue<C><<<(int)std::min<long long>((3LL * nvox + 255) / 256, 152LL * 8), 256, 0, st>>>(x, Mv, y, nvox);
    count_launch();
    VIE_CHECK_LAUNCH();
    return VIE_OK;
  }
  if (yzr) {
    VIE_TRY(yz_r_launch(d, yzr, yzxg, false, nullptr, nullptr, (const float2*)T, (const float2*)Mv, (float2*)y, st,
                        (const float2*)x));
  } else {
    auto k = k_mv_yz_inv<C>;
    VIE_TRY(set_smem(k, smemA));
    Prof pf_(sizeof(C) == 8 ? "mv_yz_inv_c64" : "mv_yz_inv_c128", st);
    k<<<gA, 256, smemA, st>>>(T, x, Mv, y, d, py, pz, XG);
  }
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

}  // namespace vie
