// Green's-tensor generators of the voxel JVIE operator and their circulant
// embedding spectra (FP64), plus the material operator M.
//
// N = I + G with G f = (k^2 + grad div) int g f, g = exp(-jkR)/(4 pi R)
// (Sec. 2).  Entries for voxel offset d != 0 (one-point rule, R = h|d|,
// r = d/|d|, V = h^3):
//   G^{ab}(d) = V g [ (k^2 - (1+jkR)/R^2) delta_ab + (3 + 3jkR - k^2R^2)/R^2 r_a r_b ]
// and for d = 0 the field at the centre of the equal-volume sphere,
//   G^{aa}(0) = -1/3 + (2/3)((1 + jka) exp(-jka) - 1),  a = (3V/4pi)^(1/3).
// Each of the 6 unique components (xx, xy, xz, yy, yz, zz; N^{ab} = N^{ba},
// remark after Eq. sys_mat) is a 3-level Toeplitz generator over offsets
// (-(n-1)..n-1) per axis.  It is placed in an L x Py x Pz circulant (offset d
// at index d mod P, other indices zero), transformed in FP64, and only the
// non-negative-frequency octant is kept: the component has parity +-1 in each
// axis (the r_a r_b factor), so its spectrum has the same parity.
#include <math.h>

#include <algorithm>

#include "greens.cuh"
#include "internal.h"

namespace vie {

// fill the padded circulant of component c: out[Pz][Py][L]
__global__ void k_gen_padded(double2* __restrict__ out, int c, MvDims d, double h, double k, double2 self) {
  const long long P = (long long)d.L * d.Py * d.Pz;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < P;
       idx += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(idx % d.L);
    const long long r = idx / d.L;
    const int iy = (int)(r % d.Py);
    const int iz = (int)(r / d.Py);
    int dx, dy, dz;
    bool ok = true;
    if (ix < d.nx) dx = ix; else if (ix > d.L - d.nx) dx = ix - d.L; else { dx = 0; ok = false; }
    if (iy < d.ny) dy = iy; else if (iy > d.Py - d.ny) dy = iy - d.Py; else { dy = 0; ok = false; }
    if (iz < d.nz) dz = iz; else if (iz > d.Pz - d.nz) dz = iz - d.Pz; else { dz = 0; ok = false; }
    out[idx] = ok ? gen_entry(c, dx, dy, dz, h, k, self) : make_double2(0.0, 0.0);
  }
}

// keep the non-negative octant, scaled by 1/(L Py Pz)
__global__ void k_octant(const double2* __restrict__ full, double2* __restrict__ s128,
                         float2* __restrict__ s64, int c, MvDims d, double scale) {
  const long long Q = (long long)d.Lh * d.Pyh * d.Pzh;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < Q;
       idx += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(idx % d.Lh);
    const long long r = idx / d.Lh;
    const int ky = (int)(r % d.Pyh);
    const int kz = (int)(r / d.Pyh);
    double2 v = full[((long long)kz * d.Py + ky) * d.L + kx];
    v.x *= scale;
    v.y *= scale;
    s128[(long long)c * Q + idx] = v;
    s64[(long long)c * Q + idx] = make_float2((float)v.x, (float)v.y);
  }
}

vie_status build_spectra(vie_plan_s* P) {
  const MvDims& d = P->d;
  const long long Pn = (long long)d.L * d.Py * d.Pz;
  const long long Q = (long long)d.Lh * d.Pyh * d.Pzh;
  VIE_TRY(P->spec128.alloc(sizeof(double2) * 6 * Q));
  VIE_TRY(P->spec64.alloc(sizeof(float2) * 6 * Q));
  DevBuf full, xsplit;
  VIE_TRY(full.alloc(sizeof(double2) * Pn));
  const size_t xs = fft_scratch_elems<double2>(*P->fL, d.Py * d.Pz);
  if (xs) VIE_TRY(xsplit.alloc(sizeof(double2) * xs));
  const double2 self = self_term_value(P->h, P->kb);
  const int threads = 256;
  const int grid = (int)std::min<long long>((Pn + threads - 1) / threads, 152LL * 16);
  for (int c = 0; c < 6; ++c) {
    k_gen_padded<<<grid, threads, 0, P->st>>>(full.as<double2>(), c, d, P->h, P->kb, self);
    count_launch();
    VIE_CHECK_LAUNCH();
    double2* f = full.as<double2>();
    // x lines: contiguous, Py*Pz of them
    LineDesc lx = lines_flat(d.L, d.L, d.Py * d.Pz, d.L, 1, d.L, 1);
    VIE_TRY(fft_lines<double2>(f, f, lx, *P->fL, -1, 1.0, xsplit.as<double2>(), P->st));
    // y lines: stride L, lines (x, z)
    LineDesc ly{d.Py, d.Py, d.L * d.Pz, d.L, d.Pz, 1, (long long)d.L * d.Py, 0, d.L,
                1, (long long)d.L * d.Py, 0, d.L};
    VIE_TRY(fft_lines<double2>(f, f, ly, *P->fPy, -1, 1.0, nullptr, P->st));
    // z lines: stride L*Py, lines (x, y)
    LineDesc lz = lines_flat(d.Pz, d.Pz, d.L * d.Py, 1, (long long)d.L * d.Py, 1, (long long)d.L * d.Py);
    VIE_TRY(fft_lines<double2>(f, f, lz, *P->fPz, -1, 1.0, nullptr, P->st));
    const int g2 = (int)std::min<long long>((Q + threads - 1) / threads, 152LL * 16);
    k_octant<<<g2, threads, 0, P->st>>>(f, P->spec128.as<double2>(), P->spec64.as<float2>(), c, d,
                                        1.0 / (double)Pn);
    count_launch();
    VIE_CHECK_LAUNCH();
  }
  VIE_CUDA(cudaStreamSynchronize(P->st));
  return VIE_OK;
}

// M = (eps/eps_bg - 1) / (eps/eps_bg)  (Sec. 2, after Eq. JVIE)
__global__ void k_material(const double2* __restrict__ eps, double2* __restrict__ M128,
                           float2* __restrict__ M64, long long n, double eps_bg) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 e = eps[i];
    const double er = e.x / eps_bg, ei = e.y / eps_bg;
    // 1 - 1/e
    const double den = er * er + ei * ei;
    const double mr = 1.0 - er / den, mi = ei / den;
    M128[i] = make_double2(mr, mi);
    M64[i] = make_float2((float)mr, (float)mi);
  }
}

vie_status set_material(vie_plan_s* P, const double2* eps) {
  const long long n = (long long)P->nx * P->ny * P->nz;
  if (!P->M128.p) {
    VIE_TRY(P->M128.alloc(sizeof(double2) * n));
    VIE_TRY(P->M64.alloc(sizeof(float2) * n));
  }
  const int threads = 256;
  const int grid = (int)std::min<long long>((n + threads - 1) / threads, 152LL * 8);
  k_material<<<grid, threads, 0, P->st>>>(eps, P->M128.as<double2>(), P->M64.as<float2>(), n, P->eps_bg);
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

}  // namespace vie

namespace vie {

// Launch wrappers over explicit buffers (used by the allocation-free matvec
// entry point); the plan path above is unchanged.
vie_status launch_gen_padded(double2* out, int c, const MvDims& d, double h, double kb, cudaStream_t st) {
  const long long Pn = (long long)d.L * d.Py * d.Pz;
  const int threads = 256;
  const int grid = (int)std::min<long long>((Pn + threads - 1) / threads, 152LL * 16);
  k_gen_padded<<<grid, threads, 0, st>>>(out, c, d, h, kb, self_term_value(h, kb));
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

vie_status launch_octant(const double2* full, double2* s128, float2* s64, int c, const MvDims& d, cudaStream_t st) {
  const long long Q = (long long)d.Lh * d.Pyh * d.Pzh;
  const long long Pn = (long long)d.L * d.Py * d.Pz;
  const int threads = 256;
  const int grid = (int)std::min<long long>((Q + threads - 1) / threads, 152LL * 16);
  k_octant<<<grid, threads, 0, st>>>(full, s128, s64, c, d, 1.0 / (double)Pn);
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

vie_status launch_material(const double2* eps, double2* M128, float2* M64, long long n, double eps_bg,
                           cudaStream_t st) {
  const int threads = 256;
  const int grid = (int)std::min<long long>((n + threads - 1) / threads, 152LL * 8);
  k_material<<<grid, threads, 0, st>>>(eps, M128, M64, n, eps_bg);
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

}  // namespace vie
