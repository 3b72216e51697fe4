// Matvec workspace and precision conversions (kernels of the matvec proper
// are in matvec_impl.cuh, instantiated by matvec_f32.cu and matvec_f64.cu).
#include <algorithm>

#include "internal.h"

namespace vie {

vie_status matvec_alloc(vie_plan_s* P) {
  const MvDims& d = P->d;
  const long long nT = 3LL * d.Pz * d.Py * d.nx;
  VIE_TRY(P->T128.alloc(sizeof(double2) * nT));
  VIE_TRY(P->T64.alloc(sizeof(float2) * nT));
  // the fused x pass holds 3 lines of length L in shared memory; larger
  // embeddings go through the full x-spectrum S instead
  const long long nS = 3LL * d.Pz * d.Py * d.L;
  P->fused_x128 = (size_t)3 * d.L * sizeof(double2) <= 200 * 1024;
  P->fused_x64 = (size_t)3 * d.L * sizeof(float2) <= 200 * 1024;
  if (!P->fused_x128) VIE_TRY(P->S128.alloc(sizeof(double2) * nS));
  // (complex FP32 split over a cluster keeps its lines in shared memory)
  const bool unfused64 = !P->fused_x64 && P->xq == 1;
  if (unfused64) VIE_TRY(P->S64.alloc(sizeof(float2) * nS));
  const int nl = 3 * d.Py * d.Pz;
  const size_t x128 = P->fused_x128 ? 0 : fft_scratch_elems<double2>(*P->fL, nl);
  const size_t x64 = unfused64 ? fft_scratch_elems<float2>(*P->fL, nl) : 0;
  if (x128) VIE_TRY(P->X128.alloc(sizeof(double2) * x128));
  if (x64) VIE_TRY(P->X64.alloc(sizeof(float2) * x64));
  // cross-sections whose Py x Pz slab does not fit shared memory take the
  // y- and z-transforms as separate line passes through U[3][nz][Py][nx]
  P->yz_split = (long long)d.Py * d.Pz > 4096;
  if (P->yz_split) {
    const long long nU = 3LL * d.nz * d.Py * d.nx;
    VIE_TRY(P->U128.alloc(sizeof(double2) * nU));
    VIE_TRY(P->U64.alloc(sizeof(float2) * nU));
  }
  const long long n3 = 3LL * d.nx * d.ny * d.nz;
  VIE_TRY(P->xin64.alloc(sizeof(float2) * n3));
  VIE_TRY(P->xout64.alloc(sizeof(float2) * n3));
  return VIE_OK;
}

// precision conversions
__global__ void k_widen(const float2* __restrict__ a, double2* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = make_double2(a[i].x, a[i].y);
}
__global__ void k_narrow(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
vie_status widen(const float2* a, double2* b, long long n, cudaStream_t st) {
  const int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
  k_widen<<<grid, 256, 0, st>>>(a, b, n);
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}
vie_status narrow(const double2* a, float2* b, long long n, cudaStream_t st) {
  const int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
  k_narrow<<<grid, 256, 0, st>>>(a, b, n);
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

}  // namespace vie
