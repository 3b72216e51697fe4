// Common device/host helpers for libvie: complex arithmetic on float2/double2,
// error reporting and launch utilities.  All code targets sm_103a only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/vie.h"

namespace vie {

// ---------------------------------------------------------------------------
// error state (thread-local message, see vie_last_error)
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);

#define VIE_CUDA(call)                                                          \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      ::vie::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,               \
                       cudaGetErrorString(e_));                                 \
      return VIE_ECUDA;                                                         \
    }                                                                           \
  } while (0)

#define VIE_CHECK_LAUNCH()                                                      \
  do {                                                                          \
    cudaError_t e_ = cudaGetLastError();                                        \
    if (e_ != cudaSuccess) {                                                    \
      ::vie::set_error("%s:%d launch: %s", __FILE__, __LINE__,                  \
                       cudaGetErrorString(e_));                                 \
      return VIE_ECUDA;                                                         \
    }                                                                           \
  } while (0)

#define VIE_TRY(expr)                                                           \
  do {                                                                          \
    vie_status s_ = (expr);                                                     \
    if (s_ < 0) return s_;                                                      \
  } while (0)

// Let a kernel use the device's whole opt-in dynamic shared memory (less its
// static shared memory) and check that `need` bytes fit.  Every caller sets
// the same value, so a plan built on another host thread can never lower the
// limit under a launch in flight.  Cached per device and kernel.
vie_status smem_optin_raw(const void* kern, size_t need);
// Without the opt-in a block may use 48 KB of static and dynamic shared
// memory together: the opt-in is skipped only for requests of at most 32 KB,
// which leaves 16 KB for the kernel's static arrays.
template <class K>
inline vie_status smem_optin(K* kern, size_t need) {
  return need <= 32 * 1024 ? VIE_OK : smem_optin_raw((const void*)kern, need);
}

// ---------------------------------------------------------------------------
// complex types
// ---------------------------------------------------------------------------
template <class T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <class T> using cplx = typename cplx_of<T>::type;

template <class C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

template <class C>
__host__ __device__ __forceinline__ C cmake(typename real_of<C>::type re, typename real_of<C>::type im) {
  C r; r.x = re; r.y = im; return r;
}
template <class C> __host__ __device__ __forceinline__ C czero() { return cmake<C>(0, 0); }
template <class C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <class C> __host__ __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <class C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <class C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  return cmake<C>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <class C> __host__ __device__ __forceinline__ C cscale(C a, typename real_of<C>::type s) {
  return cmake<C>(a.x * s, a.y * s);
}
template <class C> __host__ __device__ __forceinline__ C cconj(C a) { return cmake<C>(a.x, -a.y); }
template <class C> __host__ __device__ __forceinline__ typename real_of<C>::type cabs2(C a) {
  return a.x * a.x + a.y * a.y;
}
// acc += a * b
template <class C> __host__ __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <class C> __host__ __device__ __forceinline__ void cfmac(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

template <class Cto, class Cfrom> __host__ __device__ __forceinline__ Cto cconv(Cfrom a) {
  return cmake<Cto>((typename real_of<Cto>::type)a.x, (typename real_of<Cto>::type)a.y);
}

// 1/z for double2
__host__ __device__ __forceinline__ double2 cinv(double2 z) {
  double d = 1.0 / (z.x * z.x + z.y * z.y);
  return make_double2(z.x * d, -z.y * d);
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

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// SM count of the current device (cached per process; one device per process)
int sm_count();

}  // namespace vie
