// vie_matvec_static: the complex-FP64 matvec y = x - M (x + G x) for callers
// that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a
// host framework that owns all device memory through its own pool, in a
// real-time loop with a fixed memory budget, or in a process that forbids
// libraries from growing their footprint after start-up.  Such a caller
// cannot create a plan (vie_plan_create allocates the generator spectra and
// the matvec intermediate), so this entry point takes only the caller's
// buffers and keeps every temporary -- FFT twiddles, the material operator,
// the generator spectra and the yz-transformed intermediate -- in one
// file-scope device array of kStaticScratchBytes (64 MiB).  That array is part of
// the library image: every GPU that loads libvie holds it until the process
// exits, used or not.
//
// Sharing: every call uses the same array and leaves its contents behind.
// Each call rewrites every region it reads before reading it (the padded
// generator grid, the spectra, M and the intermediate are written in full),
// so nothing has to start at zero.  Two calls whose GPU work overlaps (two
// streams, or two host threads) race on the array and corrupt each other.
#include <math.h>

#include <algorithm>

#include "internal.h"

namespace vie {

vie_status launch_gen_padded(double2* out, int c, const MvDims& d, double h, double kb, cudaStream_t st);
vie_status launch_octant(const double2* full, double2* s128, float2* s64, int c, const MvDims& d, cudaStream_t st);
vie_status launch_material(const double2* eps, double2* M128, float2* M64, long long n, double eps_bg,
                           cudaStream_t st);

constexpr size_t kStaticScratchBytes = 64ull << 20;   // 64 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on the current device.  Host code may
// not use the symbol itself as a pointer, and the address can change when a
// device's context is re-created (cudaDeviceReset), so it is looked up on
// every call (a host-side query that allocates nothing).
static vie_status static_scratch(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    set_error("vie_matvec_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return VIE_ECUDA;
  }
  *out = p;
  return VIE_OK;
}

// tw[k] = exp(-2 pi i k / n), computed on the device
__global__ void k_twiddles(double2* __restrict__ tw, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)k / (double)n, &s, &c);
    tw[k] = make_double2(c, -s);
  }
}

static bool factor_radices(int n, FftPlanDev& p) {
  if (!fft_factorize(n, p)) return false;
  fft_plan_finalize(p);
  return true;
}

// true if the byte ranges [a, a + na) and [b, b + nb) share a byte
static bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
  return pa < pb + nb && pb < pa + na;
}

struct Carve {
  unsigned char* base;
  size_t off = 0, cap;
  void* take(size_t bytes) {
    off = (off + 255) & ~size_t(255);
    void* p = base + off;
    off += bytes;
    return off <= cap ? p : nullptr;
  }
};

static size_t static_need(const MvDims& d) {
  const size_t N = (size_t)d.nx * d.ny * d.nz;
  const size_t Q = (size_t)d.Lh * d.Pyh * d.Pzh;
  const size_t work = std::max((size_t)d.L * d.Py * d.Pz, (size_t)3 * d.nx * d.Py * d.Pz);
  size_t s = 0;
  auto add = [&](size_t b) { s = ((s + 255) & ~size_t(255)) + b; };
  add(sizeof(double2) * d.L);
  add(sizeof(double2) * d.Py);
  add(sizeof(double2) * d.Pz);
  add(sizeof(double2) * N);
  add(sizeof(float2) * N);
  add(sizeof(double2) * 6 * Q);
  add(sizeof(float2) * 6 * Q);
  add(sizeof(double2) * work);
  return s;
}

static int embed(int n) { return 2 * fft_next_smooth(n); }

}  // namespace vie

using namespace vie;

extern "C" vie_status vie_matvec_static(int nx, int ny, int nz, double h, double k0, double eps_bg,
                                        const void* eps_dev, const void* x_dev, void* y_dev, void* cuda_stream) {
  if (nx < 1 || ny < 1 || nz < 1 || !(h > 0) || !(k0 >= 0) || !(eps_bg > 0) || !eps_dev || !x_dev || !y_dev) {
    set_error("vie_matvec_static: invalid arguments");
    return VIE_EINVAL;
  }
  {
    // y is written while x and eps are still read: no byte of y may alias them
    const size_t nvox = (size_t)nx * ny * nz;
    if (overlaps(x_dev, 3 * nvox * sizeof(double2), y_dev, 3 * nvox * sizeof(double2)) ||
        overlaps(eps_dev, nvox * sizeof(double2), y_dev, 3 * nvox * sizeof(double2))) {
      set_error("vie_matvec_static: y overlaps x or eps");
      return VIE_EINVAL;
    }
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  vie_plan_s P;   // geometry only: owns no device memory
  MvDims& d = P.d;
  d.nx = nx; d.ny = ny; d.nz = nz;
  d.L = embed(nx); d.Py = embed(ny); d.Pz = embed(nz);
  d.Lh = d.L / 2 + 1; d.Pyh = d.Py / 2 + 1; d.Pzh = d.Pz / 2 + 1;
  if ((long long)d.Py * d.Pz > 4096 || (size_t)3 * d.L * sizeof(double2) > 200 * 1024) {
    set_error("vie_matvec_static: grid %dx%dx%d outside the supported shapes (nx <= 2130, Py*Pz <= 4096)", nx, ny, nz);
    return VIE_EINVAL;
  }
  const size_t need = static_need(d);
  if (need > kStaticScratchBytes) {
    set_error("vie_matvec_static: grid %dx%dx%d needs %zu bytes of scratch, more than the %zu available", nx, ny, nz,
              need, kStaticScratchBytes);
    return VIE_EINVAL;
  }
  void* base = nullptr;
  VIE_TRY(static_scratch(&base));
  Carve cv{(unsigned char*)base, 0, kStaticScratchBytes};
  const long long N = (long long)nx * ny * nz;
  const long long Q = (long long)d.Lh * d.Pyh * d.Pzh;
  const size_t work = std::max((size_t)d.L * d.Py * d.Pz, (size_t)3 * d.nx * d.Py * d.Pz);
  double2* twL = (double2*)cv.take(sizeof(double2) * d.L);
  double2* twY = (double2*)cv.take(sizeof(double2) * d.Py);
  double2* twZ = (double2*)cv.take(sizeof(double2) * d.Pz);
  double2* M128 = (double2*)cv.take(sizeof(double2) * N);
  float2* M64 = (float2*)cv.take(sizeof(float2) * N);
  double2* s128 = (double2*)cv.take(sizeof(double2) * 6 * Q);
  float2* s64 = (float2*)cv.take(sizeof(float2) * 6 * Q);
  double2* wk = (double2*)cv.take(sizeof(double2) * work);
  if (!wk) { set_error("vie_matvec_static: scratch layout overflow"); return VIE_EINVAL; }

  // transform lengths with twiddles in the static array
  FftLen fL, fY, fZ;
  fL.n = d.L; fY.n = d.Py; fZ.n = d.Pz;
  if (!factor_radices(d.L, fL.pn64) || !factor_radices(d.Py, fY.pn64) || !factor_radices(d.Pz, fZ.pn64)) {
    set_error("vie_matvec_static: embedding length not 7-smooth");
    return VIE_EINVAL;
  }
  fL.pn64.tw = twL; fY.pn64.tw = twY; fZ.pn64.tw = twZ;
  k_twiddles<<<ceil_div(d.L, 256), 256, 0, st>>>(twL, d.L);
  k_twiddles<<<ceil_div(d.Py, 256), 256, 0, st>>>(twY, d.Py);
  k_twiddles<<<ceil_div(d.Pz, 256), 256, 0, st>>>(twZ, d.Pz);
  count_launch(3);
  VIE_CHECK_LAUNCH();
  P.fL = &fL; P.fPy = &fY; P.fPz = &fZ;
  P.fused_x128 = true;

  // generator spectra (FP64), one component at a time through the work area
  const double kb = k0 * sqrt(eps_bg);
  for (int c = 0; c < 6; ++c) {
    VIE_TRY(launch_gen_padded(wk, c, d, h, kb, st));
    LineDesc lx = lines_flat(d.L, d.L, d.Py * d.Pz, d.L, 1, d.L, 1);
    VIE_TRY(fft_lines<double2>(wk, wk, lx, fL, -1, 1.0, nullptr, st));
    LineDesc ly{d.Py, d.Py, d.L * d.Pz, d.L, d.Pz, 1, (long long)d.L * d.Py, 0, d.L,
                1, (long long)d.L * d.Py, 0, d.L};
    VIE_TRY(fft_lines<double2>(wk, wk, ly, fY, -1, 1.0, nullptr, st));
    LineDesc lz = lines_flat(d.Pz, d.Pz, d.L * d.Py, 1, (long long)d.L * d.Py, 1, (long long)d.L * d.Py);
    VIE_TRY(fft_lines<double2>(wk, wk, lz, fZ, -1, 1.0, nullptr, st));
    VIE_TRY(launch_octant(wk, s128, s64, c, d, st));
  }
  VIE_TRY(launch_material((const double2*)eps_dev, M128, M64, N, eps_bg, st));
  // the three matvec passes, intermediate in the work area
  return matvec<double2>(&P, (const double2*)x_dev, (double2*)y_dev, M128, s128, wk, nullptr, st);
}
