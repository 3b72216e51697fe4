// Batched line FFTs through shared memory, with Bluestein's chirp-z
// decomposition for lengths that are not 7-smooth.
#include <math.h>
#include <stdarg.h>

#include <algorithm>
#include <atomic>
#include <complex>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "fft.cuh"
#include "prof.h"

namespace vie {

static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;   // this thread's share (graph capture accounting)
void count_launch(int n) {
  g_launches += n;
  t_launches += n;
}
long long launches_total() { return g_launches.load(); }
long long launches_thread() { return t_launches; }

bool fft_smooth(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

int fft_next_smooth(int n) {
  if (n < 1) n = 1;
  while (!fft_smooth(n)) ++n;
  return n;
}

static int next_pow2(int n) {
  int m = 1;
  while (m < n) m <<= 1;
  return m;
}

// radix sequence: 8s, then one 4 or 2, then 3s, 5s, 7s (the order the fused
// x pass and the line kernels assume); false if n is not 7-smooth or needs
// more than FFT_MAX_PASSES passes
bool fft_factorize(int n, FftPlanDev& p) {
  p.n = n;
  p.npass = 0;
  int m = n, a = 0;
  while (m % 2 == 0) { m /= 2; ++a; }
  auto push = [&p](int r) {
    if (p.npass >= FFT_MAX_PASSES) return false;
    p.radix[p.npass++] = r;
    return true;
  };
  for (; a >= 3; a -= 3)
    if (!push(8)) return false;
  if (a == 2 && !push(4)) return false;
  if (a == 1 && !push(2)) return false;
  for (int r : {3, 5, 7})
    for (; m % r == 0; m /= r)
      if (!push(r)) return false;
  return m == 1;
}

template <class C>
static vie_status upload(const std::vector<std::complex<double>>& v, C** out) {
  std::vector<C> h(v.size());
  for (size_t i = 0; i < v.size(); ++i) h[i] = cmake<C>((typename real_of<C>::type)v[i].real(),
                                                        (typename real_of<C>::type)v[i].imag());
  VIE_CUDA(cudaMalloc((void**)out, sizeof(C) * (v.size() ? v.size() : 1)));
  VIE_CUDA(cudaMemcpy(*out, h.data(), sizeof(C) * v.size(), cudaMemcpyHostToDevice));
  return VIE_OK;
}

static vie_status make_plan(int n, FftPlanDev& p64, FftPlanDev& p32) {
  if (!fft_factorize(n, p64)) { set_error("fft: %d is not 7-smooth", n); return VIE_EINVAL; }
  fft_plan_finalize(p64);
  p32 = p64;
  std::vector<std::complex<double>> tw(n);
  for (int k = 0; k < n; ++k) {
    const double a = -2.0 * M_PI * (double)k / (double)n;
    tw[k] = std::complex<double>(cos(a), sin(a));
  }
  double2* t64; float2* t32;
  VIE_TRY(upload(tw, &t64));
  VIE_TRY(upload(tw, &t32));
  p64.tw = t64;
  p32.tw = t32;
  return VIE_OK;
}

// host radix-2 FFT (sign -1), used once per Bluestein length for the chirp
// spectrum
static void host_fft_pow2(std::vector<std::complex<double>>& a) {
  const size_t n = a.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    for (size_t i = 0; i < n; i += len) {
      for (size_t k = 0; k < len / 2; ++k) {
        const double ang = -2.0 * M_PI * (double)k / (double)len;
        const std::complex<double> w(cos(ang), sin(ang));
        const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
    }
  }
}

static std::mutex g_fft_mu;
static std::map<int, std::unique_ptr<FftLen>>* g_fft_cache = nullptr;

vie_status fft_get(int n, const FftLen** out) {
  std::lock_guard<std::mutex> lk(g_fft_mu);
  if (!g_fft_cache) g_fft_cache = new std::map<int, std::unique_ptr<FftLen>>();
  auto it = g_fft_cache->find(n);
  if (it != g_fft_cache->end()) { *out = it->second.get(); return VIE_OK; }
  if (n < 1) { set_error("fft: bad length %d", n); return VIE_EINVAL; }
  std::unique_ptr<FftLen> f(new FftLen());
  f->n = n;
  if (fft_smooth(n)) {
    VIE_TRY(make_plan(n, f->pn64, f->pn32));
  } else {
    f->bluestein = true;
    f->M = next_pow2(2 * n - 1);
    const int M = f->M;
    VIE_TRY(make_plan(M, f->pm64, f->pm32));
    std::vector<std::complex<double>> b(n);
    for (int k = 0; k < n; ++k) {
      const long long e = ((long long)k * k) % (2LL * n);
      const double a = M_PI * (double)e / (double)n;
      b[k] = std::complex<double>(cos(a), sin(a));
    }
    std::vector<std::complex<double>> cf(M, 0.0), ci(M, 0.0);
    for (int j = 0; j < n; ++j) {
      cf[j] = b[j];
      ci[j] = std::conj(b[j]);
      if (j > 0) { cf[M - j] = b[j]; ci[M - j] = std::conj(b[j]); }
    }
    host_fft_pow2(cf);
    host_fft_pow2(ci);
    for (int j = 0; j < M; ++j) { cf[j] /= (double)M; ci[j] /= (double)M; }
    VIE_TRY(upload(b, &f->chirp64));
    VIE_TRY(upload(b, &f->chirp32));
    VIE_TRY(upload(cf, &f->hatf64));
    VIE_TRY(upload(cf, &f->hatf32));
    VIE_TRY(upload(ci, &f->hati64));
    VIE_TRY(upload(ci, &f->hati32));
  }
  // A pageable cudaMemcpy may return before its DMA lands, and the tables are
  // read by kernels on non-blocking streams: make them complete before the
  // length becomes visible to any caller.
  VIE_CUDA(cudaStreamSynchronize(cudaStreamLegacy));
  *out = f.get();
  (*g_fft_cache)[n] = std::move(f);
  return VIE_OK;
}

template <class C> static const FftPlanDev& plan_n(const FftLen& f);
template <> const FftPlanDev& plan_n<double2>(const FftLen& f) { return f.bluestein ? f.pm64 : f.pn64; }
template <> const FftPlanDev& plan_n<float2>(const FftLen& f) { return f.bluestein ? f.pm32 : f.pn32; }

template <class C> int fft_max_len() { return (int)((200 * 1024) / sizeof(C)) - 64; }
template int fft_max_len<float2>();
template int fft_max_len<double2>();

// pre/post modes: 0 none, 1 multiply, 2 multiply by conjugate.
// MAXE == 0: out-of-place (ping-pong) passes over two tile copies; MAXE > 0:
// in-place passes, for lines too long to double-buffer.
template <class C, int MAXE>
__global__ void __launch_bounds__(MAXE == 0 ? 256 : 1024)
    k_fft_lines(const C* __restrict__ in, C* __restrict__ out, LineDesc d, FftPlanDev p, int sign, int lpc,
                const C* __restrict__ pre, int pre_mode, int pre_stride, int pre_off, const C* __restrict__ post,
                int post_mode, const C* __restrict__ post2, int post2_mode, double scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  using T = typename real_of<C>::type;
  const int n = p.n;
  const int pitch = n + 1;
  const int l0 = blockIdx.x * lpc;
  const int nl = min(lpc, d.nlines - l0);
  const int E = nl * n;
  auto split = [&](int e, int& li, int& i) {
    if (d.ies == 1) { li = e / n; i = e - li * n; } else { i = e / nl; li = e - i * nl; }
  };
  batched_copy<8>(
      E,
      [&](int e) {
        int li, i;
        split(e, li, i);
        C v = czero<C>();
        if (i < d.n_in) {
          v = in[line_in_off(d, l0 + li) + (long long)i * d.ies];
          if (pre_mode) { C w = pre[i * pre_stride + pre_off]; if (pre_mode == 2) w.y = -w.y; v = cmul(v, w); }
        }
        return v;
      },
      [&](int e, C v) {
        int li, i;
        split(e, li, i);
        s[li * pitch + i] = v;
      });
  __syncthreads();
  SmemLines L{nl, nl, pitch, 0, 1, 0};
  C* res = s;
  if constexpr (MAXE == 0) {
    res = fft_smem_pp(s, s + (size_t)lpc * pitch, p, L, sign);
  } else {
    fft_smem<MAXE>(s, p, L, sign);
  }
  const T sc = (T)scale;
  const int Eo = nl * d.n_out;
  for (int e = threadIdx.x; e < Eo; e += blockDim.x) {
    int li, f;
    if (d.oes == 1) { li = e / d.n_out; f = e - li * d.n_out; } else { f = e / nl; li = e - f * nl; }
    const int l = l0 + li;
    C v = res[li * pitch + f];
    if (post_mode) { C w = post[f]; if (post_mode == 2) w.y = -w.y; v = cmul(v, w); }
    if (post2_mode) { C w = post2[f]; if (post2_mode == 2) w.y = -w.y; v = cmul(v, w); }
    const long long off = line_out_off(d, l) + (long long)f * d.oes;
    out[off] = cscale(v, sc);
  }
}

// Bluestein's chirp-z transform of whole lines in one kernel, when the
// convolution length M fits shared memory: a_i = x_i c_i, FFT_M, times the
// chirp spectrum, inverse FFT_M, times c_f, with c = conj(b) (forward) or b
// (inverse) -- the two launches of the staged transform with the M-point
// intermediate kept in shared memory instead of a global scratch line.
template <class C, int MAXE>
__global__ void __launch_bounds__(MAXE == 0 ? 256 : 1024)
    k_fft_bluestein(const C* __restrict__ in, C* __restrict__ out, LineDesc d, FftPlanDev p, int lpc,
                    const C* __restrict__ chirp, int cmode, const C* __restrict__ hat, double scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  using T = typename real_of<C>::type;
  const int M = p.n;
  const int pitch = M + 1;
  const int l0 = blockIdx.x * lpc;
  const int nl = min(lpc, d.nlines - l0);
  const int E = nl * M;
  auto split = [&](int e, int& li, int& i) {
    if (d.ies == 1) { li = e / M; i = e - li * M; } else { i = e / nl; li = e - i * nl; }
  };
  auto cw = [&](int i) {
    C w = chirp[i];
    if (cmode == 2) w.y = -w.y;
    return w;
  };
  batched_copy<8>(
      E,
      [&](int e) {
        int li, i;
        split(e, li, i);
        C v = czero<C>();
        if (i < d.n_in) v = cmul(in[line_in_off(d, l0 + li) + (long long)i * d.ies], cw(i));
        return v;
      },
      [&](int e, C v) {
        int li, i;
        split(e, li, i);
        s[li * pitch + i] = v;
      });
  __syncthreads();
  SmemLines L{nl, nl, pitch, 0, 1, 0};
  C* res = s;
  if constexpr (MAXE == 0) {
    res = fft_smem_pp(s, s + (size_t)lpc * pitch, p, L, -1);
  } else {
    fft_smem<MAXE>(s, p, L, -1);
  }
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    const int li = e / M, k = e - li * M;
    res[li * pitch + k] = cmul(res[li * pitch + k], hat[k]);
  }
  __syncthreads();
  if constexpr (MAXE == 0) {
    res = fft_smem_pp(res, res == s ? s + (size_t)lpc * pitch : s, p, L, +1);
  } else {
    fft_smem<MAXE>(s, p, L, +1);
  }
  const T sc = (T)scale;
  const int Eo = nl * d.n_out;
  for (int e = threadIdx.x; e < Eo; e += blockDim.x) {
    int li, f;
    if (d.oes == 1) { li = e / d.n_out; f = e - li * d.n_out; } else { f = e / nl; li = e - f * nl; }
    const C v = cmul(res[li * pitch + f], cw(f));
    out[line_out_off(d, l0 + li) + (long long)f * d.oes] = cscale(v, sc);
  }
}

// ---------------------------------------------------------------------------
// Power-of-two lines of n = 32 N1 points (N1 = 8, 16, 32) in complex FP32,
// one warp per G = 32 / N1 lines, the arithmetic in registers.  With input
// i = l + 32 r and output o = k1 + N1 k2,
//   X[k1 + N1 k2] = sum_l W_32^{l k2} W_n^{l k1} sum_r x[l + 32 r] W_N1^{r k1},
// so lane l first transforms its own N1 elements, scales them by W_n^{l k1},
// and after one transpose through shared memory lane (g, k1) transforms the
// 32 values over l.  Both transforms are radix-2 decimation in time.
// ---------------------------------------------------------------------------
template <int N>
__host__ __device__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 1; b < N; b <<= 1) { r = (r << 1) | (i & 1); i >>= 1; }
  return r;
}

// natural-order N-point transform (N <= 32) of v; w32[j] = W_32^j, j < 16
template <int N>
__device__ __forceinline__ void dft_reg(float2 (&v)[N], const float2 (&w32)[16]) {
  float2 a[N];
#pragma unroll
  for (int i = 0; i < N; ++i) a[bitrev<N>(i)] = v[i];
#pragma unroll
  for (int m = 1; m < N; m <<= 1) {
#pragma unroll
    for (int k = 0; k < N; k += 2 * m) {
#pragma unroll
      for (int j = 0; j < m; ++j) {
        const float2 x = a[k + j];
        const float2 b = j == 0 ? a[k + j + m] : cmul(a[k + j + m], w32[j * (16 / m)]);   // W_{2m}^j
        a[k + j] = make_float2(x.x + b.x, x.y + b.y);
        a[k + j + m] = make_float2(x.x - b.x, x.y - b.y);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = a[i];
}

template <int N1>
__global__ void __launch_bounds__(128) k_fft_warp(const float2* __restrict__ in, float2* __restrict__ out, LineDesc d,
                                                  const float2* __restrict__ tw, int sign, float scale) {
  constexpr int G = 32 / N1;
  constexpr int N = 32 * N1;
  __shared__ float2 sm[4][32][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int line0 = (blockIdx.x * 4 + warp) * G;
  if (line0 >= d.nlines) return;   // whole warps only; no block barrier below
  float2 w32[16];   // W_32^j with the transform's sign
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    w32[j] = tw[j * (N / 32)];
    if (sign > 0) w32[j].y = -w32[j].y;
  }
  float2 v[G][N1];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int line = line0 + g;
    const bool ok = line < d.nlines;
    const long long off = ok ? line_in_off(d, line) : 0;
#pragma unroll
    for (int r = 0; r < N1; ++r) {
      const int i = lane + 32 * r;
      v[g][r] = (ok && i < d.n_in) ? in[off + i] : make_float2(0.f, 0.f);
    }
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    dft_reg<N1>(v[g], w32);
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) {   // W_n^{l k1}
      float2 t = tw[lane * k1];
      if (sign > 0) t.y = -t.y;
      v[g][k1] = cmul(v[g][k1], t);
    }
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) sm[warp][g * N1 + k1][lane] = v[g][k1];
  }
  __syncwarp();
  float2 z[32];
#pragma unroll
  for (int l = 0; l < 32; ++l) z[l] = sm[warp][lane][l];
  dft_reg<32>(z, w32);
  const int g = lane / N1, k1 = lane - g * N1;
  const int line = line0 + g;
  if (line < d.nlines) {
    const long long off = line_out_off(d, line);
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      const int o = k1 + N1 * k2;
      if (o < d.n_out) out[off + o] = make_float2(z[k2].x * scale, z[k2].y * scale);
    }
  }
}

static vie_status launch_warp_fft(const float2* in, float2* out, const LineDesc& d, const FftPlanDev& p, int sign,
                                  double scale, cudaStream_t st) {
  const int N1 = p.n / 32, G = 32 / N1;
  const int grid = (d.nlines + 4 * G - 1) / (4 * G);
  Prof pf_("fft_warp_c64", st);
  const float2* tw = (const float2*)p.tw;
  if (N1 == 32) k_fft_warp<32><<<grid, 128, 0, st>>>(in, out, d, tw, sign, (float)scale);
  else if (N1 == 16) k_fft_warp<16><<<grid, 128, 0, st>>>(in, out, d, tw, sign, (float)scale);
  else k_fft_warp<8><<<grid, 128, 0, st>>>(in, out, d, tw, sign, (float)scale);
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

template <class C>
static vie_status launch_lines(const C* in, C* out, const LineDesc& d, const FftPlanDev& p, int sign,
                               const C* pre, int pre_mode, int pre_stride, int pre_off, const C* post, int post_mode,
                               const C* post2, int post2_mode, double scale, cudaStream_t st) {
  const int n = p.n;
  if (n > fft_max_len<C>()) { set_error("fft: line length %d too long for shared memory", n); return VIE_EINVAL; }
  if (d.nlines <= 0) return VIE_OK;
  const size_t line_bytes = (size_t)(n + 1) * sizeof(C);
  const bool pp = 2 * line_bytes <= 200 * 1024;
  const size_t budget = pp ? 24 * 1024 : 48 * 1024;      // per tile copy
  int lpc = (int)(budget / line_bytes);
  if (lpc < 1) lpc = 1;
  if (lpc > d.nlines) lpc = d.nlines;
  if (lpc > 64) lpc = 64;
  const int grid = (d.nlines + lpc - 1) / lpc;
  if (pp) {
    const size_t smem = 2 * (size_t)lpc * line_bytes;
    auto kern = k_fft_lines<C, 0>;
    VIE_TRY(smem_optin(kern, smem));
    Prof pf_(sizeof(C) == 8 ? "fft_lines_c64" : "fft_lines_c128", st);
    kern<<<grid, 256, smem, st>>>(in, out, d, p, sign, lpc, pre, pre_mode, pre_stride, pre_off, post, post_mode,
                                  post2, post2_mode, scale);
    count_launch();
    VIE_CHECK_LAUNCH();
    return VIE_OK;
  }
  const long long E = (long long)lpc * n;
  int threads = 128;
  while (threads < 1024 && E > 8LL * threads) threads *= 2;
  const int per = (int)((E + threads - 1) / threads);
  const size_t smem = (size_t)lpc * line_bytes;
#define VIE_LAUNCH_LINES(ME)                                                                      \
  {                                                                                               \
    auto kern = k_fft_lines<C, ME>;                                                               \
    if (smem > 48 * 1024)                                                                         \
      VIE_TRY(smem_optin(kern, smem));                                                                 \
    Prof pf_(sizeof(C) == 8 ? "fft_lines_c64" : "fft_lines_c128", st);                           \
    kern<<<grid, threads, smem, st>>>(in, out, d, p, sign, lpc, pre, pre_mode, pre_stride, pre_off, \
                                      post, post_mode, post2, post2_mode, scale);                \
  }
  if (per <= 16) VIE_LAUNCH_LINES(16)
  else if (per <= 32) VIE_LAUNCH_LINES(32)
  else { set_error("fft: tile of %lld elements too large", E); return VIE_EINVAL; }
#undef VIE_LAUNCH_LINES
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

template <class C> struct Tabs;
template <> struct Tabs<double2> {
  static const double2* chirp(const FftLen& f) { return f.chirp64; }
  static const double2* hatf(const FftLen& f) { return f.hatf64; }
  static const double2* hati(const FftLen& f) { return f.hati64; }
};
template <> struct Tabs<float2> {
  static const float2* chirp(const FftLen& f) { return f.chirp32; }
  static const float2* hatf(const FftLen& f) { return f.hatf32; }
  static const float2* hati(const FftLen& f) { return f.hati32; }
};

// y[j] = post[j] * scale * (E[j mod n/2] + w^j O[j mod n/2]), w = exp(sign 2 pi i / n):
// the decimation-in-time combination of the two half-length transforms of
// the even- and odd-indexed inputs.
template <class C>
__global__ void k_dit_combine(const C* __restrict__ E, const C* __restrict__ O, C* __restrict__ out, LineDesc d,
                              int n, const C* __restrict__ tw, int sign, const C* __restrict__ post, int post_mode,
                              double scale) {
  using T = typename real_of<C>::type;
  const int n2 = n / 2;
  const long long total = (long long)d.nlines * d.n_out;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(idx / d.n_out), j = (int)(idx - (long long)l * d.n_out);
    const int jh = j < n2 ? j : j - n2;
    C w = tw[j];
    if (sign > 0) w.y = -w.y;
    C v = cadd(E[(long long)l * n2 + jh], cmul(w, O[(long long)l * n2 + jh]));
    if (post_mode) { C q = post[j]; if (post_mode == 2) q.y = -q.y; v = cmul(v, q); }
    out[line_out_off(d, l) + (long long)j * d.oes] = cscale(v, (T)scale);
  }
}

// Transform of length p.n with optional multipliers; lines longer than
// shared memory holds are split once by decimation in time (scratch: nlines
// * p.n elements).
template <class C>
static vie_status launch_len(const C* in, C* out, const LineDesc& d, const FftPlanDev& p, int sign, const C* pre,
                             int pre_mode, const C* post, int post_mode, double scale, C* split_tmp, cudaStream_t st) {
  if (p.n <= fft_max_len<C>())
    return launch_lines<C>(in, out, d, p, sign, pre, pre_mode, 1, 0, post, post_mode, nullptr, 0, scale, st);
  const int n = p.n, n2 = n / 2;
  if (n % 2 || n2 > fft_max_len<C>()) { set_error("fft: length %d too long", n); return VIE_EINVAL; }
  if (!split_tmp) { set_error("fft: length %d needs split scratch", n); return VIE_EINVAL; }
  const FftLen* h;
  VIE_TRY(fft_get(n2, &h));
  const FftPlanDev& ph = plan_n<C>(*h);
  C* E = split_tmp;
  C* O = split_tmp + (size_t)d.nlines * n2;
  // half transforms of the even / odd inputs (their multipliers at indices 2j, 2j + 1)
  LineDesc de = d;
  de.ies = 2 * d.ies;
  de.n_in = (d.n_in + 1) / 2;
  de.n_out = n2;
  de.os1 = n2; de.os2 = (long long)n2 * d.nl1; de.os3 = (long long)n2 * d.nl1 * d.nl2; de.oes = 1;
  VIE_TRY(launch_lines<C>(in, E, de, ph, sign, pre, pre_mode, 2, 0, nullptr, 0, nullptr, 0, 1.0, st));
  LineDesc dod = de;
  dod.n_in = d.n_in / 2;
  VIE_TRY(launch_lines<C>(in + d.ies, O, dod, ph, sign, pre, pre_mode, 2, 1, nullptr, 0, nullptr, 0, 1.0, st));
  const long long total = (long long)d.nlines * d.n_out;
  const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
  k_dit_combine<C><<<grid, 256, 0, st>>>(E, O, out, d, n, (const C*)p.tw, sign, post, post_mode, scale);
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

// One-kernel Bluestein transform of d's lines (M = f.M fits shared memory):
// the tiling of launch_lines for lines of length M.
template <class C>
static vie_status launch_bluestein(const C* in, C* out, const LineDesc& d, const FftLen& f, int sign, double scale,
                                   cudaStream_t st) {
  const FftPlanDev& p = plan_n<C>(f);
  const int M = p.n;
  if (d.nlines <= 0) return VIE_OK;
  const C* chirp = Tabs<C>::chirp(f);
  const C* hat = sign < 0 ? Tabs<C>::hatf(f) : Tabs<C>::hati(f);
  const int cmode = sign < 0 ? 2 : 1;
  const size_t line_bytes = (size_t)(M + 1) * sizeof(C);
  const bool pp = 2 * line_bytes <= 200 * 1024;
  const size_t budget = pp ? 24 * 1024 : 48 * 1024;
  int lpc = (int)(budget / line_bytes);
  if (lpc < 1) lpc = 1;
  if (lpc > d.nlines) lpc = d.nlines;
  if (lpc > 64) lpc = 64;
  const int grid = (d.nlines + lpc - 1) / lpc;
  Prof pf_(sizeof(C) == 8 ? "fft_bluestein_c64" : "fft_bluestein_c128", st);
  if (pp) {
    const size_t smem = 2 * (size_t)lpc * line_bytes;
    auto kern = k_fft_bluestein<C, 0>;
    VIE_TRY(smem_optin(kern, smem));
    kern<<<grid, 256, smem, st>>>(in, out, d, p, lpc, chirp, cmode, hat, scale);
  } else {
    const long long E = (long long)lpc * M;
    int threads = 128;
    while (threads < 1024 && E > 8LL * threads) threads *= 2;
    const int per = (int)((E + threads - 1) / threads);
    const size_t smem = (size_t)lpc * line_bytes;
    if (per <= 16) {
      auto kern = k_fft_bluestein<C, 16>;
      VIE_TRY(smem_optin(kern, smem));
      kern<<<grid, threads, smem, st>>>(in, out, d, p, lpc, chirp, cmode, hat, scale);
    } else if (per <= 32) {
      auto kern = k_fft_bluestein<C, 32>;
      VIE_TRY(smem_optin(kern, smem));
      kern<<<grid, threads, smem, st>>>(in, out, d, p, lpc, chirp, cmode, hat, scale);
    } else {
      set_error("fft: Bluestein tile of %lld elements too large", E);
      return VIE_EINVAL;
    }
  }
  count_launch();
  VIE_CHECK_LAUNCH();
  return VIE_OK;
}

template <class C>
size_t fft_scratch_elems(const FftLen& f, int nlines) {
  // a Bluestein line that fits shared memory runs in one kernel and needs no
  // scratch; a longer one needs its M-point intermediate and the split's
  const size_t len = f.bluestein ? (size_t)f.M : (size_t)f.n;
  if (len <= (size_t)fft_max_len<C>()) return 0;
  return (size_t)nlines * len * (f.bluestein ? 2 : 1);
}
template size_t fft_scratch_elems<float2>(const FftLen&, int);
template size_t fft_scratch_elems<double2>(const FftLen&, int);

template <class C>
vie_status fft_lines(const C* in, C* out, const LineDesc& d, const FftLen& f, int sign, double scale, C* tmp,
                     cudaStream_t st) {
  if (d.n_in > f.n || d.n_out > f.n) { set_error("fft: line desc exceeds length"); return VIE_EINVAL; }
  if (!f.bluestein) {
    // power-of-two complex-FP32 lines of 256..1024 contiguous points: the warp-register transform
    if (sizeof(C) == 8 && d.ies == 1 && d.oes == 1 && (f.n == 256 || f.n == 512 || f.n == 1024))
      return launch_warp_fft((const float2*)in, (float2*)out, d, plan_n<float2>(f), sign, scale, st);
    return launch_len<C>(in, out, d, plan_n<C>(f), sign, nullptr, 0, nullptr, 0, scale, tmp, st);
  }
  if (f.M <= fft_max_len<C>()) return launch_bluestein<C>(in, out, d, f, sign, scale, st);
  if (!tmp) { set_error("fft: Bluestein length %d needs a scratch buffer", f.n); return VIE_EINVAL; }
  C* split = f.M > fft_max_len<C>() ? tmp + (size_t)d.nlines * f.M : nullptr;
  // step 1: a_k = x_k * conj(b_k) (forward) or x_k * b_k (inverse), FFT_M, times chirp spectrum
  LineDesc d1 = d;
  d1.os1 = f.M; d1.os2 = (long long)f.M * d.nl1; d1.os3 = (long long)f.M * d.nl1 * d.nl2;
  d1.oes = 1; d1.n_out = f.M;
  const C* chirp = Tabs<C>::chirp(f);
  const C* hat = sign < 0 ? Tabs<C>::hatf(f) : Tabs<C>::hati(f);
  VIE_TRY(launch_len<C>(in, tmp, d1, plan_n<C>(f), -1, chirp, sign < 0 ? 2 : 1, hat, 1, 1.0, split, st));
  // step 2: inverse FFT_M (the 1/M is in the chirp spectrum), times conj(b_f) or b_f
  LineDesc d2 = d;
  d2.n_in = f.M; d2.is1 = f.M; d2.is2 = (long long)f.M * d.nl1; d2.is3 = (long long)f.M * d.nl1 * d.nl2;
  d2.ies = 1;
  return launch_len<C>(tmp, out, d2, plan_n<C>(f), +1, nullptr, 0, chirp, sign < 0 ? 2 : 1, scale, split, st);
}

template vie_status fft_lines<double2>(const double2*, double2*, const LineDesc&, const FftLen&, int,
                                       double, double2*, cudaStream_t);
template vie_status fft_lines<float2>(const float2*, float2*, const LineDesc&, const FftLen&, int,
                                      double, float2*, cudaStream_t);

}  // namespace vie
