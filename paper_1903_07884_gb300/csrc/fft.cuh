// Mixed-radix Stockham FFT in shared memory (radices 2, 3, 4, 5, 7, 8).
//
// One pass with radix R and current span Ns combines R sub-transforms of
// length Ns into one of length Ns*R: butterfly j (0 <= j < n/R) reads
// x[j + r n/R], multiplies by exp(sign 2 pi i (j mod Ns) r / (Ns R)), takes an
// R-point DFT and writes y[(j/Ns) Ns R + (j mod Ns) + q Ns].  Passes run in
// place: every thread loads all of its butterflies into registers, the block
// synchronises, then stores (every element is read and written exactly once
// per pass).  Forward transforms use sign -1 (F_{fk} = exp(-2 pi i f k / n)),
// inverse transforms sign +1 without the 1/n factor.
#pragma once

#include "vie_common.cuh"

namespace vie {

constexpr int FFT_MAX_PASSES = 16;

// Exact quotient t / d for 0 <= t, t * d < 2^32 by one high multiply with
// m = ceil(2^32 / d) (m = 0 encodes d = 1).
struct FastDiv {
  unsigned d, m;
};
// m = ceil(2^32 / d) = floor((2^32 - 1) / d) + 1 for d >= 2, in 32-bit
// arithmetic: a 64-bit division would run as an FP64 subroutine on the device,
// and FP64 issues at a small fraction of the FP32 rate on this part
__host__ __device__ inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f;
  f.d = d;
  f.m = d <= 1 ? 0u : 0xFFFFFFFFu / d + 1u;
  return f;
}
__device__ __forceinline__ unsigned fdiv(unsigned t, FastDiv f) { return f.m ? __umulhi(t, f.m) : t; }

// Device-side description of one transform length.
struct FftPlanDev {
  int n;
  int npass;
  int radix[FFT_MAX_PASSES];
  const void* tw;   // n twiddles exp(-2 pi i k / n) in the kernel's complex type
  // per pass: span Ns before the pass, its fast divisor, butterflies per line
  // n/R and twiddle stride n/(Ns R)
  int ns[FFT_MAX_PASSES];
  FastDiv ns_div[FFT_MAX_PASSES];
  FastDiv nb_div[FFT_MAX_PASSES];
  int tws[FFT_MAX_PASSES];
};

// Fill the per-pass fields from n and the radix list.
inline void fft_plan_finalize(FftPlanDev& p) {
  int Ns = 1;
  for (int i = 0; i < p.npass; ++i) {
    const int R = p.radix[i];
    p.ns[i] = Ns;
    p.ns_div[i] = make_fastdiv((unsigned)Ns);
    p.nb_div[i] = make_fastdiv((unsigned)(p.n / R));
    p.tws[i] = p.n / (Ns * R);
    Ns *= R;
  }
}

// Element-wise copy of E items by the block, U items per thread at a time:
// the U loads (load(e), global memory) are all issued before the first store
// (store(e, v), usually shared memory), so a thread keeps U requests in flight
// instead of waiting out the memory latency once per item.
template <int U, class F, class G>
__device__ __forceinline__ void batched_copy(int E, F load, G store) {
  using V = decltype(load(0));
  for (int e0 = threadIdx.x; e0 < E; e0 += U * blockDim.x) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < E) v[u] = load(e);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < E) store(e, v[u]);
    }
  }
}

// Lines in shared memory: line l = l1 + nl1 * l2 (l1 < nl1) starts at
// l1*ls1 + l2*ls2 and holds element i at offset i*es.
struct SmemLines {
  int nlines, nl1, ls1, ls2, es;
  int line_fast;    // thread mapping: 1 = consecutive threads walk lines
};

// cos/sin(2 pi q / R) for R = 3, 5, 7 (elementary values).
template <int R> struct RootTab;
template <> struct RootTab<3> {
  static __device__ __forceinline__ double c(int q) { return q == 0 ? 1.0 : -0.5; }
  static __device__ __forceinline__ double s(int q) {
    return q == 0 ? 0.0 : (q == 1 ? 0.86602540378443864676 : -0.86602540378443864676);
  }
};
template <> struct RootTab<5> {
  static __device__ __forceinline__ double c(int q) {
    switch (q) { case 0: return 1.0; case 1: case 4: return 0.30901699437494742410;
                 default: return -0.80901699437494742410; }
  }
  static __device__ __forceinline__ double s(int q) {
    switch (q) { case 0: return 0.0; case 1: return 0.95105651629515357212;
                 case 2: return 0.58778525229247312917; case 3: return -0.58778525229247312917;
                 default: return -0.95105651629515357212; }
  }
};
template <> struct RootTab<7> {
  static __device__ __forceinline__ double c(int q) {
    switch (q) { case 0: return 1.0; case 1: case 6: return 0.62348980185873353053;
                 case 2: case 5: return -0.22252093395631440429;
                 default: return -0.90096886790241912624; }
  }
  static __device__ __forceinline__ double s(int q) {
    switch (q) { case 0: return 0.0; case 1: return 0.78183148246802980871;
                 case 2: return 0.97492791218182360702; case 3: return 0.43388373911755812048;
                 case 4: return -0.43388373911755812048; case 5: return -0.97492791218182360702;
                 default: return -0.78183148246802980871; }
  }
};

// multiply by (sign * i)
template <class C> __device__ __forceinline__ C mul_si(C a, int sign) {
  return sign < 0 ? cmake<C>(a.y, -a.x) : cmake<C>(-a.y, a.x);
}

template <int R, class C> struct Dft;

template <class C> struct Dft<2, C> {
  static __device__ __forceinline__ void run(C* v, int) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
  }
};
template <class C> struct Dft<4, C> {
  static __device__ __forceinline__ void run(C* v, int sign) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = mul_si(csub(v[1], v[3]), sign);
    v[0] = cadd(t0, t2); v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3); v[3] = csub(t1, t3);
  }
};
template <class C> struct Dft<8, C> {
  static __device__ __forceinline__ void run(C* v, int sign) {
    using T = typename real_of<C>::type;
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, C>::run(e, sign);
    Dft<4, C>::run(o, sign);
    const T h = (T)0.70710678118654752440;
    // w8^q for q = 1, 2, 3 with w8 = exp(sign i pi / 4)
    C o1 = cmake<C>(h * (o[1].x - sign * o[1].y), h * (o[1].y + sign * o[1].x));
    C o2 = mul_si(o[2], sign);
    C o3 = cmake<C>(h * (-o[3].x - sign * o[3].y), h * (-o[3].y + sign * o[3].x));
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
  }
};
template <int R, class C> struct DftOdd {
  static __device__ __forceinline__ void run(C* v, int sign) {
    using T = typename real_of<C>::type;
    C out[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      C acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const int e = (r * q) % R;
        const T c = (T)RootTab<R>::c(e), s = (T)(sign * RootTab<R>::s(e));
        acc.x += v[r].x * c - v[r].y * s;
        acc.y += v[r].x * s + v[r].y * c;
      }
      out[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = out[q];
  }
};
template <class C> struct Dft<3, C> : DftOdd<3, C> {};
template <class C> struct Dft<5, C> : DftOdd<5, C> {};
template <class C> struct Dft<7, C> : DftOdd<7, C> {};

template <class C>
__device__ __forceinline__ int sl_offset(const SmemLines& L, FastDiv nl1, int line) {
  const int l2 = (int)fdiv((unsigned)line, nl1);
  const int l1 = line - l2 * L.nl1;
  return l1 * L.ls1 + l2 * L.ls2;
}

// One radix-R pass over all lines.  MAXE bounds the elements a thread holds:
// the caller guarantees n * nlines <= MAXE * blockDim.x.
template <int R, int MAXE, class C>
__device__ __forceinline__ void fft_pass(C* s, const FftPlanDev& p, int ps, const SmemLines& L, FastDiv nl1,
                                         FastDiv nlines, const C* __restrict__ tw, int sign) {
  constexpr int MB = (MAXE + R - 1) / R;
  const int n = p.n;
  const int nb = n / R;
  const int total = nb * L.nlines;
  const int Ns = p.ns[ps];
  const FastDiv nsd = p.ns_div[ps], nbd = p.nb_div[ps];
  const int tws = p.tws[ps];
  C v[MB][R];
#pragma unroll
  for (int b = 0; b < MB; ++b) {
    const int t = threadIdx.x + b * blockDim.x;
    if (t < total) {
      int line, j;
      if (L.line_fast) { j = (int)fdiv((unsigned)t, nlines); line = t - j * L.nlines; }
      else { line = (int)fdiv((unsigned)t, nbd); j = t - line * nb; }
      const C* base = s + sl_offset<C>(L, nl1, line);
      const int k = j - (int)fdiv((unsigned)j, nsd) * Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = base[(j + r * nb) * L.es];
      if (Ns > 1) {
        if (sizeof(C) == 8) {
          // FP32: powers of one table twiddle (a few ulp, below the FFT's own error)
          C w1 = tw[k * tws];
          if (sign > 0) w1.y = -w1.y;
          C wr = w1;
#pragma unroll
          for (int r = 1; r < R; ++r) {
            v[b][r] = cmul(v[b][r], wr);
            if (r + 1 < R) wr = cmul(wr, w1);
          }
        } else {
#pragma unroll
          for (int r = 1; r < R; ++r) {
            C w = tw[k * r * tws];
            if (sign > 0) w.y = -w.y;
            v[b][r] = cmul(v[b][r], w);
          }
        }
      }
      Dft<R, C>::run(v[b], sign);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < MB; ++b) {
    const int t = threadIdx.x + b * blockDim.x;
    if (t < total) {
      int line, j;
      if (L.line_fast) { j = (int)fdiv((unsigned)t, nlines); line = t - j * L.nlines; }
      else { line = (int)fdiv((unsigned)t, nbd); j = t - line * nb; }
      C* base = s + sl_offset<C>(L, nl1, line);
      const int jq = (int)fdiv((unsigned)j, nsd);
      const int k = j - jq * Ns;
      const int o = jq * Ns * R + k;
#pragma unroll
      for (int q = 0; q < R; ++q) base[(o + q * Ns) * L.es] = v[b][q];
    }
  }
  __syncthreads();
}

// Transform every line in shared memory (sign -1 forward, +1 inverse).
template <int MAXE, class C>
__device__ __forceinline__ void fft_smem(C* s, const FftPlanDev& p, const SmemLines& L, int sign) {
  const C* tw = (const C*)p.tw;
  const FastDiv nl1 = make_fastdiv((unsigned)L.nl1);
  const FastDiv nlines = make_fastdiv((unsigned)L.nlines);
  for (int ps = 0; ps < p.npass; ++ps) {
    switch (p.radix[ps]) {
      case 8: fft_pass<8, MAXE>(s, p, ps, L, nl1, nlines, tw, sign); break;
      case 4: fft_pass<4, MAXE>(s, p, ps, L, nl1, nlines, tw, sign); break;
      case 2: fft_pass<2, MAXE>(s, p, ps, L, nl1, nlines, tw, sign); break;
      case 3: fft_pass<3, MAXE>(s, p, ps, L, nl1, nlines, tw, sign); break;
      case 5: fft_pass<5, MAXE>(s, p, ps, L, nl1, nlines, tw, sign); break;
      default: fft_pass<7, MAXE>(s, p, ps, L, nl1, nlines, tw, sign); break;
    }
  }
}

// ---------------------------------------------------------------------------
// Out-of-place (ping-pong) passes: each butterfly reads its R inputs from one
// shared buffer and writes its R outputs to the other, so a thread holds one
// butterfly at a time and every pass needs a single barrier.  Used whenever
// two copies of the tile fit in shared memory.
// ---------------------------------------------------------------------------
template <int R, class C>
__device__ __forceinline__ void fft_pass_pp(const C* __restrict__ in, C* __restrict__ out, const FftPlanDev& p,
                                            int ps, const SmemLines& L, FastDiv nl1, FastDiv nlines,
                                            const C* __restrict__ tw, int sign) {
  const int n = p.n;
  const int nb = n / R;
  const int total = nb * L.nlines;
  const int Ns = p.ns[ps];
  const FastDiv nsd = p.ns_div[ps], nbd = p.nb_div[ps];
  const int tws = p.tws[ps];
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int line, j;
    if (L.line_fast) { j = (int)fdiv((unsigned)t, nlines); line = t - j * L.nlines; }
    else { line = (int)fdiv((unsigned)t, nbd); j = t - line * nb; }
    const int off = sl_offset<C>(L, nl1, line);
    const int jq = (int)fdiv((unsigned)j, nsd);
    const int k = j - jq * Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[off + (j + r * nb) * L.es];
    if (Ns > 1) {
      if (sizeof(C) == 8) {
        C w1 = tw[k * tws];
        if (sign > 0) w1.y = -w1.y;
        C wr = w1;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          v[r] = cmul(v[r], wr);
          if (r + 1 < R) wr = cmul(wr, w1);
        }
      } else {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = tw[k * r * tws];
          if (sign > 0) w.y = -w.y;
          v[r] = cmul(v[r], w);
        }
      }
    }
    Dft<R, C>::run(v, sign);
    const int o = jq * Ns * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) out[off + (o + q * Ns) * L.es] = v[q];
  }
}

// Transform every line; the data start in buffer a and end in the returned
// buffer (a or b, same layout).  Ends with a barrier.
template <class C>
__device__ __forceinline__ C* fft_smem_pp(C* a, C* b, const FftPlanDev& p, const SmemLines& L, int sign) {
  const C* tw = (const C*)p.tw;
  const FastDiv nl1 = make_fastdiv((unsigned)L.nl1);
  const FastDiv nlines = make_fastdiv((unsigned)L.nlines);
  C* in = a;
  C* out = b;
  for (int ps = 0; ps < p.npass; ++ps) {
    switch (p.radix[ps]) {
      case 8: fft_pass_pp<8>(in, out, p, ps, L, nl1, nlines, tw, sign); break;
      case 4: fft_pass_pp<4>(in, out, p, ps, L, nl1, nlines, tw, sign); break;
      case 2: fft_pass_pp<2>(in, out, p, ps, L, nl1, nlines, tw, sign); break;
      case 3: fft_pass_pp<3>(in, out, p, ps, L, nl1, nlines, tw, sign); break;
      case 5: fft_pass_pp<5>(in, out, p, ps, L, nl1, nlines, tw, sign); break;
      default: fft_pass_pp<7>(in, out, p, ps, L, nl1, nlines, tw, sign); break;
    }
    __syncthreads();
    C* t = in;
    in = out;
    out = t;
  }
  return in;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// Is n a product of 2, 3, 5, 7?
bool fft_smooth(int n);
// Smallest 7-smooth integer >= n.
int fft_next_smooth(int n);
// Radix sequence of a 7-smooth length (fills p.n, p.npass, p.radix; the
// caller runs fft_plan_finalize); false if n is not 7-smooth or needs more
// than FFT_MAX_PASSES passes.
bool fft_factorize(int n, FftPlanDev& p);

// One transform length with its twiddle tables (or a Bluestein chirp-z
// decomposition through a smooth length M >= 2n - 1 when n is not smooth).
struct FftLen {
  int n = 0;
  bool bluestein = false;
  int M = 0;
  FftPlanDev pn64{}, pn32{};       // plans for n (smooth case)
  FftPlanDev pm64{}, pm32{};       // plans for M (Bluestein case)
  // Bluestein tables: chirp b_k = exp(i pi k^2 / n) (k < n) and the scaled
  // spectra of the wrapped chirp for the forward and inverse transforms.
  double2* chirp64 = nullptr; float2* chirp32 = nullptr;
  double2* hatf64 = nullptr;  float2* hatf32 = nullptr;
  double2* hati64 = nullptr;  float2* hati32 = nullptr;
};

// Per-process cache of transform lengths (device memory lives until exit).
vie_status fft_get(int n, const FftLen** out);

// Description of a batch of lines in global memory: line l = l1 + nl1*(l2 +
// nl2*l3) has input element i at l1*is1 + l2*is2 + l3*is3 + i*ies and output
// element f at l1*os1 + l2*os2 + l3*os3 + f*oes.
struct LineDesc {
  int n_in;            // input elements per line (zero-padded to the length)
  int n_out;           // output elements per line
  int nlines;
  int nl1, nl2;
  long long is1, is2, is3, ies;
  long long os1, os2, os3, oes;
};

__host__ __device__ __forceinline__ long long line_in_off(const LineDesc& d, int l) {
  const int l1 = l % d.nl1, r = l / d.nl1;
  const int l2 = r % d.nl2, l3 = r / d.nl2;
  return (long long)l1 * d.is1 + (long long)l2 * d.is2 + (long long)l3 * d.is3;
}
__host__ __device__ __forceinline__ long long line_out_off(const LineDesc& d, int l) {
  const int l1 = l % d.nl1, r = l / d.nl1;
  const int l2 = r % d.nl2, l3 = r / d.nl2;
  return (long long)l1 * d.os1 + (long long)l2 * d.os2 + (long long)l3 * d.os3;
}

// Lines with one level of indexing: line l at l*is (input) and l*os (output).
inline LineDesc lines_flat(int n_in, int n_out, int nlines, long long is, long long ies, long long os,
                           long long oes) {
  LineDesc d{n_in, n_out, nlines, nlines, 1, is, 0, 0, ies, os, 0, 0, oes};
  return d;
}

// Batched FFT of lines through shared memory, any supported length (smooth
// lengths directly; others by Bluestein; lines longer than shared memory by
// one decimation-in-time split).  `tmp` must hold fft_scratch_elems<C>(f,
// nlines) elements when that is non-zero.  sign -1 forward, +1 inverse
// (unnormalised); `scale` multiplies every output.  Out-of-place or in place
// when input and output footprints coincide.
template <class C>
vie_status fft_lines(const C* in, C* out, const LineDesc& d, const FftLen& f, int sign,
                     double scale, C* tmp, cudaStream_t st);

// Largest line length that fft_lines can hold in shared memory for type C
// (longer even lengths, up to twice this, are split once).
template <class C> int fft_max_len();

// Scratch elements (of type C) that fft_lines needs for nlines lines of this
// transform length: Bluestein buffer and/or the split of an over-long line.
template <class C> size_t fft_scratch_elems(const FftLen& f, int nlines);

void count_launch(int n = 1);

}  // namespace vie
