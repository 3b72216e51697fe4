// Green's-tensor generator entries of the voxel JVIE operator (FP64), shared
// by the spectra assembly and the preconditioner's Chan coefficients.
//
// G^{ab}(d), d != 0 (one-point rule, R = h|d|, r = d/|d|, V = h^3):
//   V g(R) [ (k^2 - (1+jkR)/R^2) delta_ab + (3 + 3jkR - k^2R^2)/R^2 r_a r_b ],
//   g(R) = exp(-jkR)/(4 pi R);
// G^{aa}(0) = -1/3 + (2/3)((1 + jka) exp(-jka) - 1), a = (3V/(4 pi))^(1/3)
// (field at the centre of the equal-volume sphere).  Pairs c = 0..5 are
// xx, xy, xz, yy, yz, zz.
#pragma once

#include <math.h>

#include "vie_common.cuh"

namespace vie {

__host__ __device__ inline double2 self_term_value(double h, double k) {
  const double V = h * h * h;
  const double a = cbrt(3.0 * V / (4.0 * M_PI));
  const double x = k * a;
  double s, c;
  sincos(x, &s, &c);
  // (1 + jx) e^{-jx} = cos x + x sin x + j (x cos x - sin x)
  const double re = c + x * s, im = x * c - s;
  return make_double2(-1.0 / 3.0 + (2.0 / 3.0) * (re - 1.0), (2.0 / 3.0) * im);
}

__device__ __forceinline__ void pair_of(int c, int& a, int& b) {
  // xx xy xz yy yz zz
  const int A[6] = {0, 0, 0, 1, 1, 2};
  const int B[6] = {0, 1, 2, 1, 2, 2};
  a = A[c];
  b = B[c];
}

__device__ __forceinline__ double2 gen_entry(int c, int dx, int dy, int dz, double h, double k, double2 self) {
  int a, b;
  pair_of(c, a, b);
  if (dx == 0 && dy == 0 && dz == 0) return a == b ? self : make_double2(0.0, 0.0);
  const double d2 = (double)dx * dx + (double)dy * dy + (double)dz * dz;
  const double dist = sqrt(d2);
  const double R = h * dist;
  const double V = h * h * h;
  const double kR = k * R;
  double sn, cs;
  sincos(kR, &sn, &cs);
  const double inv4piR = V / (4.0 * M_PI * R);
  const double gr = cs * inv4piR, gi = -sn * inv4piR;       // V g
  const double iR2 = 1.0 / (R * R);
  const double d[3] = {(double)dx / dist, (double)dy / dist, (double)dz / dist};
  const double rr = d[a] * d[b];
  double vr = (3.0 - kR * kR) * iR2 * rr;
  double vi = 3.0 * kR * iR2 * rr;
  if (a == b) {
    vr += k * k - iR2;
    vi += -kR * iR2;
  }
  return make_double2(gr * vr - gi * vi, gr * vi + gi * vr);
}

}  // namespace vie
