// Temporal bases of Sec. 3 (Eq. 3), T and its first three derivatives (device and host).
// CPPIF: on the piece (j-1, j], j = 0..Q, T is the Lagrange polynomial through the samples
// n, n-1, ..., n-Q seen from one sample (Horner).  BLIF: the approximate prolate spheroidal
// interpolant sinc(u) w(u) of half-width M (Knab's window), made causal by extrapolating the
// samples it reaches ahead of the test time (Sec. 3.1.2; the weights are set up on the host).
#pragma once
#include "aim_internal.h"

__host__ __device__ __forceinline__ void cppif_eval(const TBasis& tb, double v, double T[4]) {
  T[0] = T[1] = T[2] = T[3] = 0.0;
  double jr = ceil(v);
  if (jr < 0.0 || jr > (double)tb.Q) return;
  const double* c = tb.coef[(int)jr];
  const int Q = tb.Q;
  double p0 = 0, p1 = 0, p2 = 0, p3 = 0;
  for (int p = Q; p >= 0; --p) p0 = p0 * v + c[p];
  for (int p = Q; p >= 1; --p) p1 = p1 * v + p * c[p];
  for (int p = Q; p >= 2; --p) p2 = p2 * v + p * (p - 1) * c[p];
  for (int p = Q; p >= 3; --p) p3 = p3 * v + p * (p - 1) * (p - 2) * c[p];
  T[0] = p0; T[1] = p1; T[2] = p2; T[3] = p3;
}


// f(x) = sin(x)/x and its first three derivatives: below |x| = 1 the Taylor series
// f = sum_n c_n x^(2n), c_n = (-1)^n/(2n+1)!, differentiated term by term (Horner in x^2),
// else the derivatives of sin(x) * x^-1
__host__ __device__ __forceinline__ void sinc_derivs(double x, double f[4]) {
  if (fabs(x) < 1.0) {
    double c[12];
    double fct = 1.0;
    for (int n = 0; n < 12; ++n) {
      c[n] = (n & 1) ? -fct : fct;
      fct /= (2.0 * n + 2.0) * (2.0 * n + 3.0);
    }
    const double x2 = x * x;
    double h0 = 0.0, h1 = 0.0, h2 = 0.0, h3 = 0.0;
    for (int n = 11; n >= 0; --n) {
      const double a = 2.0 * n;
      h0 = h0 * x2 + c[n];
      if (n >= 1) {
        h1 = h1 * x2 + c[n] * a;
        h2 = h2 * x2 + c[n] * a * (a - 1.0);
      }
      if (n >= 2) h3 = h3 * x2 + c[n] * a * (a - 1.0) * (a - 2.0);
    }
    f[0] = h0;
    f[1] = x * h1;
    f[2] = h2;
    f[3] = x * h3;
    return;
  }
  double sn, cs;
  sincos(x, &sn, &cs);
  const double i1 = 1.0 / x, i2 = i1 * i1, i3 = i2 * i1, i4 = i2 * i2;
  f[0] = sn * i1;
  f[1] = cs * i1 - sn * i2;
  f[2] = -sn * i1 - 2.0 * cs * i2 + 2.0 * sn * i3;
  f[3] = -cs * i1 + 3.0 * sn * i2 + 6.0 * cs * i3 - 6.0 * sn * i4;
}

// r_k(x) = i_k(x) / x^k, k = 0..3 (i_k the modified spherical Bessel functions), so that
// G(s) = sinh(b sqrt s)/sqrt s has G^(k)(s) = b^(2k+1) r_k(b sqrt s) / 2^k
__host__ __device__ __forceinline__ void sph_in_ratio(double x, double r[4]) {
  if (x < 4.0) {
    // r_k = sum_j (x^2/2)^j / (j! (2k+2j+1)!!), positive terms
    const double h = 0.5 * x * x;
    double dfact = 1.0;  // (2k+1)!!
    for (int k = 0; k < 4; ++k) {
      dfact *= (k == 0) ? 1.0 : (2.0 * k + 1.0);
      double term = 1.0 / dfact, sum = term;
      for (int j = 1; j <= 24; ++j) {
        term *= h / ((double)j * (2.0 * k + 2.0 * j + 1.0));
        sum += term;
      }
      r[k] = sum;
    }
    return;
  }
  const double sh = sinh(x), ch = cosh(x), x2 = x * x;
  r[0] = sh / x;
  r[1] = (x * ch - sh) / (x2 * x);
  r[2] = ((x2 + 3.0) * sh - 3.0 * x * ch) / (x2 * x2 * x);
  r[3] = ((x2 * x + 15.0 * x) * ch - (6.0 * x2 + 15.0) * sh) / (x2 * x2 * x2 * x);
}

// the BLIF T(u) = sinc(u) w(u) on |u| < M and its first three derivatives (product rule;
// w through s = M^2 - u^2: w' = -2u G', w'' = 4u^2 G'' - 2G', w''' = -8u^3 G''' + 12u G'')
__host__ __device__ __forceinline__ void blif_eval(const TBasis& tb, double u, double T[4]) {
  T[0] = T[1] = T[2] = T[3] = 0.0;
  const double M = (double)tb.Q;
  if (!(fabs(u) < M)) return;
  const double pi = aimc::kPi;
  double f[4];
  sinc_derivs(pi * u, f);
  const double S0 = f[0], S1 = pi * f[1], S2 = pi * pi * f[2], S3 = pi * pi * pi * f[3];
  double r[4];
  sph_in_ratio(tb.b * sqrt(M * M - u * u), r);
  const double b = tb.b, b3 = b * b * b, b5 = b3 * b * b, b7 = b5 * b * b;
  const double G0 = b * r[0], G1 = b3 * r[1] * 0.5, G2 = b5 * r[2] * 0.25, G3 = b7 * r[3] * 0.125;
  const double w0 = G0 * tb.invG0;
  const double w1 = -2.0 * u * G1 * tb.invG0;
  const double w2 = (4.0 * u * u * G2 - 2.0 * G1) * tb.invG0;
  const double w3 = (-8.0 * u * u * u * G3 + 12.0 * u * G2) * tb.invG0;
  T[0] = S0 * w0;
  T[1] = S1 * w0 + S0 * w1;
  T[2] = S2 * w0 + 2.0 * S1 * w1 + S0 * w2;
  T[3] = S3 * w0 + 3.0 * S2 * w1 + 3.0 * S1 * w2 + S0 * w3;
}

// The time factor of delay m at x = R/(c dt): T(m - x) for the CPPIF; for the BLIF
// T(m - x) plus, for m < M, the extrapolated samples sum_p ext[p][m] T(-p - x).
__host__ __device__ __forceinline__ void tb_eval(const TBasis& tb, int m, double x, double T[4]) {
  if (tb.kind == AIM_CPPIF) {
    cppif_eval(tb, (double)m - x, T);
    return;
  }
  blif_eval(tb, (double)m - x, T);
  if (m < tb.Q) {
    for (int p = 1; p < tb.Q; ++p) {
      double Tp[4];
      blif_eval(tb, -(double)p - x, Tp);
      const double e = tb.ext[p][m];
      for (int i = 0; i < 4; ++i) T[i] += e * Tp[i];
    }
  }
}
