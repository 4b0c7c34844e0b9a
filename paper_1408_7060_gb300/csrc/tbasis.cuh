// Causal piecewise-polynomial interpolatory temporal basis (CPPIF), Sec. 3 (Eq. 3):
// on the piece (j-1, j], j = 0..Q, T is the Lagrange polynomial through the samples
// n, n-1, ..., n-Q seen from one sample; T and its first three derivatives by Horner.
#pragma once
#include "aim_internal.h"

__device__ __forceinline__ void cppif_eval(const TBasis& tb, double v, double T[4]) {
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

