// Parameter blocks of the setup kernels and the launch helpers shared with operator.cu.
#pragma once
#include <vector>

#include "aim_internal.h"
#include "setup_host.h"

struct TimeK {
  double dt, wc, kc, cdt;
  double cA, cP;  // mu / (4 pi) and 1 / (4 pi eps) of the background medium
  TBasis tb;
};

struct SetupGeom {
  const double* V;
  const int* F;
  const int* rtri;
  const int* rfree;
  const double* len;
  const double* area;
  const double* qp;
  const double* qw;
  const double* cent;
  double mean_edge;
};

struct GaussRule {
  int n;
  double x[8], w[8];
};

void setup_device_tables(aim_ctx* c, HostMesh& hm, const std::vector<int>& anchor);
// full (unpruned) in-place 3-D FFT of an L^3 complex128 array, forward
void fft3d_full_c128(aim_ctx* c, double2* G);
