// RCS of a marched current envelope (Sec. 2.4): device helpers of aim_march_spectrum
// and aim_rcs.
#pragma once
#include <complex>

#include "aim_internal.h"

constexpr int kMaxRcsFreq = 64;  // frequencies per call

struct RcsPhases {  // one complex factor per frequency, passed by value
  int n;
  double2 w[kMaxRcsFreq];
};

// That(w) = int T(u) e^{-j w u} du over the basis' support (Eq. 3): 24-point Gauss-Legendre
// per CPPIF piece, or per unit interval of the BLIF's (-M, M)
std::complex<double> basis_spectrum(const TBasis& tb, double w);
// acc[f][b][k] += e^{-j omega_f l dt} x[b][k] (nb right-hand sides of the context's ns)
void rcs_dft_accum(aim_ctx* c, int nb, int l, int n_freq, const double* omega, const double2* x, double2* acc);
// acc[f] *= s.w[f]
void rcs_scale(aim_ctx* c, int nb, const RcsPhases& s, double2* acc);
// sig[f][b][d] from spec[f][b][ns]; dirs [nd][6] (rhat, pol), fk [n_freq][2] (k, prefactor), device
void rcs_farfield(aim_ctx* c, int n_freq, int nb, const double2* spec, int nd, const double* dirs, const double* fk,
                  double* sig);
