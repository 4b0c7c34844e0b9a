// Bistatic RCS of a marched current envelope at chosen frequencies (Sec. 2.4): the
// frequency-domain currents of the march for a unit incident field, and their
// co-polarised far field.
//
//  * envelope convention x(t) = Re{x~(t) e^{j w_c t}}: the spectrum at f > 0 is half the
//    envelope's at Omega = 2 pi (f - f_c), and the half cancels between scattered and
//    incident fields;
//  * the current envelope is the CPPIF interpolant of its samples (Eq. 3), so
//    X~(Omega) = dt That(Omega dt) sum_l I_l e^{-j Omega l dt}, That(w) = int T(u) e^{-j w u} du;
//  * the incident envelope of Eq. 1 at the origin, g(t - t_d) e^{-j w_c t_d}, has the
//    transform E~(Omega) = sigma sqrt(2 pi) exp(-sigma^2 Omega^2 / 2) exp(-j (w_c + Omega) t_d);
//  * X~ / E~ is the frequency-domain current for the unit plane wave p e^{-j k k.r} at f
//    (the time-differentiated EFIE of Eq. 4 at one frequency is the frequency-domain
//    EFIE times j w), whose far field is E = -j w mu/(4 pi) e^{-j k r}/r F with
//    F = (I - r r) . sum_k I_k int S_k(r') e^{+j k r.r'} dS' (7-point cubature), and
//    sigma = 4 pi |pol . E r|^2.
#include <cmath>
#include <complex>
#include <vector>

#include "aim_internal.h"
#include "rcs.h"
#include "setup_host.h"

namespace {

constexpr int kT = 256;

// acc[f][b][k] += w_f x[b][k] for the step's phases w_f = e^{-j Omega_f l dt}
__global__ void __launch_bounds__(kT) k_dft_accum(RcsPhases ph, long long n, const double2* __restrict__ x,
                                                   double2* __restrict__ acc) {
  for (long long i = blockIdx.x * (long long)kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
    const double2 v = x[i];
    for (int f = 0; f < ph.n; ++f) {
      const double2 w = ph.w[f];
      double2& a = acc[(size_t)f * n + i];
      a.x += w.x * v.x - w.y * v.y;
      a.y += w.x * v.y + w.y * v.x;
    }
  }
}

__global__ void __launch_bounds__(kT) k_scale_freq(RcsPhases s, long long n, double2* __restrict__ acc) {
  for (long long i = blockIdx.x * (long long)kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT)
    for (int f = 0; f < s.n; ++f) {
      const double2 w = s.w[f];
      double2& a = acc[(size_t)f * n + i];
      a = make_double2(w.x * a.x - w.y * a.y, w.x * a.y + w.y * a.x);
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One block per (direction d, right-hand side b, frequency f): the radiation vector of
// spec[f][b] summed over every cubature point of every face, then projected.
// dirs: [nd][6] (rhat, pol); fk: [n_freq][2] (k, 4 pi (w mu0 / 4 pi)^2).
__global__ void __launch_bounds__(kT) k_rcs(int nt, const int* __restrict__ tbk, const double* __restrict__ tbs,
                                             const int* __restrict__ tbf, const double* __restrict__ len,
                                             const double* __restrict__ area, const double* __restrict__ V,
                                             const double* __restrict__ qp, const double* __restrict__ qw, int ns,
                                             int nb, const double2* __restrict__ spec, const double* __restrict__ fk,
                                             const double* __restrict__ dirs, int nd, double* __restrict__ sig) {
  const int d = blockIdx.x, b = blockIdx.y, f = blockIdx.z;
  const double* rd = dirs + 6 * d;
  const double rx = rd[0], ry = rd[1], rz = rd[2];
  const double k = fk[2 * f];
  const double2* I = spec + ((size_t)f * nb + b) * ns;
  double a[6] = {0, 0, 0, 0, 0, 0};  // (re, im) of x, y, z
  for (int idx = threadIdx.x; idx < nt * 7; idx += kT) {
    const int t = idx / 7, q = idx % 7;
    const double* r = qp + 21 * t + 3 * q;
    double sn, cs;
    sincos(k * (rx * r[0] + ry * r[1] + rz * r[2]), &sn, &cs);
    const double wq = qw[7 * t + q];
    for (int e = 0; e < 3; ++e) {
      const int kk = tbk[3 * t + e];
      if (kk < 0) continue;
      const double cS = tbs[3 * t + e] * len[kk] / (2.0 * area[t]) * wq;
      const double2 Ik = I[kk];
      const double pr = cS * (Ik.x * cs - Ik.y * sn), pi = cS * (Ik.x * sn + Ik.y * cs);
      const double* vf = V + 3 * tbf[3 * t + e];
      for (int x = 0; x < 3; ++x) {
        const double dx = r[x] - vf[x];
        a[2 * x] += pr * dx;
        a[2 * x + 1] += pi * dx;
      }
    }
  }
  __shared__ double part[kT / 32][6];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = 0; i < 6; ++i) {
    const double s = warp_sum_d(a[i]);
    if (lane == 0) part[warp][i] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int w = 0; w < kT / 32; ++w)
      for (int i = 0; i < 6; ++i) v[i] += part[w][i];
    const double* pol = rd + 3;
    // e = pol . (v - r (r . v)), real and imaginary parts
    const double rvr = rx * v[0] + ry * v[2] + rz * v[4], rvi = rx * v[1] + ry * v[3] + rz * v[5];
    const double er = pol[0] * (v[0] - rx * rvr) + pol[1] * (v[2] - ry * rvr) + pol[2] * (v[4] - rz * rvr);
    const double ei = pol[0] * (v[1] - rx * rvi) + pol[1] * (v[3] - ry * rvi) + pol[2] * (v[5] - rz * rvi);
    sig[((size_t)f * nb + b) * nd + d] = fk[2 * f + 1] * (er * er + ei * ei);
  }
}

int blocks_for(long long n) { return (int)std::min<long long>((n + kT - 1) / kT, 152LL * 16); }

}  // namespace

std::complex<double> basis_spectrum(const TBasis& tb, double w) {
  std::vector<double> x, wt;
  host_gauss_legendre(24, x, wt);
  std::complex<double> s = 0.0;
  if (tb.kind == AIM_BLIF) {  // smooth on (-M, M): 24 points on each unit interval
    for (int j = -tb.Q; j < tb.Q; ++j)
      for (size_t i = 0; i < x.size(); ++i) {
        const double u = j + 0.5 + 0.5 * x[i];
        s += 0.5 * wt[i] * host_blif_value(tb, u) * std::exp(std::complex<double>(0.0, -w * u));
      }
    return s;
  }
  for (int j = 0; j <= tb.Q; ++j) {  // CPPIF piece (j-1, j]
    for (size_t i = 0; i < x.size(); ++i) {
      const double u = j - 0.5 + 0.5 * x[i];
      double T = 0;
      for (int p = tb.Q; p >= 0; --p) T = T * u + tb.coef[j][p];
      s += 0.5 * wt[i] * T * std::exp(std::complex<double>(0.0, -w * u));
    }
  }
  return s;
}

void rcs_dft_accum(aim_ctx* c, int nb, int l, int n_freq, const double* omega, const double2* x, double2* acc) {
  RcsPhases ph{};
  ph.n = n_freq;
  for (int f = 0; f < n_freq; ++f) {
    const double a = -omega[f] * l * c->dt;
    ph.w[f] = make_double2(std::cos(a), std::sin(a));
  }
  const long long n = (long long)nb * c->ns;
  k_dft_accum<<<blocks_for(n), kT, 0, c->stream>>>(ph, n, x, acc);
  AIM_CHECK_LAUNCH();
}

void rcs_scale(aim_ctx* c, int nb, const RcsPhases& s, double2* acc) {
  const long long n = (long long)nb * c->ns;
  k_scale_freq<<<blocks_for(n), kT, 0, c->stream>>>(s, n, acc);
  AIM_CHECK_LAUNCH();
}

void rcs_farfield(aim_ctx* c, int n_freq, int nb, const double2* spec, int nd, const double* dirs, const double* fk,
                  double* sig) {
  k_rcs<<<dim3(nd, nb, n_freq), kT, 0, c->stream>>>(c->nt, c->d_tbk, c->d_tbs, c->d_tbf, c->d_len, c->d_area,
                                                      c->d_v, c->d_qp, c->d_qw, c->ns, nb, spec, fk, dirs, nd, sig);
  AIM_CHECK_LAUNCH();
}
