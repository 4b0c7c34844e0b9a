// Excitation from envelope samples, far-field envelopes, and their adjoints: the
// pieces that turn the march of Eq. 5 into a differentiable map from incident-envelope
// samples to a far-field objective.  (The paper has no adjoint; these operators are
// the linear maps around its march.)
//
//  * incident envelope e(tau) = sum_i a_i T(tau/dt - i) (the CPPIF of Eq. 3 as the
//    interpolant of the samples a_i), plane wave p e(t - r.k/c) e^{-j k_c r.k}; tested
//    as in Eq. 4:  V_l[k] = sum_i a_i <S_k, p (DT)(l - i - r.k/(c dt)) e^{-j k_c r.k}>,
//    (DT)(u) = T'(u)/dt + j w_c T(u);
//  * far-field envelope in direction r, transverse unit vectors e_1, e_2:
//    F_q(n) = -mu/(4 pi) sum_l sum_k I_l[k] int S_k.e_q (DT)(n - l + r.r'/(c dt))
//             e^{+j k_c r.r'} dS'.
// Every sum runs over the Cowper 7-point cubature of the two triangles of each RWG;
// for each cubature point only the Q+1 time indices inside the support of T
// contribute, so no tap table is stored.
#include <algorithm>
#include <cmath>
#include <vector>

#include "aim_internal.h"
#include "tbasis.cuh"

namespace {

constexpr int kT = 256;

struct WaveArgs {
  double kx, ky, kz, px, py, pz;
};

struct DirArgs {
  int nd;
  const double* r;   // [nd][3]
  const double* e1;  // [nd][3]
  const double* e2;  // [nd][3]
};

struct MeshArgs {
  const int* rtri;
  const int* rfree;
  const double* len;
  const double* area;
  const double* V;
  const double* qp;
  const double* qw;
  int ns;
  double dt, wc, kc, cdt;
  double mu;  // permeability of the background medium
  TBasis tb;
};

__device__ __forceinline__ double2 dt_basis(const MeshArgs& m, double v) {  // (DT)(v)
  double T[4];
  cppif_eval(m.tb, v, T);
  return make_double2(T[1] / m.dt, m.wc * T[0]);
}

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmc(double2 a, double2 b) {  // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// V_l[k], l = l0..l0+n_steps-1 into out[l - l0] (thread per (l, k))
__global__ void __launch_bounds__(kT) k_exc_samples(MeshArgs m, WaveArgs w, int i0, int n_samp,
                                                    const double2* __restrict__ a, int l0, int n_steps,
                                                    double2* __restrict__ out) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n_steps * m.ns) return;
  const int l = (int)(idx / m.ns) + l0, k = (int)(idx % m.ns);
  double2 acc = make_double2(0, 0);
  for (int side = 0; side < 2; ++side) {
    const int t = m.rtri[2 * k + side];
    const double* vf = m.V + 3 * m.rfree[2 * k + side];
    const double cS = (side == 0 ? 1.0 : -1.0) * m.len[k] / (2.0 * m.area[t]);
    for (int q = 0; q < 7; ++q) {
      const double* r = m.qp + 21 * t + 3 * q;
      const double rk = r[0] * w.kx + r[1] * w.ky + r[2] * w.kz;
      const double u = rk / m.cdt;
      double s, c;
      sincos(-m.kc * rk, &s, &c);
      const double sp = cS * ((r[0] - vf[0]) * w.px + (r[1] - vf[1]) * w.py + (r[2] - vf[2]) * w.pz);
      const double wt = m.qw[7 * t + q] * sp;
      const int ilo = max(i0, (int)floor(l - u - m.tb.Q)), ihi = min(i0 + n_samp - 1, (int)ceil(l - u + 1));
      double2 sum = make_double2(0, 0);
      for (int i = ilo; i <= ihi; ++i) {
        const double2 f = dt_basis(m, l - i - u);
        const double2 p = cm(f, a[i - i0]);
        sum.x += p.x;
        sum.y += p.y;
      }
      const double2 e = cm(sum, make_double2(c, s));
      acc.x += wt * e.x;
      acc.y += wt * e.y;
    }
  }
  out[(size_t)(l - l0) * m.ns + k] = acc;
}

template <class T>
__device__ __forceinline__ T wsum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double2 block_sum(double2 v) {
  __shared__ double red[2][kT / 32];
  v.x = wsum(v.x);
  v.y = wsum(v.y);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = v.x;
    red[1][threadIdx.x >> 5] = v.y;
  }
  __syncthreads();
  double2 s = make_double2(0, 0);
  if (threadIdx.x == 0)
    for (int q = 0; q < kT / 32; ++q) {
      s.x += red[0][q];
      s.y += red[1][q];
    }
  __syncthreads();
  return s;
}

// grad_i (+)= sum_l sum_k conj(B_{l-i}[k]) lam_l[k] over l = l0..l0+n_steps-1, lam_l =
// lam[l - l0] (or its conjugate with conj_lam); block per sample i = i0 + blockIdx.x
__global__ void __launch_bounds__(kT) k_exc_samples_adj(MeshArgs m, WaveArgs w, int i0, int l0, int n_steps,
                                                        const double2* __restrict__ lam, int conj_lam, int accumulate,
                                                        double2* __restrict__ grad) {
  const int i = i0 + blockIdx.x;
  double2 acc = make_double2(0, 0);
  for (int k = threadIdx.x; k < m.ns; k += blockDim.x) {
    for (int side = 0; side < 2; ++side) {
      const int t = m.rtri[2 * k + side];
      const double* vf = m.V + 3 * m.rfree[2 * k + side];
      const double cS = (side == 0 ? 1.0 : -1.0) * m.len[k] / (2.0 * m.area[t]);
      for (int q = 0; q < 7; ++q) {
        const double* r = m.qp + 21 * t + 3 * q;
        const double rk = r[0] * w.kx + r[1] * w.ky + r[2] * w.kz;
        const double u = rk / m.cdt;
        double s, c;
        sincos(-m.kc * rk, &s, &c);
        const double sp = cS * ((r[0] - vf[0]) * w.px + (r[1] - vf[1]) * w.py + (r[2] - vf[2]) * w.pz);
        const double wt = m.qw[7 * t + q] * sp;
        const int llo = max(l0, (int)floor(i + u - 1)), lhi = min(l0 + n_steps - 1, (int)ceil(i + u + m.tb.Q));
        for (int l = llo; l <= lhi; ++l) {
          const double2 f = cm(dt_basis(m, l - i - u), make_double2(c, s));
          double2 lv = lam[(size_t)(l - l0) * m.ns + k];
          if (conj_lam) lv.y = -lv.y;
          const double2 p = cmc(f, lv);
          acc.x += wt * p.x;
          acc.y += wt * p.y;
        }
      }
    }
  }
  const double2 sum = block_sum(acc);
  if (threadIdx.x == 0) {
    if (accumulate) {
      grad[blockIdx.x].x += sum.x;
      grad[blockIdx.x].y += sum.y;
    } else {
      grad[blockIdx.x] = sum;
    }
  }
}

// F[n - n0][d][q] (+)= the contribution of I_l, l = l0..l0+n_steps-1 (I_l = I[l - l0]), for
// n = n1..n1+gridDim.x/nd-1 (block per (n, d))
__global__ void __launch_bounds__(kT) k_farfield(MeshArgs m, DirArgs d, int l0, int n_steps,
                                                 const double2* __restrict__ I, int n0, int n1, int accumulate,
                                                 double2* __restrict__ F) {
  const int n = n1 + blockIdx.x / d.nd, di = blockIdx.x % d.nd;
  const double* rh = d.r + 3 * di;
  const double* e1 = d.e1 + 3 * di;
  const double* e2 = d.e2 + 3 * di;
  double2 a1 = make_double2(0, 0), a2 = make_double2(0, 0);
  for (int k = threadIdx.x; k < m.ns; k += blockDim.x) {
    for (int side = 0; side < 2; ++side) {
      const int t = m.rtri[2 * k + side];
      const double* vf = m.V + 3 * m.rfree[2 * k + side];
      const double cS = (side == 0 ? 1.0 : -1.0) * m.len[k] / (2.0 * m.area[t]);
      for (int q = 0; q < 7; ++q) {
        const double* r = m.qp + 21 * t + 3 * q;
        const double rr = r[0] * rh[0] + r[1] * rh[1] + r[2] * rh[2];
        const double wv = rr / m.cdt;
        double s, c;
        sincos(m.kc * rr, &s, &c);
        const double sx = cS * (r[0] - vf[0]), sy = cS * (r[1] - vf[1]), sz = cS * (r[2] - vf[2]);
        const double p1 = m.qw[7 * t + q] * (sx * e1[0] + sy * e1[1] + sz * e1[2]);
        const double p2 = m.qw[7 * t + q] * (sx * e2[0] + sy * e2[1] + sz * e2[2]);
        const int llo = max(l0, (int)floor(n + wv - m.tb.Q)), lhi = min(l0 + n_steps - 1, (int)ceil(n + wv + 1));
        double2 sum = make_double2(0, 0);
        for (int l = llo; l <= lhi; ++l) {
          const double2 p = cm(dt_basis(m, n - l + wv), I[(size_t)(l - l0) * m.ns + k]);
          sum.x += p.x;
          sum.y += p.y;
        }
        const double2 e = cm(sum, make_double2(c, s));
        a1.x += p1 * e.x;
        a1.y += p1 * e.y;
        a2.x += p2 * e.x;
        a2.y += p2 * e.y;
      }
    }
  }
  const double cf = -m.mu / (4.0 * aimc::kPi);
  const double2 s1 = block_sum(a1);
  const double2 s2 = block_sum(a2);
  if (threadIdx.x == 0) {
    double2* f = F + ((size_t)(n - n0) * d.nd + di) * 2;
    if (accumulate) {
      f[0].x += cf * s1.x;
      f[0].y += cf * s1.y;
      f[1].x += cf * s2.x;
      f[1].y += cf * s2.y;
    } else {
      f[0] = make_double2(cf * s1.x, cf * s1.y);
      f[1] = make_double2(cf * s2.x, cf * s2.y);
    }
  }
}

// G_l[k] = conj(-mu/4pi) sum_n sum_{d,q} conj(A_{n-l}[d][q][k]) F[n][d][q] for l = l0..l0+n_steps-1
// into G[l - l0] (conjugated with conj_out); thread per (l, k)
__global__ void __launch_bounds__(kT) k_farfield_adj(MeshArgs m, DirArgs d, int l0, int n_steps, int n0, int n_out,
                                                     const double2* __restrict__ F, int conj_out,
                                                     double2* __restrict__ G) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)n_steps * m.ns) return;
  const int l = (int)(idx / m.ns) + l0, k = (int)(idx % m.ns);
  double2 acc = make_double2(0, 0);
  for (int di = 0; di < d.nd; ++di) {
    const double* rh = d.r + 3 * di;
    const double* e1 = d.e1 + 3 * di;
    const double* e2 = d.e2 + 3 * di;
    for (int side = 0; side < 2; ++side) {
      const int t = m.rtri[2 * k + side];
      const double* vf = m.V + 3 * m.rfree[2 * k + side];
      const double cS = (side == 0 ? 1.0 : -1.0) * m.len[k] / (2.0 * m.area[t]);
      for (int q = 0; q < 7; ++q) {
        const double* r = m.qp + 21 * t + 3 * q;
        const double rr = r[0] * rh[0] + r[1] * rh[1] + r[2] * rh[2];
        const double wv = rr / m.cdt;
        double s, c;
        sincos(m.kc * rr, &s, &c);
        const double sx = cS * (r[0] - vf[0]), sy = cS * (r[1] - vf[1]), sz = cS * (r[2] - vf[2]);
        const double p1 = m.qw[7 * t + q] * (sx * e1[0] + sy * e1[1] + sz * e1[2]);
        const double p2 = m.qw[7 * t + q] * (sx * e2[0] + sy * e2[1] + sz * e2[2]);
        const int nlo = max(n0, (int)floor(l - wv - 1)), nhi = min(n0 + n_out - 1, (int)ceil(l - wv + m.tb.Q));
        for (int n = nlo; n <= nhi; ++n) {
          const double2 f = cm(dt_basis(m, n - l + wv), make_double2(c, s));
          const double2* Fn = F + ((size_t)(n - n0) * d.nd + di) * 2;
          const double2 u1 = cmc(f, Fn[0]), u2 = cmc(f, Fn[1]);
          acc.x += p1 * u1.x + p2 * u2.x;
          acc.y += p1 * u1.y + p2 * u2.y;
        }
      }
    }
  }
  const double cf = -m.mu / (4.0 * aimc::kPi);  // real: conj(cf) = cf
  G[(size_t)(l - l0) * m.ns + k] = make_double2(cf * acc.x, conj_out ? -cf * acc.y : cf * acc.y);
}

// valT[m][e] = val[m][perm[e]]: the near-zone values of the transposed matrices
__global__ void k_gather_transpose(int nnz, int nm, const int* __restrict__ perm, const double2* __restrict__ val,
                                   double2* __restrict__ valT) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)nnz * nm) return;
  const int e = (int)(idx % nnz), mm = (int)(idx / nnz);
  valT[idx] = val[(size_t)mm * nnz + perm[e]];
}

MeshArgs mesh_args(aim_ctx* c) {
  MeshArgs m;
  m.rtri = c->d_rtri;
  m.rfree = c->d_rfree;
  m.len = c->d_len;
  m.area = c->d_area;
  m.V = c->d_v;
  m.qp = c->d_qp;
  m.qw = c->d_qw;
  m.ns = c->ns;
  m.dt = c->dt;
  m.wc = c->wc;
  m.kc = c->kc;
  m.cdt = c->c_med * c->dt;
  m.mu = c->mu_med;
  if (c->tb.kind != AIM_CPPIF)
    throw AimError{AIM_ERR_ARG, "the sampled-envelope excitation and far field interpolate with the CPPIF only"};
  m.tb = c->tb;
  return m;
}

}  // namespace

// time reach of the cubature points in units of dt: every point r has |r.u| / (c dt) <= this
// for any unit u (the largest vertex distance from the origin bounds the points)
static double reach(aim_ctx* c) { return c->rmax / (c->c_med * c->dt); }

void adj_excitation_samples(aim_ctx* c, const double* khat, const double* phat, int i0, int n_samp,
                            const double2* a, int l0, int n_steps, double2* V) {
  WaveArgs w{khat[0], khat[1], khat[2], phat[0], phat[1], phat[2]};
  const long long n = (long long)n_steps * c->ns;
  k_exc_samples<<<(int)((n + kT - 1) / kT), kT, 0, c->stream>>>(mesh_args(c), w, i0, n_samp, a, l0, n_steps, V);
  AIM_CHECK_LAUNCH();
}

// grad over the samples i0..i0+n_samp-1; with accumulate only the samples whose taps reach
// steps l0..l0+n_steps-1 are visited (the others receive nothing)
void adj_excitation_samples_adjoint(aim_ctx* c, const double* khat, const double* phat, int i0, int n_samp,
                                    int l0, int n_steps, const double2* lam, bool conj_lam, bool accumulate,
                                    double2* grad) {
  WaveArgs w{khat[0], khat[1], khat[2], phat[0], phat[1], phat[2]};
  int ia = i0, ib = i0 + n_samp - 1;
  if (accumulate) {  // B_{l-i} is non-zero only for l - i - u in (-1, Q], |u| <= reach
    const double u = reach(c);
    ia = std::max(ia, (int)std::floor(l0 - u - c->tb.Q) - 1);
    ib = std::min(ib, (int)std::ceil(l0 + n_steps - 1 + u + 1) + 1);
    if (ib < ia) return;
  }
  k_exc_samples_adj<<<ib - ia + 1, kT, 0, c->stream>>>(mesh_args(c), w, ia, l0, n_steps, lam, conj_lam ? 1 : 0,
                                                     accumulate ? 1 : 0, grad + (ia - i0));
  AIM_CHECK_LAUNCH();
}

// F over n = n0..n0+n_out-1; with accumulate only the n the steps l0..l0+n_steps-1 reach
void adj_farfield(aim_ctx* c, int nd, const double* d_dirs, int l0, int n_steps, const double2* I, int n0, int n_out,
                  bool accumulate, double2* F) {
  DirArgs d{nd, d_dirs, d_dirs + 3 * nd, d_dirs + 6 * nd};
  int na = n0, nb_ = n0 + n_out - 1;
  if (accumulate) {  // A_{n-l} is non-zero only for n - l + w in (-1, Q], |w| <= reach
    const double u = reach(c);
    na = std::max(na, (int)std::floor(l0 - u - 1) - 1);
    nb_ = std::min(nb_, (int)std::ceil(l0 + n_steps - 1 + u + c->tb.Q) + 1);
    if (nb_ < na) return;
  }
  k_farfield<<<(nb_ - na + 1) * nd, kT, 0, c->stream>>>(mesh_args(c), d, l0, n_steps, I, n0, na, accumulate ? 1 : 0,
                                                        F);
  AIM_CHECK_LAUNCH();
}

void adj_farfield_adjoint(aim_ctx* c, int nd, const double* d_dirs, int l0, int n_steps, int n0, int n_out,
                          const double2* F, bool conj_out, double2* G) {
  DirArgs d{nd, d_dirs, d_dirs + 3 * nd, d_dirs + 6 * nd};
  const long long n = (long long)n_steps * c->ns;
  k_farfield_adj<<<(int)((n + kT - 1) / kT), kT, 0, c->stream>>>(mesh_args(c), d, l0, n_steps, n0, n_out, F,
                                                                conj_out ? 1 : 0, G);
  AIM_CHECK_LAUNCH();
}

// transposed near-zone values (same pattern: the near relation is symmetric)
void adj_ensure_near_transpose(aim_ctx* c) {
  if (c->d_nearT || c->nnz == 0) return;
  const int ns = c->ns;
  const long long nnz = c->nnz;
  std::vector<int> perm(nnz);
  for (int k = 0; k < ns; ++k)
    for (int e = c->h_rowptr[k]; e < c->h_rowptr[k + 1]; ++e) {
      const int j = c->h_col[e];
      const int* b = c->h_col.data() + c->h_rowptr[j];
      const int* en = c->h_col.data() + c->h_rowptr[j + 1];
      const int* f = std::lower_bound(b, en, k);
      if (f == en || *f != k) throw AimError{AIM_ERR_ARG, "near-zone pattern is not symmetric"};
      perm[e] = (int)(f - c->h_col.data());
    }
  const int nm = c->n_delays + 1;
  int* d_perm = (int*)aim_alloc(c, nnz * sizeof(int));
  c->d_nearT = (double2*)aim_alloc(c, (size_t)nm * nnz * sizeof(double2));
  AIM_CUDA(cudaMemcpyAsync(d_perm, perm.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  const long long n = nnz * nm;
  k_gather_transpose<<<(int)((n + kT - 1) / kT), kT, 0, c->stream>>>((int)nnz, nm, d_perm, c->d_near, c->d_nearT);
  AIM_CHECK_LAUNCH();
  AIM_CUDA(cudaStreamSynchronize(c->stream));
}
