// Device-side setup of the ET-AIM tables (Sec. 4; Eq. 5), all in FP64:
//  * anterpolation coefficients (stage i) by moment matching up to order 3 per
//    axis (Sec. 5.1).  Matching every monomial xi^a with 0 <= a_x,a_y,a_z <= 3 on the
//    4x4x4 stencil is solved exactly by L_c[n,k] = int S_k^c(r) l_nx(xi_x) l_ny(xi_y)
//    l_nz(xi_z) dS with l_i the cubic Lagrange polynomials on the stencil nodes; the
//    integral is evaluated with a 6x6 Gauss-Legendre rule on the collapsed triangle
//    (exact for the degree-10 integrand);
//  * N_g from the largest node-to-node distance of the active grid (after Eq. 4);
//  * the delayed grid kernels G^A_m, G^phi_m on the zero-padded (2N, 2N, LZ) grid
//    (LZ: the z transform length of the active box) and their spectra (stage ii),
//    stored as the even-symmetric octant;
//  * the near-zone Galerkin entries Z_m[k,k'] (Eq. 4 entries, EFIE, singularity
//    extraction) minus their grid approximation L^T G_m L (stage iv).
#include <algorithm>
#include <cmath>
#include <vector>

#include "aim_internal.h"
#include "fft_kernels.cuh"
#include "setup_host.h"
#include "setup_gpu.h"
#include "tbasis.cuh"

// ------------------------------------------------------------------ temporal basis

// f^A_m(R) = (D^2 T)(m - R/c dt) e^{-j k R},  f^phi_m(R) = T(m - R/c dt) e^{-j k R}
// with (D^2 T)(u) = T''/dt^2 + 2 j w T'/dt - w^2 T (envelope derivative D = d/dt + j w)
__device__ __forceinline__ void time_kernels(const TimeK& p, int m, double R, double2& fA, double2& fP) {
  double T[4];
  tb_eval(p.tb, m, R / p.cdt, T);
  double re = T[2] / (p.dt * p.dt) - p.wc * p.wc * T[0];
  double im = 2.0 * p.wc * T[1] / p.dt;
  double s, c;
  sincos(-p.kc * R, &s, &c);
  fA = make_double2(re * c - im * s, re * s + im * c);
  fP = make_double2(T[0] * c, T[0] * s);
}

// values at R = 0+ and the one-sided R-derivatives there
__device__ __forceinline__ void time_kernels_at0(const TimeK& p, int m, double2& fA0, double2& fP0,
                                                 double2& dA0, double2& dP0) {
  double T[4];
  tb_eval(p.tb, m, 0.0, T);
  const double dt2 = p.dt * p.dt, w2 = p.wc * p.wc;
  fA0 = make_double2(T[2] / dt2 - w2 * T[0], 2.0 * p.wc * T[1] / p.dt);
  fP0 = make_double2(T[0], 0.0);
  double2 d1 = make_double2(T[3] / dt2 - w2 * T[1], 2.0 * p.wc * T[2] / p.dt);  // (D^2 T)'
  // d/dR [g(m - R/cdt) e^{-jkR}] = -g'/cdt - j k g
  dA0 = make_double2(-d1.x / p.cdt + p.kc * fA0.y, -d1.y / p.cdt - p.kc * fA0.x);
  dP0 = make_double2(-T[1] / p.cdt, -p.kc * T[0]);
}

// grid kernel value at integer offset (dx,dy,dz): G = f(R)/R, G(0) = 0
__device__ __forceinline__ void grid_kernel(const TimeK& p, int m, double h, int dx, int dy, int dz,
                                            double2& gA, double2& gP) {
  double fx = dx, fy = dy, fz = dz;
  double R = h * sqrt(fx * fx + fy * fy + fz * fz);
  if (R > 0.0) {
    time_kernels(p, m, R, gA, gP);
    gA = make_double2(gA.x / R, gA.y / R);
    gP = make_double2(gP.x / R, gP.y / R);
  } else {
    gA = gP = make_double2(0.0, 0.0);
  }
}

// ------------------------------------------------------------------ closed-form potentials
// I0 = int_T 1/|r - r'| dS',  I1 = int_T (r' - r)/|r - r'| dS'  (edge-sum form of
// Wilton et al. 1984 / Graglia 1993; signed distance P0 to each edge line).
__device__ void potential_integrals(const double* r, const double* A, const double* B, const double* C,
                                    double& I0, double I1[3]) {
  double e1[3], e2[3], n[3];
  for (int d = 0; d < 3; ++d) { e1[d] = B[d] - A[d]; e2[d] = C[d] - A[d]; }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int d = 0; d < 3; ++d) n[d] /= nn;
  double d0 = (r[0] - A[0]) * n[0] + (r[1] - A[1]) * n[1] + (r[2] - A[2]) * n[2];
  double rho[3] = {r[0] - d0 * n[0], r[1] - d0 * n[1], r[2] - d0 * n[2]};
  double ad = fabs(d0);
  double scale = fmax(sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]),
                      sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]));
  double tiny = (1e-13 * scale) * (1e-13 * scale);
  const double* P[4] = {A, B, C, A};
  double s0 = 0, sv[3] = {0, 0, 0};
  for (int ei = 0; ei < 3; ++ei) {
    const double* a = P[ei];
    const double* b = P[ei + 1];
    double t[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double tl = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    for (int d = 0; d < 3; ++d) t[d] /= tl;
    double u[3] = {t[1] * n[2] - t[2] * n[1], t[2] * n[0] - t[0] * n[2], t[0] * n[1] - t[1] * n[0]};
    double lp = (b[0] - rho[0]) * t[0] + (b[1] - rho[1]) * t[1] + (b[2] - rho[2]) * t[2];
    double lm = (a[0] - rho[0]) * t[0] + (a[1] - rho[1]) * t[1] + (a[2] - rho[2]) * t[2];
    double P0 = (a[0] - rho[0]) * u[0] + (a[1] - rho[1]) * u[1] + (a[2] - rho[2]) * u[2];
    double R0s = P0 * P0 + d0 * d0;
    double Rp = sqrt(R0s + lp * lp), Rm = sqrt(R0s + lm * lm);
    double Lg = 0.0, at = 0.0;
    if (R0s > tiny) {
      double num = lp >= 0 ? Rp + lp : R0s / (Rp - lp);
      double den = lm >= 0 ? Rm + lm : R0s / (Rm - lm);
      if (num > 0 && den > 0) Lg = log(num / den);
      at = atan(P0 * lp / (R0s + ad * Rp)) - atan(P0 * lm / (R0s + ad * Rm));
    }
    s0 += P0 * Lg - ad * at;
    double f = 0.5 * (R0s * Lg + lp * Rp - lm * Rm);
    for (int d = 0; d < 3; ++d) sv[d] += f * u[d];
  }
  I0 = s0;
  for (int d = 0; d < 3; ++d) I1[d] = sv[d] - d0 * n[d] * s0;
}

// ------------------------------------------------------------------ anterpolation rows

__device__ __forceinline__ double lagrange3(int i, double x) {
  switch (i) {
    case 0: return -(x - 1.0) * (x - 2.0) * (x - 3.0) / 6.0;
    case 1: return x * (x - 2.0) * (x - 3.0) / 2.0;
    case 2: return -x * (x - 1.0) * (x - 3.0) / 2.0;
    default: return x * (x - 1.0) * (x - 2.0) / 6.0;
  }
}

__global__ void k_lambda(SetupGeom g, const int* __restrict__ anchor, double ox, double oy, double oz,
                         double h, GaussRule gr, double* __restrict__ lam) {
  const int k = blockIdx.x;
  const int t = threadIdx.x;  // stencil slot (dz*4 + dy)*4 + dx
  const int dx = t & 3, dy = (t >> 2) & 3, dz = t >> 4;
  const double ra[3] = {ox + h * anchor[3 * k], oy + h * anchor[3 * k + 1], oz + h * anchor[3 * k + 2]};
  double acc[4] = {0, 0, 0, 0};
  for (int side = 0; side < 2; ++side) {
    const int tr = g.rtri[2 * k + side];
    const double sg = side == 0 ? 1.0 : -1.0;
    const double* vf = g.V + 3 * g.rfree[2 * k + side];
    const double area = g.area[tr];
    const double cS = sg * g.len[k] / (2.0 * area), cD = sg * g.len[k] / area;
    const double* A = g.V + 3 * g.F[3 * tr];
    const double* B = g.V + 3 * g.F[3 * tr + 1];
    const double* C = g.V + 3 * g.F[3 * tr + 2];
    for (int i = 0; i < gr.n; ++i)
      for (int j = 0; j < gr.n; ++j) {
        // collapsed triangle: barycentric (s(1-u), s u, 1-s), Jacobian 2 s (area-relative)
        double s = gr.x[i], u = gr.x[j];
        double w = gr.w[i] * gr.w[j] * 2.0 * s * area;
        double b0 = s * (1.0 - u), b1 = s * u, b2 = 1.0 - s;
        double r[3];
        for (int d = 0; d < 3; ++d) r[d] = b0 * A[d] + b1 * B[d] + b2 * C[d];
        double phi = w * lagrange3(dx, (r[0] - ra[0]) / h) * lagrange3(dy, (r[1] - ra[1]) / h) *
                     lagrange3(dz, (r[2] - ra[2]) / h);
        for (int d = 0; d < 3; ++d) acc[d] += cS * (r[d] - vf[d]) * phi;
        acc[3] += cD * phi;
      }
  }
  for (int c = 0; c < 4; ++c) lam[((size_t)k * 4 + c) * 64 + t] = acc[c];
}

// ------------------------------------------------------------------ N_g

__global__ void k_max_dist2(const int* __restrict__ cand, int nc, int N, int* __restrict__ best) {
  int local = 0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)nc * nc;
       idx += (long long)gridDim.x * blockDim.x) {
    int a = cand[idx / nc], b = cand[idx % nc];
    int ax = a % N, ay = (a / N) % N, az = a / (N * N);
    int bx = b % N, by = (b / N) % N, bz = b / (N * N);
    int d2 = (ax - bx) * (ax - bx) + (ay - by) * (ay - by) + (az - bz) * (az - bz);
    local = max(local, d2);
  }
  for (int o = 16; o > 0; o >>= 1) local = max(local, __shfl_xor_sync(0xffffffffu, local, o));
  if ((threadIdx.x & 31) == 0) atomicMax(best, local);
}

// ------------------------------------------------------------------ grid kernels

// G_m on the (2N, 2N, LZ) padded grid [z][y][x]: offset i for i < H, i - length for
// i > H, plane H unused (0), with H = N in x and y and H = LZ/2 in z
__global__ void k_kernel_grid(TimeK p, int m, int N, int LZ, double h, double2* __restrict__ GA,
                              double2* __restrict__ GP) {
  const long long L = 2 * N;
  const long long M = L * L * LZ;
  const int HZ = LZ / 2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < M;
       idx += (long long)gridDim.x * blockDim.x) {
    int ix = (int)(idx % L), iy = (int)((idx / L) % L), iz = (int)(idx / (L * L));
    double2 a = make_double2(0, 0), b = make_double2(0, 0);
    if (ix != N && iy != N && iz != HZ) {
      int dx = ix < N ? ix : ix - (int)L, dy = iy < N ? iy : iy - (int)L, dz = iz < HZ ? iz : iz - LZ;
      grid_kernel(p, m, h, dx, dy, dz, a, b);
    }
    GA[idx] = a;
    GP[idx] = b;
  }
}

// the octant [LZ/2 + 1][N + 1][N + 1] of the (2N, 2N, LZ) spectrum
__global__ void k_extract_octant(const double2* __restrict__ G, int N, int LZ, double scale,
                                 double2* __restrict__ o64, float2* __restrict__ o32) {
  const int n1 = N + 1;
  const long long L = 2 * N;
  const int noct = n1 * n1 * (LZ / 2 + 1);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < noct; idx += gridDim.x * blockDim.x) {
    int x = idx % n1, y = (idx / n1) % n1, z = idx / (n1 * n1);
    double2 v = G[((long long)z * L + y) * L + x];
    v = make_double2(scale * v.x, scale * v.y);
    o64[idx] = v;
    o32[idx] = make_float2((float)v.x, (float)v.y);
  }
}

// real-space table of G_m for offsets 0..D per axis: [m][kind][(D+1)^3]
__global__ void k_kernel_table(TimeK p, int nm, int D, double h, double2* __restrict__ tab) {
  const int D1 = D + 1, V3 = D1 * D1 * D1;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nm * V3; idx += gridDim.x * blockDim.x) {
    int m = idx / V3, r = idx % V3;
    int dx = r % D1, dy = (r / D1) % D1, dz = r / (D1 * D1);
    double2 a, b;
    grid_kernel(p, m, h, dx, dy, dz, a, b);
    tab[(size_t)(2 * m) * V3 + r] = a;
    tab[(size_t)(2 * m + 1) * V3 + r] = b;
  }
}

// ------------------------------------------------------------------ near zone

__device__ __forceinline__ bool singular_pair(const SetupGeom& g, int t, int tp) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (g.F[3 * t + a] == g.F[3 * tp + b]) return true;
  // centroid distance, plain IEEE arithmetic (no contraction)
  double dx = __dsub_rn(g.cent[3 * t], g.cent[3 * tp]);
  double dy = __dsub_rn(g.cent[3 * t + 1], g.cent[3 * tp + 1]);
  double dz = __dsub_rn(g.cent[3 * t + 2], g.cent[3 * tp + 2]);
  double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
  return d < __dmul_rn(2.0, g.mean_edge);
}

// Z_m[k,k'] for near pair e and delay m (one thread each):
//   mu/4pi int int S_k.S_k' f^A_m(R)/R + 1/(4 pi eps) int int div S_k div S_k' f^phi_m(R)/R,
// Cowper 7-point rules; singular triangle pairs: f(R)/R = f(0)/R + (f(R)-f(0))/R with the
// first inner integral in closed form.
__global__ void k_near_direct(SetupGeom g, TimeK p, int nnz, int nm, const int* __restrict__ prow,
                              const int* __restrict__ pcol, double2* __restrict__ zout) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)nnz * nm) return;
  const int e = (int)(idx % nnz), m = (int)(idx / nnz);
  const int k = prow[e], kp = pcol[e];
  const double cA = p.cA, cP = p.cP;
  double2 Z = make_double2(0, 0);
  double2 fA0, fP0, dA0, dP0;
  time_kernels_at0(p, m, fA0, fP0, dA0, dP0);
  for (int a = 0; a < 2; ++a) {
    const int t = g.rtri[2 * k + a];
    const double sa = a == 0 ? 1.0 : -1.0;
    const double* vf = g.V + 3 * g.rfree[2 * k + a];
    const double ck = sa * g.len[k] / (2.0 * g.area[t]), dk = sa * g.len[k] / g.area[t];
    for (int b = 0; b < 2; ++b) {
      const int tp = g.rtri[2 * kp + b];
      const double sb = b == 0 ? 1.0 : -1.0;
      const double* vfp = g.V + 3 * g.rfree[2 * kp + b];
      const double cp = sb * g.len[kp] / (2.0 * g.area[tp]), dp = sb * g.len[kp] / g.area[tp];
      const bool sing = singular_pair(g, t, tp);
      double2 IA = make_double2(0, 0), IP = make_double2(0, 0);
      for (int qa = 0; qa < 7; ++qa) {
        const double* ra = g.qp + 21 * t + 3 * qa;
        const double wa = g.qw[7 * t + qa];
        const double rho[3] = {ra[0] - vf[0], ra[1] - vf[1], ra[2] - vf[2]};
        for (int qb = 0; qb < 7; ++qb) {
          const double* rb = g.qp + 21 * tp + 3 * qb;
          const double ww = wa * g.qw[7 * tp + qb];
          const double dx = ra[0] - rb[0], dy = ra[1] - rb[1], dz = ra[2] - rb[2];
          const double R = sqrt(dx * dx + dy * dy + dz * dz);
          double2 fA, fP, hA, hP;
          time_kernels(p, m, R, fA, fP);
          if (sing) {
            if (R == 0.0) {
              hA = dA0;
              hP = dP0;
            } else {
              hA = make_double2((fA.x - fA0.x) / R, (fA.y - fA0.y) / R);
              hP = make_double2((fP.x - fP0.x) / R, (fP.y - fP0.y) / R);
            }
          } else {
            hA = make_double2(fA.x / R, fA.y / R);
            hP = make_double2(fP.x / R, fP.y / R);
          }
          const double dot = rho[0] * (rb[0] - vfp[0]) + rho[1] * (rb[1] - vfp[1]) + rho[2] * (rb[2] - vfp[2]);
          IA.x += ww * dot * hA.x;
          IA.y += ww * dot * hA.y;
          IP.x += ww * hP.x;
          IP.y += ww * hP.y;
        }
        if (sing) {
          double I0, I1[3];
          const double* A = g.V + 3 * g.F[3 * tp];
          const double* B = g.V + 3 * g.F[3 * tp + 1];
          const double* C = g.V + 3 * g.F[3 * tp + 2];
          potential_integrals(ra, A, B, C, I0, I1);
          // int_T' (r' - v')/R dS' = I1 + (r - v') I0
          double sdot = 0.0;
          for (int d = 0; d < 3; ++d) sdot += rho[d] * (I1[d] + (ra[d] - vfp[d]) * I0);
          IA.x += fA0.x * wa * sdot;
          IA.y += fA0.y * wa * sdot;
          IP.x += fP0.x * wa * I0;
          IP.y += fP0.y * wa * I0;
        }
      }
      const double sA = cA * ck * cp, sP = cP * dk * dp;
      Z.x += sA * IA.x + sP * IP.x;
      Z.y += sA * IA.y + sP * IP.y;
    }
  }
  zout[(size_t)m * nnz + e] = Z;
}

// subtract the grid approximation sum_c coef_c L_c[.,k]^T G_m L_c[.,k'] (one warp per (e, m))
__global__ void k_precorrect(int nnz, int nm, const int* __restrict__ prow, const int* __restrict__ pcol,
                             const int* __restrict__ anchor, const double* __restrict__ lam,
                             const double2* __restrict__ tab, int D, double cA, double cP,
                             double2* __restrict__ zout) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (long long)nnz * nm) return;
  const int e = (int)(w % nnz), m = (int)(w / nnz);
  const int k = prow[e], kp = pcol[e];
  const int D1 = D + 1, V3 = D1 * D1 * D1;
  const double2* tA = tab + (size_t)(2 * m) * V3;
  const double2* tP = tab + (size_t)(2 * m + 1) * V3;
  const int bx = anchor[3 * k] - anchor[3 * kp], by = anchor[3 * k + 1] - anchor[3 * kp + 1],
            bz = anchor[3 * k + 2] - anchor[3 * kp + 2];
  const double* lk = lam + (size_t)k * 256;
  const double* lkp = lam + (size_t)kp * 256;
  double2 acc = make_double2(0, 0);
  for (int s = lane; s < 64; s += 32) {
    const int sx = s & 3, sy = (s >> 2) & 3, sz = s >> 4;
    double2 a[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int q = 0; q < 64; ++q) {
      const int qx = q & 3, qy = (q >> 2) & 3, qz = q >> 4;
      const int dx = abs(bx + sx - qx), dy = abs(by + sy - qy), dz = abs(bz + sz - qz);
      const int gi = (dz * D1 + dy) * D1 + dx;
      const double2 gA = tA[gi], gP = tP[gi];
      for (int c = 0; c < 3; ++c) {
        const double l = lkp[c * 64 + q];
        a[c].x += gA.x * l;
        a[c].y += gA.y * l;
      }
      const double l = lkp[192 + q];
      a[3].x += gP.x * l;
      a[3].y += gP.y * l;
    }
    for (int c = 0; c < 4; ++c) {
      const double l = lk[c * 64 + s] * (c < 3 ? cA : cP);
      acc.x += l * a[c].x;
      acc.y += l * a[c].y;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) {
    double2 z = zout[(size_t)m * nnz + e];
    zout[(size_t)m * nnz + e] = make_double2(z.x - acc.x, z.y - acc.y);
  }
}

__global__ void k_diag_inverse(int ns, int nnz, const int* __restrict__ rowptr, const int* __restrict__ col,
                               const double2* __restrict__ z0direct, const double2* __restrict__ zdiag_fallback,
                               double2* __restrict__ dinv) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  double2 d = zdiag_fallback ? zdiag_fallback[k] : make_double2(0, 0);
  for (int e = rowptr[k]; e < rowptr[k + 1]; ++e)
    if (col[e] == k) d = z0direct[e];
  double n = d.x * d.x + d.y * d.y;
  dinv[k] = n > 0 ? make_double2(d.x / n, -d.y / n) : make_double2(1.0, 0.0);
}

// position of column k in the sorted CSR row [e0, e1), or -1
__device__ __forceinline__ int csr_find(const int* __restrict__ col, int e0, int e1, int k) {
  while (e0 < e1) {
    const int mid = (e0 + e1) >> 1;
    const int v = col[mid];
    if (v == k) return mid;
    if (v < k) e0 = mid + 1;
    else e1 = mid;
  }
  return -1;
}

// Near-zone sparse approximate inverse (right preconditioner, no counterpart in the
// paper): column k of M minimises || Zn[:, S] m - e_k ||_2, Zn = Z_0 on near pairs (0 off
// the pattern), S the near set of k (CSR row k).  Normal equations G m = g with
//   G[i][j] = sum_r conj(Zn[r, S_i]) Zn[r, S_j]   (r over the near sets of S_i and S_j,
//             merged from their sorted CSR rows),   g[i] = conj(Zn[k, S_i]).
// One block per k: G (Hermitian; upper triangle computed, lower mirrored) in shared
// memory, Gaussian elimination with partial pivoting (largest |a|, lowest row on ties)
// of the augmented n x (n+1) system, FP64; back substitution by one warp; m scattered to
// M[S_i, k] (the entry of column k in CSR row S_i).  A zero pivot sets *status and
// leaves the column zero.
constexpr int kSaiThreads = 128;
template <class T> struct SaiReal;
template <> struct SaiReal<double2> { using R = double; };
template <> struct SaiReal<float2> { using R = float; };

// T: the complex type of the elimination (double2, or float2 for wide patterns: the
// factorisation is O(n^3) and GB300's FP64 rate is low; G is still summed in FP64).
// The local system is scaled by sigma = 1 / |Z_0[k, k]| (A' = sigma A, m = sigma m') so
// that its entries are O(1): |Z_0|^2 of a time-differentiated EFIE exceeds FP32's range.
template <class T>
__global__ void __launch_bounds__(kSaiThreads) k_near_sai(const int* __restrict__ rowptr, const int* __restrict__ col,
                                                          const double2* __restrict__ z0, double2* __restrict__ M,
                                                          int* __restrict__ status) {
  using R = typename SaiReal<T>::R;
  extern __shared__ __align__(16) unsigned char sai_smem[];
  T* a = reinterpret_cast<T*>(sai_smem);  // row i at a[i * (n + 1)], column n = right-hand side
  __shared__ int piv;
  __shared__ R pbest;
  __shared__ double sig;
  const int k = blockIdx.x, tid = threadIdx.x;
  const int e0 = rowptr[k], n = rowptr[k + 1] - e0, ld = n + 1;
  const int* S = col + e0;
  if (tid == 0) {
    const int ek = csr_find(col, e0, e0 + n, k);
    const double2 d = ek >= 0 ? z0[ek] : make_double2(1, 0);
    const double ad = sqrt(d.x * d.x + d.y * d.y);
    sig = ad > 0 ? 1.0 / ad : 1.0;
  }
  __syncthreads();
  const double s2 = sig * sig;
  for (int t = tid; t < n * n; t += kSaiThreads) {
    const int i = t / n, j = t % n;
    if (i > j) continue;
    const int si = S[i], sj = S[j];
    int p = rowptr[si], q = rowptr[sj];
    const int pe = rowptr[si + 1], qe = rowptr[sj + 1];
    double gx = 0, gy = 0;
    while (p < pe && q < qe) {  // r in the sets of S_i and S_j, ascending
      const int rp = col[p], rq = col[q];
      if (rp < rq) {
        ++p;
      } else if (rq < rp) {
        ++q;
      } else {
        const int r0 = rowptr[rp], r1 = rowptr[rp + 1];
        const double2 zi = z0[csr_find(col, r0, r1, si)], zj = z0[csr_find(col, r0, r1, sj)];
        gx += zi.x * zj.x + zi.y * zj.y;  // conj(zi) zj
        gy += zi.x * zj.y - zi.y * zj.x;
        ++p;
        ++q;
      }
    }
    a[i * ld + j] = T{(R)(s2 * gx), (R)(s2 * gy)};
  }
  for (int i = tid; i < n; i += kSaiThreads) {
    const double2 z = z0[e0 + i];  // Zp[k, S_i]
    a[i * ld + n] = T{(R)(sig * z.x), (R)(-sig * z.y)};
  }
  __syncthreads();
  for (int t = tid; t < n * n; t += kSaiThreads) {
    const int i = t / n, j = t % n;
    if (i > j) a[i * ld + j] = T{a[j * ld + i].x, -a[j * ld + i].y};
  }
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    if (tid < 32) {
      R best = -1;
      int bi = c;
      for (int r = c + tid; r < n; r += 32) {
        const T v = a[r * ld + c];
        const R m2 = v.x * v.x + v.y * v.y;
        if (m2 > best) {
          best = m2;
          bi = r;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const R ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (tid == 0) {
        piv = bi;
        pbest = best;
      }
    }
    __syncthreads();
    if (!(pbest > (R)0)) {
      if (tid == 0) atomicExch(status, 1);
      for (int i = tid; i < n; i += kSaiThreads) a[i * ld + n] = T{0, 0};
      __syncthreads();
      break;
    }
    if (piv != c)
      for (int j = c + tid; j <= n; j += kSaiThreads) {
        const T t = a[c * ld + j];
        a[c * ld + j] = a[piv * ld + j];
        a[piv * ld + j] = t;
      }
    __syncthreads();
    const T d = a[c * ld + c];
    const R dn = d.x * d.x + d.y * d.y;
    const int w = n - c;  // columns c+1 .. n
    for (int t = tid; t < (n - c - 1) * w; t += kSaiThreads) {
      const int r = c + 1 + t / w, j = c + 1 + t % w;
      const T q = a[r * ld + c];
      const T f = T{(q.x * d.x + q.y * d.y) / dn, (q.y * d.x - q.x * d.y) / dn};  // q / d
      const T u = a[c * ld + j];
      a[r * ld + j] = T{a[r * ld + j].x - (f.x * u.x - f.y * u.y), a[r * ld + j].y - (f.x * u.y + f.y * u.x)};
    }
    __syncthreads();
  }
  if (tid < 32) {
    for (int r = n - 1; r >= 0; --r) {
      R sx = 0, sy = 0;
      for (int j = r + 1 + tid; j < n; j += 32) {
        const T u = a[r * ld + j], x = a[j * ld + n];
        sx += u.x * x.x - u.y * x.y;
        sy += u.x * x.y + u.y * x.x;
      }
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
      }
      if (tid == 0) {
        const T d = a[r * ld + r], b = a[r * ld + n];
        const R dn = d.x * d.x + d.y * d.y;
        const T t = T{b.x - sx, b.y - sy};
        a[r * ld + n] = dn > (R)0 ? T{(t.x * d.x + t.y * d.y) / dn, (t.y * d.x - t.x * d.y) / dn} : T{0, 0};
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += kSaiThreads) {
    const int r = S[i];
    const int e = csr_find(col, rowptr[r], rowptr[r + 1], k);
    if (e >= 0) M[e] = make_double2(sig * (double)a[i * ld + n].x, sig * (double)a[i * ld + n].y);
  }
}

__global__ void k_round_c64(const double2* __restrict__ in, long long n, float2* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// ------------------------------------------------------------------ host driver

static int launch_blocks(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  return (int)std::min<long long>(std::max<long long>(b, 1), 152LL * 64);
}

void setup_device_tables(aim_ctx* c, HostMesh& hm, const std::vector<int>& anchor) {
  cudaStream_t st = c->stream;
  const int N = c->N, L = c->L, ns = c->ns;
  TimeK tk;
  tk.dt = c->dt;
  tk.wc = c->wc;
  tk.kc = c->kc;
  tk.cdt = c->c_med * c->dt;
  tk.cA = c->mu_med / (4.0 * aimc::kPi);
  tk.cP = 1.0 / (4.0 * aimc::kPi * c->eps_med);
  tk.tb = c->tb;

  SetupGeom g;
  g.V = c->d_v;
  g.F = c->d_tri;
  g.rtri = c->d_rtri;
  g.rfree = c->d_rfree;
  g.len = c->d_len;
  g.area = c->d_area;
  g.qp = c->d_qp;
  g.qw = c->d_qw;
  g.cent = c->d_cent;
  g.mean_edge = c->mean_edge;

  // ---- anterpolation rows (FP64) and their FP32 copy
  GaussRule gr;
  {
    std::vector<double> x, w;
    host_gauss_legendre(6, x, w);
    gr.n = 6;
    for (int i = 0; i < 6; ++i) {
      gr.x[i] = 0.5 * (x[i] + 1.0);
      gr.w[i] = 0.5 * w[i];
    }
  }
  k_lambda<<<ns, 64, 0, st>>>(g, c->d_anchor, c->origin[0], c->origin[1], c->origin[2], c->h, gr, c->d_lam);
  AIM_CHECK_LAUNCH();
  std::vector<double> lam((size_t)ns * 256);
  AIM_CUDA(cudaMemcpyAsync(lam.data(), c->d_lam, lam.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  AIM_CUDA(cudaStreamSynchronize(st));
  {
    std::vector<float> lf(lam.size());
    for (size_t i = 0; i < lam.size(); ++i) lf[i] = (float)lam[i];
    AIM_CUDA(cudaMemcpyAsync(c->d_lamf, lf.data(), lf.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    AIM_CUDA(cudaStreamSynchronize(st));
  }
  // ---- node-major transpose (stage i as a gather)
  std::vector<int> nptr, nidx, nslot;
  host_transpose_pattern(N, anchor, ns, nptr, nidx, nslot);
  {
    std::vector<double4_32a> cf(nidx.size());
    std::vector<float4> cff(nidx.size());
    for (size_t e = 0; e < nidx.size(); ++e) {
      const double* l = &lam[(size_t)nidx[e] * 256 + nslot[e]];
      cf[e] = make_double4_32a(l[0], l[64], l[128], l[192]);
      cff[e] = make_float4((float)l[0], (float)l[64], (float)l[128], (float)l[192]);
    }
    c->d_nptr = (int*)aim_alloc(c, nptr.size() * sizeof(int));
    c->d_nidx = (int*)aim_alloc(c, nidx.size() * sizeof(int));
    c->d_ncoef = (double4_32a*)aim_alloc(c, cf.size() * sizeof(double4_32a));
    c->d_ncoeff = (float4*)aim_alloc(c, cff.size() * sizeof(float4));
    AIM_CUDA(cudaMemcpyAsync(c->d_nptr, nptr.data(), nptr.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    AIM_CUDA(cudaMemcpyAsync(c->d_nidx, nidx.data(), nidx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    AIM_CUDA(cudaMemcpyAsync(c->d_ncoef, cf.data(), cf.size() * sizeof(double4_32a), cudaMemcpyHostToDevice, st));
    AIM_CUDA(cudaMemcpyAsync(c->d_ncoeff, cff.data(), cff.size() * sizeof(float4), cudaMemcpyHostToDevice, st));
    AIM_CUDA(cudaStreamSynchronize(st));
  }
  // ---- N_g = floor(R_max/(c dt) + Q), R_max the largest active node distance
  {
    std::vector<int> cand;
    host_extreme_candidates(N, nptr, cand, c->n_active);
    int* d_cand = (int*)aim_alloc(c, std::max<size_t>(1, cand.size()) * sizeof(int));
    int* d_best = (int*)aim_alloc(c, sizeof(int));
    AIM_CUDA(cudaMemsetAsync(d_best, 0, sizeof(int), st));
    AIM_CUDA(cudaMemcpyAsync(d_cand, cand.data(), cand.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    long long work = (long long)cand.size() * (long long)cand.size();
    k_max_dist2<<<launch_blocks(work, 256), 256, 0, st>>>(d_cand, (int)cand.size(), N, d_best);
    AIM_CHECK_LAUNCH();
    int best = 0;
    AIM_CUDA(cudaMemcpyAsync(&best, d_best, sizeof(int), cudaMemcpyDeviceToHost, st));
    AIM_CUDA(cudaStreamSynchronize(st));
    double rmax = c->h * std::sqrt((double)best);
    c->n_delays = (int)std::floor(rmax / (c->c_med * c->dt) + c->tb.Q);
    if (c->n_delays + 1 > aimc::kMaxDelays) throw AimError{AIM_ERR_ARG, "too many delays (N_g + 1 > 32)"};
  }
  const int nm = c->n_delays + 1;
  // ---- twiddles W_n^t = exp(-2 pi i t / n) of the x/y (n = L) and z (n = LZ) transforms
  {
    auto table = [&](int n, double2*& d64, float2*& d32) {
      std::vector<double2> tw(n);
      std::vector<float2> twf(n);
      for (int t = 0; t < n; ++t) {
        double a = 2.0 * aimc::kPi * (double)t / (double)n;
        tw[t] = make_double2(std::cos(a), -std::sin(a));
        twf[t] = make_float2((float)tw[t].x, (float)tw[t].y);
      }
      d64 = (double2*)aim_alloc(c, n * sizeof(double2));
      d32 = (float2*)aim_alloc(c, n * sizeof(float2));
      AIM_CUDA(cudaMemcpyAsync(d64, tw.data(), n * sizeof(double2), cudaMemcpyHostToDevice, st));
      AIM_CUDA(cudaMemcpyAsync(d32, twf.data(), n * sizeof(float2), cudaMemcpyHostToDevice, st));
      AIM_CUDA(cudaStreamSynchronize(st));
    };
    table(L, c->d_tw, c->d_twf);
    table(c->LZ, c->d_twz, c->d_twzf);
  }
  // ---- kernel spectra: tabulate on the (L, L, LZ) padded grid, full 3-D FFT (FP64),
  //      keep the octant
  {
    const size_t n1 = (size_t)(N + 1);
    const size_t oct = n1 * n1 * (size_t)(c->LZ / 2 + 1);
    c->d_kspec = (double2*)aim_alloc(c, (size_t)nm * 2 * oct * sizeof(double2));
    c->d_kspecf = (float2*)aim_alloc(c, (size_t)nm * 2 * oct * sizeof(float2));
    const size_t M = (size_t)L * L * c->LZ;
    double2* GA = nullptr;
    double2* GP = nullptr;
    AIM_CUDA(cudaMalloc(&GA, M * sizeof(double2)));
    cudaError_t e2 = cudaMalloc(&GP, M * sizeof(double2));
    if (e2 != cudaSuccess) {
      cudaFree(GA);
      throw AimError{AIM_ERR_OOM, "kernel tabulation scratch"};
    }
    try {
      const double cA = c->mu_med / (4.0 * aimc::kPi), cP = 1.0 / (4.0 * aimc::kPi * c->eps_med);
      for (int m = 0; m < nm; ++m) {
        k_kernel_grid<<<launch_blocks((long long)M, 256), 256, 0, st>>>(tk, m, N, c->LZ, c->h, GA, GP);
        AIM_CHECK_LAUNCH();
        for (int kind = 0; kind < 2; ++kind) {
          double2* G = kind == 0 ? GA : GP;
          fft3d_full_c128(c, G);
          k_extract_octant<<<launch_blocks((long long)oct, 256), 256, 0, st>>>(
              G, N, c->LZ, (kind == 0 ? cA : cP) / (double)M, c->d_kspec + ((size_t)m * 2 + kind) * oct,
              c->d_kspecf + ((size_t)m * 2 + kind) * oct);
          AIM_CHECK_LAUNCH();
        }
      }
      AIM_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
      cudaFree(GA);
      cudaFree(GP);
      throw;
    }
    cudaFree(GA);
    cudaFree(GP);
  }
  // ---- near zone
  {
    std::vector<int> rowptr, col;
    host_near_pairs(hm, c->near_radius, rowptr, col);
    c->nnz = (long long)col.size();
    const int nnz = (int)col.size();
    c->d_rowptr = (int*)aim_alloc(c, (ns + 1) * sizeof(int));
    AIM_CUDA(cudaMemcpyAsync(c->d_rowptr, rowptr.data(), (ns + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    c->d_dinv = (double2*)aim_alloc(c, ns * sizeof(double2));
    // pair list for the fill: all near pairs plus the diagonal (preconditioner)
    std::vector<int> prow, pcol;
    for (int k = 0; k < ns; ++k)
      for (int e = rowptr[k]; e < rowptr[k + 1]; ++e) {
        prow.push_back(k);
        pcol.push_back(col[e]);
      }
    bool diag_in = c->near_radius >= 0;
    std::vector<int> drow;
    if (!diag_in)
      for (int k = 0; k < ns; ++k) drow.push_back(k);
    const int nfill = nnz + (int)drow.size();
    std::vector<int> frow(prow), fcol(pcol);
    frow.insert(frow.end(), drow.begin(), drow.end());
    fcol.insert(fcol.end(), drow.begin(), drow.end());
    int* d_prow = (int*)aim_alloc(c, std::max(1, nfill) * sizeof(int));
    int* d_pcol = (int*)aim_alloc(c, std::max(1, nfill) * sizeof(int));
    c->d_col = d_pcol;  // the first nnz entries are the CSR columns
    if (nfill) {
      AIM_CUDA(cudaMemcpyAsync(d_prow, frow.data(), nfill * sizeof(int), cudaMemcpyHostToDevice, st));
      AIM_CUDA(cudaMemcpyAsync(d_pcol, fcol.data(), nfill * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    double2* zdir = (double2*)aim_alloc(c, std::max<size_t>(1, (size_t)nm * nfill) * sizeof(double2));
    if (nfill) {
      long long work = (long long)nfill * nm;
      k_near_direct<<<(int)((work + 127) / 128), 128, 0, st>>>(g, tk, nfill, nm, d_prow, d_pcol, zdir);
      AIM_CHECK_LAUNCH();
    }
    // preconditioner from the direct immediate self terms Z_0[k,k]
    {
      double2* fallback = nullptr;
      if (!diag_in) fallback = zdir + nnz;  // m = 0 block, diagonal entries after the near ones
      k_diag_inverse<<<(ns + 127) / 128, 128, 0, st>>>(ns, nnz, c->d_rowptr, c->d_col, zdir, fallback, c->d_dinv);
      AIM_CHECK_LAUNCH();
    }
    // near values: Z_m - L^T G_m L on the near pairs, stored [m][nnz]
    c->d_near = (double2*)aim_alloc(c, std::max<size_t>(1, (size_t)nm * nnz) * sizeof(double2));
    if (nnz) {
      for (int m = 0; m < nm; ++m)
        AIM_CUDA(cudaMemcpyAsync(c->d_near + (size_t)m * nnz, zdir + (size_t)m * nfill, nnz * sizeof(double2),
                                 cudaMemcpyDeviceToDevice, st));
      int D = 3;
      for (int k = 0; k < ns; ++k)
        for (int e = rowptr[k]; e < rowptr[k + 1]; ++e)
          for (int d = 0; d < 3; ++d) D = std::max(D, std::abs(anchor[3 * k + d] - anchor[3 * col[e] + d]) + 3);
      const size_t V3 = (size_t)(D + 1) * (D + 1) * (D + 1);
      double2* tab = (double2*)aim_alloc(c, (size_t)nm * 2 * V3 * sizeof(double2));
      k_kernel_table<<<launch_blocks((long long)nm * V3, 256), 256, 0, st>>>(tk, nm, D, c->h, tab);
      AIM_CHECK_LAUNCH();
      long long warps = (long long)nnz * nm;
      k_precorrect<<<(int)((warps * 32 + 255) / 256), 256, 0, st>>>(nnz, nm, d_prow, d_pcol, c->d_anchor, c->d_lam,
                                                                   tab, D, tk.cA, tk.cP, c->d_near);
      AIM_CHECK_LAUNCH();
    }
    // SAI from the direct immediate entries Z_0 on its pattern: the near pairs, or the
    // pairs within precond_radius (their Z_0 filled here)
    if (c->precond == AIM_PRECOND_NEAR_SAI) {
      std::vector<int> srowptr = rowptr, scol = col;
      const double2* sz = zdir;
      c->d_srowptr = c->d_rowptr;
      c->d_scol = c->d_col;
      if (c->precond_radius != c->near_radius) {
        host_near_pairs(hm, c->precond_radius, srowptr, scol);
        const int sn = (int)scol.size();
        std::vector<int> sprow(sn);
        for (int k = 0; k < ns; ++k)
          for (int e = srowptr[k]; e < srowptr[k + 1]; ++e) sprow[e] = k;
        c->d_srowptr = (int*)aim_alloc(c, (ns + 1) * sizeof(int));
        c->d_scol = (int*)aim_alloc(c, std::max(1, sn) * sizeof(int));
        int* d_sprow = (int*)aim_alloc(c, std::max(1, sn) * sizeof(int));
        double2* zs = (double2*)aim_alloc(c, std::max(1, sn) * sizeof(double2));
        AIM_CUDA(cudaMemcpyAsync(c->d_srowptr, srowptr.data(), (ns + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
        if (sn) {
          AIM_CUDA(cudaMemcpyAsync(c->d_scol, scol.data(), sn * sizeof(int), cudaMemcpyHostToDevice, st));
          AIM_CUDA(cudaMemcpyAsync(d_sprow, sprow.data(), sn * sizeof(int), cudaMemcpyHostToDevice, st));
          k_near_direct<<<(sn + 127) / 128, 128, 0, st>>>(g, tk, sn, 1, d_sprow, c->d_scol, zs);
          AIM_CHECK_LAUNCH();
        }
        sz = zs;
      }
      c->snnz = (long long)scol.size();
      c->h_srowptr = srowptr;
      int nmax = 0;
      for (int k = 0; k < ns; ++k) nmax = std::max(nmax, srowptr[k + 1] - srowptr[k]);
      if (nmax > 144) throw AimError{AIM_ERR_ARG, "SAI preconditioner: a pattern set has more than 144 RWGs"};
      if (nmax < 1) throw AimError{AIM_ERR_ARG, "SAI preconditioner: empty pattern"};
      const bool fp64 = nmax <= 32;
      const size_t sm = (size_t)nmax * (nmax + 1) * (fp64 ? sizeof(double2) : sizeof(float2));
      auto kern = fp64 ? k_near_sai<double2> : k_near_sai<float2>;
      if (sm > 48 * 1024) AIM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      c->d_sai = (double2*)aim_alloc(c, (size_t)std::max<long long>(1, c->snnz) * sizeof(double2));
      int* d_status = (int*)aim_alloc(c, sizeof(int));
      AIM_CUDA(cudaMemsetAsync(c->d_sai, 0, (size_t)c->snnz * sizeof(double2), st));
      AIM_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));
      kern<<<ns, kSaiThreads, sm, st>>>(c->d_srowptr, c->d_scol, sz, c->d_sai, d_status);
      AIM_CHECK_LAUNCH();
      int h_status = 0;
      AIM_CUDA(cudaMemcpyAsync(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
      AIM_CUDA(cudaStreamSynchronize(st));
      if (h_status) throw AimError{AIM_ERR_ARG, "SAI preconditioner: a singular local system"};
      if (c->precision == AIM_C64) {  // the complex64 path applies M in FP32
        c->d_saif = (float2*)aim_alloc(c, (size_t)std::max<long long>(1, c->snnz) * sizeof(float2));
        k_round_c64<<<launch_blocks(c->snnz, 256), 256, 0, st>>>(c->d_sai, c->snnz, c->d_saif);
        AIM_CHECK_LAUNCH();
      }
    }
    AIM_CUDA(cudaStreamSynchronize(st));
    c->h_rowptr = rowptr;
    c->h_col = col;
  }
}

// ------------------------------------------------------------------ full 3-D FFT (setup)
#include "operator_body.cuh"

// the full FFT of a [LZ][L][L] grid (z, y, x)
template <int L>
static void fft3d_full_L(aim_ctx* c, double2* G) {
  constexpr int W = col_width<L, double2>();
  cudaStream_t st = c->stream;
  const double2* tw = c->d_tw;
  const int LZ = c->LZ;
  const int rp = std::max(1, 2048 / L);
  size_t sm = (L + rp * L + row_scratch<L>(rp)) * sizeof(double2);
  smem_opt_in(k_rows<L, false, double2>, sm);
  k_rows<L, false, double2><<<(L * LZ + rp - 1) / rp, 256, sm, st>>>(G, G, L * LZ, L, L, L, L, tw, rp);
  AIM_CHECK_LAUNCH();
  sm = (L + 2 * L * W) * sizeof(double2);
  smem_opt_in(k_cols<L, W, false, double2>, sm);
  const long long LL2 = (long long)L * L;
  // y lines: planes z (stride L^2), element stride L
  k_cols<L, W, false, double2><<<dim3(L / W, LZ, 1), 256, sm, st>>>(G, G, L, L, L, L, L, LL2, LL2, 0, 0, tw);
  AIM_CHECK_LAUNCH();
  // z lines: rows y (stride L), element stride L^2
  with_zlen(LZ, [&](auto lz) {
    constexpr int Z = decltype(lz)::value;
    if constexpr (Z <= L) {
      constexpr int WZ = col_width<Z, double2>();
      const size_t smz = (Z + 2 * Z * WZ) * sizeof(double2);
      smem_opt_in(k_cols<Z, WZ, false, double2>, smz);
      k_cols<Z, WZ, false, double2><<<dim3(L / WZ, L, 1), 256, smz, st>>>(G, G, Z, Z, LL2, LL2, L, L, L, 0, 0,
                                                                         c->d_twz);
      AIM_CHECK_LAUNCH();
    } else {
      throw AimError{AIM_ERR_ARG, "z transform longer than the padded length"};
    }
  });
}

void fft3d_full_c128(aim_ctx* c, double2* G) { AIM_DISPATCH_L(c->L, fft3d_full_L<LL>(c, G)); }
