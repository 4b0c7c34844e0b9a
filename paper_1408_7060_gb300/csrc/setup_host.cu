// Host-side bookkeeping of the setup: RWG table, cubature points, stencil anchors,
// near-zone pair list, transposed anterpolation pattern and the N_g candidate set.
// Compiled with -ffp-contract=off so that the integer decisions taken from floating
// point (anchors, near pairs) follow plain IEEE arithmetic.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <tuple>

#include "aim_internal.h"
#include "setup_host.h"

namespace {

double norm3(const double* a, const double* b) {
  double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
  return std::sqrt(dx * dx + dy * dy + dz * dz);
}

}  // namespace

// RWG ordering (Sec. 3, Eq. 3; basis of reference [14]): edges sorted by
// (lower, higher) vertex; T+ runs lower -> higher in its counter-clockwise cycle.
void host_build_rwg(const aim_mesh* m, HostMesh& hm) {
  if (!m || !m->v || !m->tri || m->nv < 4 || m->nt < 4) throw AimError{AIM_ERR_ARG, "empty mesh"};
  hm.nv = m->nv;
  hm.nt = m->nt;
  hm.V.assign(m->v, m->v + 3 * (size_t)m->nv);
  hm.F.assign(m->tri, m->tri + 3 * (size_t)m->nt);
  for (int i = 0; i < 3 * hm.nt; ++i)
    if (hm.F[i] < 0 || hm.F[i] >= hm.nv) throw AimError{AIM_ERR_MESH, "vertex index out of range"};
  struct Own {
    int64_t key;
    int t, dir, opp;
  };
  std::vector<Own> own;
  own.reserve(3 * (size_t)hm.nt);
  for (int t = 0; t < hm.nt; ++t) {
    const int* f = &hm.F[3 * t];
    for (int e = 0; e < 3; ++e) {
      int p = f[e], q = f[(e + 1) % 3], r = f[(e + 2) % 3];
      if (p == q) throw AimError{AIM_ERR_MESH, "degenerate face"};
      int lo = std::min(p, q), hi = std::max(p, q);
      own.push_back({(int64_t)lo * hm.nv + hi, t, p < q ? 1 : -1, r});
    }
  }
  std::stable_sort(own.begin(), own.end(), [](const Own& a, const Own& b) { return a.key < b.key; });
  hm.edge.clear();
  hm.rtri.clear();
  hm.rfree.clear();
  for (size_t i = 0; i < own.size();) {
    size_t j = i;
    while (j < own.size() && own[j].key == own[i].key) ++j;
    if (j - i == 1) {  // boundary edge of an open surface: no basis function
      i = j;
      continue;
    }
    if (j - i != 2 || own[i].dir == own[i + 1].dir)
      throw AimError{AIM_ERR_MESH, "non-manifold or inconsistently oriented edge"};
    const Own& pl = own[i].dir > 0 ? own[i] : own[i + 1];
    const Own& mi = own[i].dir > 0 ? own[i + 1] : own[i];
    int lo = (int)(own[i].key / hm.nv), hi = (int)(own[i].key % hm.nv);
    hm.edge.push_back(lo);
    hm.edge.push_back(hi);
    hm.rtri.push_back(pl.t);
    hm.rtri.push_back(mi.t);
    hm.rfree.push_back(pl.opp);
    hm.rfree.push_back(mi.opp);
    i = j;
  }
  hm.ns = (int)hm.edge.size() / 2;
  if (hm.ns < 1) throw AimError{AIM_ERR_MESH, "no interior edge"};
  hm.len.resize(hm.ns);
  double sum = 0.0;
  for (int k = 0; k < hm.ns; ++k) {
    hm.len[k] = norm3(&hm.V[3 * hm.edge[2 * k]], &hm.V[3 * hm.edge[2 * k + 1]]);
    sum += hm.len[k];  // plain left-to-right sum
  }
  hm.mean_edge = sum / hm.ns;
  hm.area.resize(hm.nt);
  hm.cent.resize(3 * (size_t)hm.nt);
  for (int t = 0; t < hm.nt; ++t) {
    const double* a = &hm.V[3 * hm.F[3 * t]];
    const double* b = &hm.V[3 * hm.F[3 * t + 1]];
    const double* c = &hm.V[3 * hm.F[3 * t + 2]];
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double n0 = u[1] * v[2] - u[2] * v[1], n1 = u[2] * v[0] - u[0] * v[2], n2 = u[0] * v[1] - u[1] * v[0];
    hm.area[t] = 0.5 * std::sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    if (!(hm.area[t] > 0)) throw AimError{AIM_ERR_MESH, "zero-area face"};
    for (int d = 0; d < 3; ++d) hm.cent[3 * t + d] = (a[d] + b[d] + c[d]) / 3.0;
  }
  // the three half-bases of every face
  hm.tbk.assign(3 * (size_t)hm.nt, -1);
  hm.tbs.assign(3 * (size_t)hm.nt, 0.0);
  hm.tbf.assign(3 * (size_t)hm.nt, -1);
  std::vector<int> cnt(hm.nt, 0);
  for (int k = 0; k < hm.ns; ++k)
    for (int s = 0; s < 2; ++s) {
      int t = hm.rtri[2 * k + s];
      int slot = cnt[t]++;
      hm.tbk[3 * t + slot] = k;
      hm.tbs[3 * t + slot] = s == 0 ? 1.0 : -1.0;
      hm.tbf[3 * t + slot] = hm.rfree[2 * k + s];
    }
  // Cowper's 7-point degree-5 rule: centroid (9/40) and the orbits (a, a, 1-2a),
  // a = (6 -+ sqrt 15)/21 with weights (155 -+ sqrt 15)/1200.
  const double s15 = std::sqrt(15.0);
  const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
  const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
  double bary[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                       {a1, a1, 1.0 - 2.0 * a1}, {a1, 1.0 - 2.0 * a1, a1}, {1.0 - 2.0 * a1, a1, a1},
                       {a2, a2, 1.0 - 2.0 * a2}, {a2, 1.0 - 2.0 * a2, a2}, {1.0 - 2.0 * a2, a2, a2}};
  double wq[7] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};
  hm.qp.resize(21 * (size_t)hm.nt);
  hm.qw.resize(7 * (size_t)hm.nt);
  for (int t = 0; t < hm.nt; ++t) {
    const double* a = &hm.V[3 * hm.F[3 * t]];
    const double* b = &hm.V[3 * hm.F[3 * t + 1]];
    const double* c = &hm.V[3 * hm.F[3 * t + 2]];
    for (int q = 0; q < 7; ++q) {
      for (int d = 0; d < 3; ++d) hm.qp[21 * t + 3 * q + d] = bary[q][0] * a[d] + bary[q][1] * b[d] + bary[q][2] * c[d];
      hm.qw[7 * t + q] = wq[q] * hm.area[t];
    }
  }
}

// Stencil anchors: floor((x_e - origin)/h) - 1 per axis, clamped to [0, N-4].
void host_anchors(const HostMesh& hm, int N, const double* origin, double h, std::vector<int>& anchor) {
  anchor.resize(3 * (size_t)hm.ns);
  for (int k = 0; k < hm.ns; ++k) {
    const double* a = &hm.V[3 * hm.edge[2 * k]];
    const double* b = &hm.V[3 * hm.edge[2 * k + 1]];
    for (int d = 0; d < 3; ++d) {
      double xe = 0.5 * (a[d] + b[d]);
      long long i = (long long)std::floor((xe - origin[d]) / h) - 1;
      i = std::max(0LL, std::min((long long)N - 4, i));
      anchor[3 * k + d] = (int)i;
    }
  }
}

// Near pairs: |x_e(k) - x_e(k')|^2 <= r^2 (inclusive), rows sorted by column.
void host_near_pairs(const HostMesh& hm, double r, std::vector<int>& rowptr, std::vector<int>& col) {
  const int ns = hm.ns;
  rowptr.assign(ns + 1, 0);
  col.clear();
  if (r < 0) return;
  std::vector<double> xe(3 * (size_t)ns);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int k = 0; k < ns; ++k)
    for (int d = 0; d < 3; ++d) {
      xe[3 * k + d] = 0.5 * (hm.V[3 * hm.edge[2 * k] + d] + hm.V[3 * hm.edge[2 * k + 1] + d]);
      lo[d] = std::min(lo[d], xe[3 * k + d]);
      hi[d] = std::max(hi[d], xe[3 * k + d]);
    }
  double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  double cs = std::max(r, ext / 200.0);
  if (!(cs > 0)) cs = 1.0;
  int nc[3];
  for (int d = 0; d < 3; ++d) nc[d] = std::max(1, (int)std::floor((hi[d] - lo[d]) / cs) + 1);
  auto cell = [&](int k, int d) { return std::min(nc[d] - 1, (int)std::floor((xe[3 * k + d] - lo[d]) / cs)); };
  std::vector<int> cstart((size_t)nc[0] * nc[1] * nc[2] + 1, 0), members(ns);
  std::vector<int> cid(ns);
  for (int k = 0; k < ns; ++k) {
    cid[k] = (cell(k, 2) * nc[1] + cell(k, 1)) * nc[0] + cell(k, 0);
    cstart[cid[k] + 1]++;
  }
  for (size_t i = 1; i < cstart.size(); ++i) cstart[i] += cstart[i - 1];
  std::vector<int> fill(cstart.begin(), cstart.end() - 1);
  for (int k = 0; k < ns; ++k) members[fill[cid[k]]++] = k;
  const double r2 = r * r;
  // r may exceed the cell size only when the bin grid is coarse; reach covers r
  int reach = (int)std::ceil(r / cs);
  std::vector<int> row;
  for (int k = 0; k < ns; ++k) {
    row.clear();
    int c0 = cell(k, 0), c1 = cell(k, 1), c2 = cell(k, 2);
    for (int z = std::max(0, c2 - reach); z <= std::min(nc[2] - 1, c2 + reach); ++z)
      for (int y = std::max(0, c1 - reach); y <= std::min(nc[1] - 1, c1 + reach); ++y)
        for (int x = std::max(0, c0 - reach); x <= std::min(nc[0] - 1, c0 + reach); ++x) {
          int id = (z * nc[1] + y) * nc[0] + x;
          for (int i = cstart[id]; i < cstart[id + 1]; ++i) {
            int j = members[i];
            double dx = xe[3 * k] - xe[3 * j], dy = xe[3 * k + 1] - xe[3 * j + 1], dz = xe[3 * k + 2] - xe[3 * j + 2];
            double d2 = dx * dx + dy * dy + dz * dz;
            if (d2 <= r2) row.push_back(j);
          }
        }
    std::sort(row.begin(), row.end());
    col.insert(col.end(), row.begin(), row.end());
    rowptr[k + 1] = (int)col.size();
  }
}

// Transposed anterpolation pattern: for every grid node, the (rwg, slot) entries
// in increasing rwg order.  slot t = (dz*4 + dy)*4 + dx.
void host_transpose_pattern(int N, const std::vector<int>& anchor, int ns, std::vector<int>& nptr,
                            std::vector<int>& nidx, std::vector<int>& nslot) {
  const size_t nn = (size_t)N * N * N;
  nptr.assign(nn + 1, 0);
  auto node = [&](int k, int t) {
    int dx = t & 3, dy = (t >> 2) & 3, dz = t >> 4;
    return ((size_t)(anchor[3 * k + 2] + dz) * N + (anchor[3 * k + 1] + dy)) * N + (anchor[3 * k] + dx);
  };
  for (int k = 0; k < ns; ++k)
    for (int t = 0; t < 64; ++t) nptr[node(k, t) + 1]++;
  for (size_t i = 1; i <= nn; ++i) nptr[i] += nptr[i - 1];
  std::vector<int> fill(nptr.begin(), nptr.end() - 1);
  nidx.resize((size_t)64 * ns);
  nslot.resize((size_t)64 * ns);
  for (int k = 0; k < ns; ++k)
    for (int t = 0; t < 64; ++t) {
      size_t n = node(k, t);
      nidx[fill[n]] = k;
      nslot[fill[n]] = t;
      fill[n]++;
    }
}

// Candidate nodes for the largest node-to-node distance: the end points of every
// grid line along x, y and z through the active set (every vertex of the convex
// hull of the active nodes is one of them).
void host_extreme_candidates(int N, const std::vector<int>& nptr, std::vector<int>& cand, int& n_active) {
  const size_t nn = (size_t)N * N * N;
  std::vector<uint8_t> mark(nn, 0);
  n_active = 0;
  auto act = [&](size_t n) { return nptr[n + 1] > nptr[n]; };
  for (size_t n = 0; n < nn; ++n) n_active += act(n) ? 1 : 0;
  for (int axis = 0; axis < 3; ++axis)
    for (int a = 0; a < N; ++a)
      for (int b = 0; b < N; ++b) {
        int first = -1, last = -1;
        for (int i = 0; i < N; ++i) {
          int ix = axis == 0 ? i : a, iy = axis == 1 ? i : (axis == 0 ? a : b), iz = axis == 2 ? i : b;
          size_t n = ((size_t)iz * N + iy) * N + ix;
          if (act(n)) {
            if (first < 0) first = (int)n;
            last = (int)n;
          }
        }
        if (first >= 0) {
          mark[first] = 1;
          mark[last] = 1;
        }
      }
  cand.clear();
  for (size_t n = 0; n < nn; ++n)
    if (mark[n]) cand.push_back((int)n);
}

// CPPIF piece polynomials (Sec. 3, Eq. 3): on (j-1, j],
// T(u) = prod_{k != j} (u - j + k)/(k - j), expanded in ascending powers of u.
void host_cppif(int Q, TBasis& tb) {
  if (Q < 1 || Q > aimc::kMaxOrder) throw AimError{AIM_ERR_ARG, "CPPIF order must be 1..4"};
  std::memset(&tb, 0, sizeof(tb));
  tb.kind = AIM_CPPIF;
  tb.Q = Q;
  for (int j = 0; j <= Q; ++j) {
    double c[aimc::kMaxOrder + 1] = {1.0};
    int deg = 0;
    for (int k = 0; k <= Q; ++k) {
      if (k == j) continue;
      double a0 = 1.0, a1 = 1.0 / (double)(k - j);  // (u + (k - j)) / (k - j)
      double nc[aimc::kMaxOrder + 1] = {0};
      for (int p = 0; p <= deg; ++p) {
        nc[p] += c[p] * a0;
        nc[p + 1] += c[p] * a1;
      }
      ++deg;
      for (int p = 0; p <= deg; ++p) c[p] = nc[p];
    }
    for (int p = 0; p <= Q; ++p) tb.coef[j][p] = c[p];
  }
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
// BLIF of half-width M for the band fraction beta = f_bw dt (Sec. 3.1.2): guard band
// b = pi (1 - 2 beta), 1/G(M^2) = M / sinh(b M), and the extrapolation weights.  Each row
// ext[p] (p = 1..M-1) is the least-squares fit of exp(j w_n p) by sum_q ext[p][q]
// exp(-j w_n q), q = 0..M-1, over the 2M frequencies w_n = 2 pi beta (-1 + 2n/(2M-1)).  The
// frequency set is symmetric, so the solution is real: it is the least-squares solution of
// the real system [cos(w_n q); -sin(w_n q)] e = [cos(w_n p); sin(w_n p)] (4M rows), solved
// here by Gram-Schmidt with one re-orthogonalisation and back substitution.
void host_blif(int M, double beta, TBasis& tb) {
  if (M < 2 || M > aimc::kMaxHalfWidth) throw AimError{AIM_ERR_ARG, "BLIF half-width must be 2..5"};
  if (!(beta > 0.0 && beta < 0.5)) throw AimError{AIM_ERR_ARG, "blif_band (f_bw dt) must lie in (0, 1/2)"};
  std::memset(&tb, 0, sizeof(tb));
  tb.kind = AIM_BLIF;
  tb.Q = M;
  tb.b = aimc::kPi * (1.0 - 2.0 * beta);
  tb.invG0 = (double)M / std::sinh(tb.b * M);
  const int nw = 2 * M, rows = 2 * nw;
  std::vector<double> A((size_t)rows * M), Q((size_t)rows * M), R((size_t)M * M, 0.0);
  for (int n = 0; n < nw; ++n) {
    const double w = 2.0 * aimc::kPi * beta * (-1.0 + 2.0 * n / (double)(nw - 1));
    for (int q = 0; q < M; ++q) {
      A[(size_t)n * M + q] = std::cos(w * q);
      A[(size_t)(nw + n) * M + q] = -std::sin(w * q);
    }
  }
  Q = A;
  for (int j = 0; j < M; ++j) {
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i < j; ++i) {
        double d = 0.0;
        for (int r = 0; r < rows; ++r) d += Q[(size_t)r * M + i] * Q[(size_t)r * M + j];
        R[(size_t)i * M + j] += d;
        for (int r = 0; r < rows; ++r) Q[(size_t)r * M + j] -= d * Q[(size_t)r * M + i];
      }
    double nrm = 0.0;
    for (int r = 0; r < rows; ++r) nrm += Q[(size_t)r * M + j] * Q[(size_t)r * M + j];
    nrm = std::sqrt(nrm);
    R[(size_t)j * M + j] = nrm;
    for (int r = 0; r < rows; ++r) Q[(size_t)r * M + j] /= nrm;
  }
  for (int p = 1; p < M; ++p) {
    std::vector<double> rhs(rows), y(M, 0.0);
    for (int n = 0; n < nw; ++n) {
      const double w = 2.0 * aimc::kPi * beta * (-1.0 + 2.0 * n / (double)(nw - 1));
      rhs[n] = std::cos(w * p);
      rhs[nw + n] = std::sin(w * p);
    }
    for (int j = 0; j < M; ++j)
      for (int r = 0; r < rows; ++r) y[j] += Q[(size_t)r * M + j] * rhs[r];
    for (int j = M - 1; j >= 0; --j) {
      double s = y[j];
      for (int i = j + 1; i < M; ++i) s -= R[(size_t)j * M + i] * tb.ext[p][i];
      tb.ext[p][j] = s / R[(size_t)j * M + j];
    }
  }
}

// T(u) of the BLIF on the host (values only): sinc(u) sinh(b sqrt(M^2 - u^2)) /
// sqrt(M^2 - u^2) / G(M^2), the limit b / G(M^2) at |u| = M
double host_blif_value(const TBasis& tb, double u) {
  const double M = tb.Q;
  if (!(std::fabs(u) < M)) return 0.0;
  const double x = aimc::kPi * u;
  const double sinc = std::fabs(x) < 1e-8 ? 1.0 - x * x / 6.0 : std::sin(x) / x;
  const double r = std::sqrt(M * M - u * u);
  const double g = r < 1e-12 ? tb.b : std::sinh(tb.b * r) / r;
  return sinc * g * tb.invG0;
}

void host_gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(aimc::kPi * (i + 0.75) / (n + 0.5)), dp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}
