// Host-side setup bookkeeping shared by api.cu and setup_gpu.cu.
#pragma once
#include <vector>

#include "aim_internal.h"

struct HostMesh {
  int nv = 0, nt = 0, ns = 0;
  std::vector<double> V;      // [nv][3]
  std::vector<int> F;         // [nt][3]
  std::vector<int> edge;      // [ns][2]
  std::vector<int> rtri;      // [ns][2]
  std::vector<int> rfree;     // [ns][2]
  std::vector<double> len;    // [ns]
  std::vector<double> area;   // [nt]
  std::vector<double> cent;   // [nt][3]
  std::vector<int> tbk;       // [nt][3]
  std::vector<double> tbs;    // [nt][3]
  std::vector<int> tbf;       // [nt][3]
  std::vector<double> qp;     // [nt][7][3]
  std::vector<double> qw;     // [nt][7]
  double mean_edge = 0;
};

void host_build_rwg(const aim_mesh* m, HostMesh& hm);
void host_anchors(const HostMesh& hm, int N, const double* origin, double h, std::vector<int>& anchor);
void host_near_pairs(const HostMesh& hm, double r, std::vector<int>& rowptr, std::vector<int>& col);
void host_transpose_pattern(int N, const std::vector<int>& anchor, int ns, std::vector<int>& nptr,
                            std::vector<int>& nidx, std::vector<int>& nslot);
void host_extreme_candidates(int N, const std::vector<int>& nptr, std::vector<int>& cand, int& n_active);
void host_cppif(int Q, TBasis& tb);
void host_blif(int M, double beta, TBasis& tb);
double host_blif_value(const TBasis& tb, double u);
void host_gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
