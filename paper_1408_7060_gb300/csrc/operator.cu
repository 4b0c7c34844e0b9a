// Precision dispatch of the operator and the excitation kernel (Eq. 1).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <string>

#include <sys/stat.h>

#include "aim_internal.h"
#include "operator.h"

template <class C>
void body_apply(aim_ctx*, int, int, const double2*, const double2*, const double2*, double, const int*, double2*,
                VecSel, VecSel);
template <class C>
void body_forward_slab(aim_ctx*, int, const double2*, void*);
template <class C>
void body_apply_rhs(aim_ctx*, int, const SlabList&, const NearList&, const double2*, double, double2*);
template <class C>
void body_apply_rhs_pending(aim_ctx*, int, void*, const NearList&, const double2*, double, double2*);
template <class C>
void body_block_square(aim_ctx*, int, const BlockSquare&);
template <class C>
void body_tune(aim_ctx*);
template <class C>
void body_plan_fill(aim_ctx*);

void op_apply(aim_ctx* c, int m, int nb, const double2* v, const double2* dinv, const double2* base, double sign,
              const int* active, double2* y, VecSel vin, VecSel yout) {
  if (c->precision == AIM_C64)
    body_apply<float2>(c, m, nb, v, dinv, base, sign, active, y, vin, yout);
  else
    body_apply<double2>(c, m, nb, v, dinv, base, sign, active, y, vin, yout);
}

void op_apply_f64(aim_ctx* c, int m, int nb, const double2* v, const double2* base, double sign, double2* y) {
  if (c->precision == AIM_C128) {
    op_apply(c, m, nb, v, nullptr, base, sign, nullptr, y);
    return;
  }
  if (!c->d_A64 || c->ref_nb < 1) throw AimError{AIM_ERR_ARG, "FP64 operator: refinement buffers not set up"};
  // the FP64 grid buffers stand in for the context's complex64 ones for the duration
  struct Swap {
    aim_ctx* c;
    void *A, *Bf, *P, *xs;
    explicit Swap(aim_ctx* c_) : c(c_), A(c_->d_A), Bf(c_->d_Bf), P(c_->d_P), xs(c_->d_xs) {
      c->d_A = c->d_A64;
      c->d_Bf = c->d_Bf64;
      c->d_P = c->d_P64;
      c->d_xs = c->d_xs64;
    }
    ~Swap() {
      c->d_A = A;
      c->d_Bf = Bf;
      c->d_P = P;
      c->d_xs = xs;
    }
  } sw(c);
  const size_t ns = c->ns;
  for (int b0 = 0; b0 < nb; b0 += c->ref_nb) {
    const int n = std::min(c->ref_nb, nb - b0);
    body_apply<double2>(c, m, n, v + b0 * ns, nullptr, base ? base + b0 * ns : nullptr, sign, nullptr, y + b0 * ns,
                        VecSel(), VecSel());
  }
}

void op_forward_slab(aim_ctx* c, int nb, const double2* v, void* dst) {
  if (c->precision == AIM_C64)
    body_forward_slab<float2>(c, nb, v, dst);
  else
    body_forward_slab<double2>(c, nb, v, dst);
}

void op_apply_rhs(aim_ctx* c, int nb, const SlabList& sl, const NearList& nl, const double2* base, double sign,
                  double2* y) {
  if (c->precision == AIM_C64)
    body_apply_rhs<float2>(c, nb, sl, nl, base, sign, y);
  else
    body_apply_rhs<double2>(c, nb, sl, nl, base, sign, y);
}

void op_apply_rhs_pending(aim_ctx* c, int nb, void* P, const NearList& nl, const double2* base, double sign,
                          double2* y) {
  if (c->precision == AIM_C64)
    body_apply_rhs_pending<float2>(c, nb, P, nl, base, sign, y);
  else
    body_apply_rhs_pending<double2>(c, nb, P, nl, base, sign, y);
}

void op_block_square(aim_ctx* c, int nb, const BlockSquare& sq) {
  if (c->precision == AIM_C64)
    body_block_square<float2>(c, nb, sq);
  else
    body_block_square<double2>(c, nb, sq);
}

// ---------------------------------------------------------------- launch plans
// The plan cache: one JSON object per line,
//   {"key": "<gpu name>|L=<L>|LZ=<LZ>|prec=<c64|c128>|nb=<batch>", "zw": .., "cw": .., "rp": .., "ypb": ..}
// in the file named by AIM_GB300_PLAN_CACHE, else $HOME/.cache/aim_gb300_plans.jsonl.
namespace {
std::string plan_cache_path() {
  if (const char* e = std::getenv("AIM_GB300_PLAN_CACHE")) return e;
  if (const char* h = std::getenv("HOME")) return std::string(h) + "/.cache/aim_gb300_plans.jsonl";
  return "";
}

std::string plan_key(const aim_ctx* c) {
  int dev = 0;
  cudaDeviceProp prop;
  std::string name = "gpu";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  cudaGetLastError();
  for (char& ch : name)
    if (ch == '"' || ch == '|') ch = '_';
  return name + "|L=" + std::to_string(c->L) + "|LZ=" + std::to_string(c->LZ) + "|prec=" + (c->precision == AIM_C64 ? "c64" : "c128") +
         "|nb=" + std::to_string(c->batch_max);
}

int json_int(const std::string& line, const char* field) {
  const std::string f = std::string("\"") + field + "\":";
  const size_t p = line.find(f);
  return p == std::string::npos ? 0 : std::atoi(line.c_str() + p + f.size());
}

bool read_plan(const std::string& path, const std::string& key, KPlan& plan) {
  std::ifstream in(path);
  std::string line;
  bool found = false;
  while (std::getline(in, line)) {  // the last line with the key wins
    if (line.find("\"key\": \"" + key + "\"") == std::string::npos) continue;
    KPlan p;
    p.zw = json_int(line, "zw");
    p.cw = json_int(line, "cw");
    p.rp = json_int(line, "rp");
    p.ypb = json_int(line, "ypb");
    if (p.zw > 0 && p.cw > 0 && p.rp > 0 && p.ypb > 0) {
      plan = p;
      found = true;
    }
  }
  return found;
}

void append_plan(const std::string& path, const std::string& key, const KPlan& p) {
  const size_t slash = path.find_last_of('/');
  if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);  // may exist
  std::ofstream out(path, std::ios::app);
  if (!out) return;  // the cache is an optimisation: an unwritable path is not an error
  out << "{\"key\": \"" << key << "\", \"zw\": " << p.zw << ", \"cw\": " << p.cw << ", \"rp\": " << p.rp
      << ", \"ypb\": " << p.ypb << "}\n";
}
}  // namespace

void op_autotune(aim_ctx* c, int mode) {
  c->plan = KPlan();
  if (mode > 0) {
    const std::string path = plan_cache_path(), key = plan_key(c);
    KPlan p;
    if (mode == 1 && !path.empty() && read_plan(path, key, p)) {
      p.source = AIM_PLAN_CACHED;
      c->plan = p;
    } else {
      if (c->precision == AIM_C64)
        body_tune<float2>(c);
      else
        body_tune<double2>(c);
      c->plan.source = AIM_PLAN_MEASURED;
      if (!path.empty()) append_plan(path, key, c->plan);
    }
  }
  // the shapes in use, defaults included (reported by aim_get_info)
  if (c->precision == AIM_C64)
    body_plan_fill<float2>(c);
  else
    body_plan_fill<double2>(c);
}

// kernels one operator application launches: prep, anterp + x, y, z, y^-1, x^-1, interp
int op_kernel_count(const aim_ctx*) { return 7; }

size_t grid_a_elems(const aim_ctx* c, int nb) { return (size_t)nb * 4 * c->NZ * c->N * c->L; }
size_t grid_bf_elems(const aim_ctx* c, int nb) { return (size_t)nb * 4 * c->NZ * c->L * c->L; }
size_t grid_p_elems(const aim_ctx* c, int nb) { return (size_t)nb * 4 * c->NZ * c->N * c->N; }

// bytes of one history slab: [nb][4][Z][L][L] with Z = LZ (z-transformed, power-of-two
// LZ) or NZ (x/y-transformed only)
size_t op_slab_bytes(const aim_ctx* c, int nb) {
  const int L = c->L, Z = (c->LZ & (c->LZ - 1)) == 0 ? c->LZ : c->NZ;
  return (size_t)nb * 4 * Z * (size_t)L * L * (c->precision == AIM_C64 ? sizeof(float2) : sizeof(double2));
}

// V_l[k] = <S_k, p (g'(tau) + j w g(tau)) e^{-j w (r.k/c + t_d)}>,  tau = l dt - r.k/c - t_d,
// g = exp(-tau^2/(2 sigma^2)): the envelope of D E^inc for the plane wave of Eq. 1.
// 16 lanes per (b, k): lane l < 14 takes quadrature point q = l % 7 of side l / 7; the
// 16 contributions are summed by a fixed xor-butterfly.
__global__ void __launch_bounds__(128) k_excitation(int ns, int nb, const int* __restrict__ rtri,
                                                    const int* __restrict__ rfree, const double* __restrict__ len,
                                                    const double* __restrict__ area, const double* __restrict__ V,
                                                    const double* __restrict__ qp, const double* __restrict__ qw,
                                                    const double* __restrict__ kp, double sigma, double t_d, double t,
                                                    double wc, double c0, double2* __restrict__ out) {
  const long long g16 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 4;
  const int l = threadIdx.x & 15;
  const bool valid = g16 < (long long)ns * nb;  // both groups of a warp join the shuffles
  const int b = valid ? (int)(g16 / ns) : 0, k = valid ? (int)(g16 % ns) : 0;
  const double* kh = kp + 6 * b;
  const double* ph = kh + 3;
  double2 acc = make_double2(0, 0);
  if (valid && l < 14) {
    const int side = l / 7, q = l % 7;
    const int tr = rtri[2 * k + side];
    const double* vf = V + 3 * rfree[2 * k + side];
    const double cS = (side == 0 ? 1.0 : -1.0) * len[k] / (2.0 * area[tr]);
    const double* r = qp + 21 * tr + 3 * q;
    const double delay = (r[0] * kh[0] + r[1] * kh[1] + r[2] * kh[2]) / c0;
    const double tau = t - delay - t_d;
    const double g = exp(-tau * tau / (2.0 * sigma * sigma));
    double sn, cph;
    sincos(-wc * (delay + t_d), &sn, &cph);
    // (-tau/sigma^2 + j w) g e^{j phase}
    const double ar = -tau / (sigma * sigma) * g, ai = wc * g;
    const double sp = cS * ((r[0] - vf[0]) * ph[0] + (r[1] - vf[1]) * ph[1] + (r[2] - vf[2]) * ph[2]);
    const double w = qw[7 * tr + q] * sp;
    acc = make_double2(w * (ar * cph - ai * sn), w * (ar * sn + ai * cph));
  }
  for (int o = 8; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (valid && l == 0) out[(size_t)b * ns + k] = acc;
}

void op_excitation(aim_ctx* c, int nb, const double* d_kp, double sigma, double t_d, int step_l, double2* out) {
  const long long n = (long long)c->ns * nb * 16;
  KScope ks(c, AIM_K_EXCITATION);
  k_excitation<<<(int)((n + 127) / 128), 128, 0, c->stream>>>(c->ns, nb, c->d_rtri, c->d_rfree, c->d_len, c->d_area,
                                                      c->d_v, c->d_qp, c->d_qw, d_kp, sigma, t_d,
                                                      step_l * c->dt, c->wc, c->c_med, out);
  AIM_CHECK_LAUNCH();
}
