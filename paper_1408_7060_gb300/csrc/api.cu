// extern "C" entry points of the ET-AIM library (declared in include/aim.h).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "aim_internal.h"
#include "gmres.h"
#include "tma.cuh"
#include "operator.h"
#include "rcs.h"
#include "setup_gpu.h"
#include "setup_host.h"
#include "tbasis.cuh"

namespace {

void ensure_ring(aim_ctx* c);

thread_local std::string g_last_setup_error;

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class F>
int guard(aim_ctx* c, F&& f) {
  try {
    return f();
  } catch (const AimError& e) {
    if (c) c->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    if (c) c->err = "host allocation failed";
    return AIM_ERR_OOM;
  } catch (...) {
    if (c) c->err = "unexpected exception";
    return AIM_ERR_ARG;
  }
}

bool supported_n(int n) {
  return n == 8 || n == 16 || n == 32 || n == 64 || n == 96 || n == 128 || n == 384;
}

template <class T>
T* upload(aim_ctx* c, const std::vector<T>& v) {
  T* d = (T*)aim_alloc(c, std::max<size_t>(1, v.size()) * sizeof(T));
  if (!v.empty()) AIM_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  return d;
}

size_t grid_elem(const aim_ctx* c) { return c->precision == AIM_C64 ? sizeof(float2) : sizeof(double2); }

// z transform length for nz box planes: the shortest length of the z pass >= 2 nz (at most
// the padded length L = 2N >= 2 nz)
static int z_length(int nz, int L) {
  for (int lz : {16, 32, 64, 128, 192, 256, 768})
    if (lz >= 2 * nz && lz <= L) return lz;
  return L;
}

void setup_impl(aim_ctx* c, const aim_mesh* mesh, const aim_grid* grid, double near_radius, double dt,
                aim_tbasis tb, const aim_opts* opts) {
  if (!mesh || !grid || !opts) throw AimError{AIM_ERR_ARG, "null argument"};
  if (!supported_n(grid->n)) throw AimError{AIM_ERR_ARG, "grid n must be one of 8,16,32,64,96,128,384"};
  if (!(grid->h > 0) || !(dt > 0) || !(opts->f_c > 0)) throw AimError{AIM_ERR_ARG, "h, dt and f_c must be > 0"};
  if (tb.kind != AIM_CPPIF && tb.kind != AIM_BLIF) throw AimError{AIM_ERR_ARG, "temporal basis: AIM_CPPIF or AIM_BLIF"};
  if (opts->precision != AIM_C64 && opts->precision != AIM_C128) throw AimError{AIM_ERR_ARG, "precision"};
  if (opts->batch_max < 1 || opts->batch_max > 4096) throw AimError{AIM_ERR_ARG, "batch_max out of range"};
  c->N = grid->n;
  c->L = 2 * grid->n;
  c->h = grid->h;
  for (int d = 0; d < 3; ++d) c->origin[d] = grid->origin[d];
  c->dt = dt;
  c->f_c = opts->f_c;
  c->wc = 2.0 * aimc::kPi * opts->f_c;
  {
    const double er = opts->eps_r > 0 ? opts->eps_r : 1.0, mr = opts->mu_r > 0 ? opts->mu_r : 1.0;
    c->c_med = aimc::kC0 / std::sqrt(er * mr);
    c->mu_med = aimc::kMu0 * mr;
    c->eps_med = aimc::kEps0 * er;
  }
  c->kc = c->wc / c->c_med;
  c->near_radius = near_radius;
  c->precision = opts->precision;
  c->batch_max = opts->batch_max;
  c->restart = opts->gmres_restart > 0 ? std::min(opts->gmres_restart, 63) : 50;
  c->max_iter = opts->gmres_max_iter > 0 ? opts->gmres_max_iter : 500;
  if (opts->preconditioner != AIM_PRECOND_DIAG && opts->preconditioner != AIM_PRECOND_NEAR_SAI)
    throw AimError{AIM_ERR_ARG, "aim_setup: unknown preconditioner"};
  c->precond = opts->preconditioner;
  c->zero_start = opts->zero_start != 0;
  if (opts->refine < 0 || opts->refine > 64) throw AimError{AIM_ERR_ARG, "aim_setup: refine out of range"};
  c->refine = opts->precision == AIM_C64 ? opts->refine : 0;
  c->refine_every = std::max(1, opts->refine_every);
  c->rhs_blocked = opts->rhs_blocked != 0;
  c->precond_radius = opts->precond_radius > 0 ? opts->precond_radius : near_radius;
  if (c->precond == AIM_PRECOND_NEAR_SAI && c->precond_radius < 0)
    throw AimError{AIM_ERR_ARG, "aim_setup: the SAI preconditioner needs a pattern radius or a near zone"};
  {
    const char* e = std::getenv("AIM_GB300_GRAPHS");  // "0": drive the solver from the host
    c->use_graphs = !(e && e[0] == '0');
  }
  if (opts->cuda_stream) {
    c->stream = (cudaStream_t)opts->cuda_stream;
  } else {
    AIM_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  if (tb.kind == AIM_BLIF)
    host_blif(tb.order, opts->blif_band, c->tb);
  else
    host_cppif(tb.order, c->tb);

  HostMesh hm;
  host_build_rwg(mesh, hm);
  c->nv = hm.nv;
  c->nt = hm.nt;
  c->ns = hm.ns;
  c->mean_edge = hm.mean_edge;
  for (int i = 0; i < hm.nv; ++i)
    c->rmax = std::max(c->rmax, std::sqrt(hm.V[3 * i] * hm.V[3 * i] + hm.V[3 * i + 1] * hm.V[3 * i + 1] +
                                          hm.V[3 * i + 2] * hm.V[3 * i + 2]));
  c->h_edge = hm.edge;
  c->h_tri = hm.rtri;
  c->h_free = hm.rfree;
  std::vector<int> anchor;
  host_anchors(hm, c->N, c->origin, c->h, anchor);
  for (int d = 0; d < 3; ++d) {  // the active box: every stencil spans anchor .. anchor + 3
    c->box_lo[d] = c->N - 4;
    c->box_hi[d] = 3;
  }
  for (int k = 0; k < hm.ns; ++k)
    for (int d = 0; d < 3; ++d) {
      c->box_lo[d] = std::min(c->box_lo[d], anchor[3 * k + d]);
      c->box_hi[d] = std::max(c->box_hi[d], anchor[3 * k + d] + 3);
    }
  c->NZ = c->box_hi[2] - c->box_lo[2] + 1;
  c->LZ = z_length(c->NZ, c->L);

  c->d_v = upload(c, hm.V);
  c->d_tri = upload(c, hm.F);
  c->d_rtri = upload(c, hm.rtri);
  c->d_rfree = upload(c, hm.rfree);
  c->d_len = upload(c, hm.len);
  c->d_area = upload(c, hm.area);
  c->d_cent = upload(c, hm.cent);
  c->d_qp = upload(c, hm.qp);
  c->d_qw = upload(c, hm.qw);
  c->d_tbk = upload(c, hm.tbk);
  c->d_tbs = upload(c, hm.tbs);
  c->d_tbf = upload(c, hm.tbf);
  c->d_anchor = upload(c, anchor);
  {
    // interpolation visit order: RWGs sorted by the Morton code of their stencil anchors,
    // so that the warps of one block gather from neighbouring grid rows (L2 reuse)
    auto spread = [](uint64_t v) {  // 21 bits -> every third bit
      v &= 0x1fffff;
      v = (v | v << 32) & 0x1f00000000ffffULL;
      v = (v | v << 16) & 0x1f0000ff0000ffULL;
      v = (v | v << 8) & 0x100f00f00f00f00fULL;
      v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
      v = (v | v << 2) & 0x1249249249249249ULL;
      return v;
    };
    std::vector<uint64_t> key(hm.ns);
    std::vector<int> order(hm.ns);
    for (int k = 0; k < hm.ns; ++k) {
      key[k] = spread((uint64_t)anchor[3 * k]) | spread((uint64_t)anchor[3 * k + 1]) << 1 |
               spread((uint64_t)anchor[3 * k + 2]) << 2;
      order[k] = k;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
    c->d_order = upload(c, order);
  }
  c->d_lam = (double*)aim_alloc(c, (size_t)c->ns * 256 * sizeof(double));
  c->d_lamf = (float*)aim_alloc(c, (size_t)c->ns * 256 * sizeof(float));
  AIM_CUDA(cudaStreamSynchronize(c->stream));

  setup_device_tables(c, hm, anchor);
  if (c->rhs_blocked) {
    if ((c->LZ & (c->LZ - 1)) != 0)
      throw AimError{AIM_ERR_ARG, "aim_setup: the blocked right-hand side needs a power-of-two z transform"};
    while ((1 << c->blk_P) < c->n_delays) ++c->blk_P;  // 2^P >= N_g (<= 32)
  }

  // work buffers
  const int B = c->batch_max, ns = c->ns, ng = c->n_delays;
  const size_t es = grid_elem(c);
  c->d_A = aim_alloc(c, grid_a_elems(c, B) * es);
  c->d_Bf = aim_alloc(c, grid_bf_elems(c, B) * es);
  c->d_P = aim_alloc(c, grid_p_elems(c, B) * es);
  c->d_xs = aim_alloc(c, (size_t)B * ns * es);
  c->d_xd = (double2*)aim_alloc(c, (size_t)B * ns * sizeof(double2));
  c->d_vf = (float2*)aim_alloc(c, (size_t)B * ns * sizeof(float2));
  const size_t vec = (size_t)B * ns * sizeof(double2);
  c->d_iring = (double2*)aim_alloc(c, (size_t)ng * vec);
  c->d_x = (double2*)aim_alloc(c, vec);
  c->d_y = (double2*)aim_alloc(c, vec);
  c->d_b = (double2*)aim_alloc(c, vec);
  c->d_r = (double2*)aim_alloc(c, vec);
  c->d_w = (double2*)aim_alloc(c, vec);
  c->d_err = (int*)aim_alloc(c, sizeof(int));
  AIM_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  if (c->d_sai) c->d_u = (double2*)aim_alloc(c, vec);
  c->d_V = (double2*)aim_alloc(c, (size_t)(c->restart + 1) * vec);
  c->d_hist = (double2*)aim_alloc(c, (size_t)ng * vec);
  c->d_exc = (double*)aim_alloc(c, (size_t)B * 6 * sizeof(double));
  if (c->refine > 0) {
    // FP64 grid buffers for the refinement residual, for as many right-hand sides at a
    // time as fit in 8 GiB (at least one)
    const size_t per = (grid_a_elems(c, 1) + grid_bf_elems(c, 1) + grid_p_elems(c, 1)) * sizeof(double2);
    c->ref_nb = (int)std::max<size_t>(1, std::min<size_t>((size_t)B, (size_t(8) << 30) / per));
    const int rb = c->ref_nb;
    c->d_A64 = aim_alloc(c, grid_a_elems(c, rb) * sizeof(double2));
    c->d_Bf64 = aim_alloc(c, grid_bf_elems(c, rb) * sizeof(double2));
    c->d_P64 = aim_alloc(c, grid_p_elems(c, rb) * sizeof(double2));
    c->d_xs64 = aim_alloc(c, (size_t)rb * ns * sizeof(double2));
    c->d_rn = (double*)aim_alloc(c, 2 * (size_t)B * sizeof(double));
    AIM_CUDA(cudaMallocHost(&c->h_rn, 2 * (size_t)B * sizeof(double)));
  }
  gmres_alloc(c);
  if (opts->autotune < 0 || opts->autotune > 2) throw AimError{AIM_ERR_ARG, "aim_setup: autotune must be 0, 1 or 2"};
  op_autotune(c, opts->autotune);
  // run every operator kernel once outside any stream capture: sets the shared-memory
  // attributes of each instantiation and surfaces launch errors at setup
  AIM_CUDA(cudaMemsetAsync(c->d_x, 0, vec, c->stream));
  op_apply(c, 0, 1, c->d_x, nullptr, nullptr, 1.0, nullptr, c->d_y);
  if (c->refine > 0) op_apply_f64(c, 0, 1, c->d_x, nullptr, 1.0, c->d_y);
  ensure_ring(c);
  op_forward_slab(c, 1, c->d_x, c->d_ring);
  {
    SlabList sl{};
    sl.p[0] = c->d_ring;
    sl.m[0] = 1;
    sl.n = 1;
    NearList nl{};
    op_apply_rhs(c, 1, sl, nl, nullptr, 1.0, c->d_y);
  }
  AIM_CUDA(cudaStreamSynchronize(c->stream));
  c->prof = ProfState();
}

// the spectral history ring (N_g forward slabs per right-hand side) is the largest
// buffer; it is allocated on the first call that needs it
void ensure_ring(aim_ctx* c) {
  if (c->d_ring) return;
  const size_t slab = op_slab_bytes(c, c->batch_max);
  // blocked sums: 2^P >= N_g source slots and 2^(P+1) pending slots
  const int nslots = c->rhs_blocked ? 1 << c->blk_P : c->n_delays;
  c->d_ring = aim_alloc(c, (size_t)nslots * slab);
  if (c->rhs_blocked) {
    c->d_pend = aim_alloc(c, ((size_t)2 << c->blk_P) * slab);
    AIM_CUDA(cudaMemsetAsync(c->d_pend, 0, ((size_t)2 << c->blk_P) * slab, c->stream));
  }
  // TMA view for the complex64 delayed sum over the z-spectra: [slot][B*4*LZ][L][L],
  // boxes of 16 x 1 x LZ x 1
  const int L = c->L, LZ = c->LZ;
  if (c->precision == AIM_C64 && (LZ & (LZ - 1)) == 0 && LZ <= 256 && L <= 256) {
    const cuuint64_t dims[4] = {(cuuint64_t)L, (cuuint64_t)L, (cuuint64_t)c->batch_max * 4 * LZ,
                                (cuuint64_t)c->n_delays};
    const cuuint64_t strides[3] = {(cuuint64_t)L * 8, (cuuint64_t)L * L * 8, (cuuint64_t)slab};
    const cuuint32_t box[4] = {(cuuint32_t)(L < 16 ? L : 16), 1, (cuuint32_t)LZ, 1};
    c->ring_tma = encode_tiled_map(&c->ring_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, c->d_ring, dims, strides, box);
  }
}

// copy a caller array to device staging if it is a host pointer
const double2* stage_in(aim_ctx* c, const aim_c128* p, size_t n, double2* staging) {
  if (is_device_ptr(p)) return reinterpret_cast<const double2*>(p);
  AIM_CUDA(cudaMemcpyAsync(staging, p, n * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
  return staging;
}

void upload_waves(aim_ctx* c, const aim_excitation* exc) {
  if (!exc || !exc->khat || !exc->phat || exc->nb < 1 || exc->nb > c->batch_max)
    throw AimError{AIM_ERR_ARG, "excitation: nb out of range or null directions"};
  if (!(exc->sigma > 0)) throw AimError{AIM_ERR_ARG, "excitation: sigma must be > 0"};
  std::vector<double> kp((size_t)exc->nb * 6);
  for (int b = 0; b < exc->nb; ++b)
    for (int d = 0; d < 3; ++d) {
      kp[6 * b + d] = exc->khat[3 * b + d];
      kp[6 * b + 3 + d] = exc->phat[3 * b + d];
    }
  AIM_CUDA(cudaMemcpyAsync(c->d_exc, kp.data(), kp.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  AIM_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace

void* aim_alloc(aim_ctx* c, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw AimError{AIM_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e)};
  }
  c->allocs.push_back(p);
  c->device_bytes += bytes;
  return p;
}

KScope::KScope(aim_ctx* c_, int id_) : c(c_), id(id_) {
  c->prof.launches++;
  c->prof.n[id]++;
  if (c->prof.on) {
    if (c->prof.pool.empty()) {
      cudaEvent_t e;
      AIM_CUDA(cudaEventCreate(&e));
      c->prof.pool.push_back(e);
    }
    a = c->prof.pool.back();
    c->prof.pool.pop_back();
    cudaEventRecord(a, c->stream);
  }
}

KScope::~KScope() {
  if (!a) return;
  cudaEvent_t b;
  if (c->prof.pool.empty()) {
    if (cudaEventCreate(&b) != cudaSuccess) return;
  } else {
    b = c->prof.pool.back();
    c->prof.pool.pop_back();
  }
  cudaEventRecord(b, c->stream);
  c->prof.pending.push_back({id, a, b});
}

void prof_flush(aim_ctx* c) {
  for (auto& r : c->prof.pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) c->prof.ms[r.id] += ms;
    c->prof.pool.push_back(r.a);
    c->prof.pool.push_back(r.b);
  }
  c->prof.pending.clear();
  cudaGetLastError();
}

// Where the right-hand side b of each step of a march comes from and where its currents
// go.  Steps are counted j = 1..n_steps within one call.  With rev, the explicit sources
// are read and the currents stored in reversed order (j <-> n_steps + 1 - j) and
// conjugated: the adjoint march M^H lam = G is the transposed march of conj(G) in
// reversed time, conjugated.
struct StepIO {
  const aim_excitation* exc = nullptr;                  // plane waves (Eq. 1)
  int nb = 0;
  const aim_c128* src = nullptr;                        // explicit sources [n_steps][nb][ns]
  aim_c128* out = nullptr;                              // currents [n_steps][nb][ns] (may be null)
  bool rev = false;
  std::function<void(int j, double2* b)> make_src;      // custom source written to b (device)
  std::function<void(int j, const double2* x)> commit;  // after I_j is committed (device)
};

static int march_steps(aim_ctx* c, const StepIO& io, int n_steps, double tol, aim_stats* stats);

void adj_excitation_samples(aim_ctx* c, const double* khat, const double* phat, int i0, int n_samp,
                            const double2* a, int l0, int n_steps, double2* V);
void adj_excitation_samples_adjoint(aim_ctx* c, const double* khat, const double* phat, int i0, int n_samp,
                                    int l0, int n_steps, const double2* lam, bool conj_lam, bool accumulate,
                                    double2* grad);
void adj_farfield(aim_ctx* c, int nd, const double* d_dirs, int l0, int n_steps, const double2* I, int n0, int n_out,
                  bool accumulate, double2* F);
void adj_farfield_adjoint(aim_ctx* c, int nd, const double* d_dirs, int l0, int n_steps, int n0, int n_out,
                          const double2* F, bool conj_out, double2* G);
void adj_ensure_near_transpose(aim_ctx* c);

namespace {
__global__ void __launch_bounds__(256) k_conj(long long n, const double2* __restrict__ a, double2* __restrict__ b) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) {
    const double2 v = a[i];
    b[i] = make_double2(v.x, -v.y);
  }
}
void conj_copy(aim_ctx* c, size_t n, const double2* a, double2* b) {
  k_conj<<<(int)((n + 255) / 256), 256, 0, c->stream>>>((long long)n, a, b);
  AIM_CHECK_LAUNCH();
}

// the near-zone values of the transposed matrices Z_m^T for the life of one call
struct TransposeNear {
  aim_ctx* c;
  double2* fwd;
  explicit TransposeNear(aim_ctx* c_) : c(c_), fwd(c_->d_near) {
    adj_ensure_near_transpose(c);
    if (c->nnz) c->d_near = c->d_nearT;
  }
  ~TransposeNear() { c->d_near = fwd; }
};
}  // namespace

extern "C" {

int aim_setup(const aim_mesh* mesh, const aim_grid* grid, double near_radius, double dt, aim_tbasis tbasis,
              const aim_opts* opts, aim_ctx** out) {
  if (!out) return AIM_ERR_ARG;
  *out = nullptr;
  aim_ctx* c = new (std::nothrow) aim_ctx;
  if (!c) return AIM_ERR_OOM;
  int rc = guard(c, [&] {
    setup_impl(c, mesh, grid, near_radius, dt, tbasis, opts);
    return AIM_OK;
  });
  if (rc != AIM_OK) {
    g_last_setup_error = c->err;
    aim_destroy(c);
    return rc;
  }
  *out = c;
  return AIM_OK;
}

void aim_destroy(aim_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (void* p : c->allocs) cudaFree(p);
  for (auto& r : c->prof.pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->prof.pool) cudaEventDestroy(e);
  gmres_free_host(c);
  if (c->h_rn) cudaFreeHost(c->h_rn);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* aim_last_error(const aim_ctx* c) { return c ? c->err.c_str() : g_last_setup_error.c_str(); }

int aim_get_info(const aim_ctx* c, aim_info* info) {
  if (!c || !info) return AIM_ERR_ARG;
  info->ns = c->ns;
  info->n_delays = c->n_delays;
  info->n_active = c->n_active;
  info->near_nnz = c->nnz;
  info->grid_n = c->N;
  info->precision = c->precision;
  info->device_bytes = (int64_t)c->device_bytes;
  info->preconditioner = c->precond;
  info->precond_nnz = c->d_sai ? c->snnz : c->ns;
  info->refine = c->refine;
  info->refine_every = c->refine_every;
  info->plan_zw = c->plan.zw;
  info->plan_cw = c->plan.cw;
  info->plan_rp = c->plan.rp;
  info->plan_ypb = c->plan.ypb;
  info->plan_source = c->plan.source;
  for (int d = 0; d < 3; ++d) {
    info->box_lo[d] = c->box_lo[d];
    info->box_hi[d] = c->box_hi[d];
  }
  info->z_len = c->LZ;
  info->rhs_blocked = c->rhs_blocked ? 1 : 0;
  return AIM_OK;
}

int aim_time_factor(aim_tbasis tb, double blif_band, int32_t m, int32_t n, const double* x, double* out) {
  if (m < 0 || n < 0 || (n > 0 && (!x || !out))) return AIM_ERR_ARG;
  try {
    TBasis b;
    if (tb.kind == AIM_BLIF)
      host_blif(tb.order, blif_band, b);
    else if (tb.kind == AIM_CPPIF)
      host_cppif(tb.order, b);
    else
      throw AimError{AIM_ERR_ARG, "temporal basis: AIM_CPPIF or AIM_BLIF"};
    for (int32_t i = 0; i < n; ++i) tb_eval(b, m, x[i], out + 4 * (size_t)i);
  } catch (const AimError& e) {
    g_last_setup_error = e.msg;
    return e.code;
  }
  return AIM_OK;
}

int aim_num_unknowns(const aim_ctx* c, int32_t* ns, int32_t* n_delays) {
  if (!c) return AIM_ERR_ARG;
  if (ns) *ns = c->ns;
  if (n_delays) *n_delays = c->n_delays;
  return AIM_OK;
}

int aim_rwg_table(const aim_ctx* c, int32_t* edge, int32_t* tri, int32_t* free_vertex) {
  if (!c) return AIM_ERR_ARG;
  const size_t n = 2 * (size_t)c->ns;
  if (edge) std::memcpy(edge, c->h_edge.data(), n * sizeof(int32_t));
  if (tri) std::memcpy(tri, c->h_tri.data(), n * sizeof(int32_t));
  if (free_vertex) std::memcpy(free_vertex, c->h_free.data(), n * sizeof(int32_t));
  return AIM_OK;
}

int aim_matvec(aim_ctx* c, int32_t m, int32_t nb, const aim_c128* x, aim_c128* y) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (!x || !y || nb < 1 || nb > c->batch_max || m < 0 || m > c->n_delays)
      throw AimError{AIM_ERR_ARG, "aim_matvec: bad delay, batch or pointer"};
    const size_t n = (size_t)nb * c->ns;
    const double2* xs = stage_in(c, x, n, c->d_x);
    const bool ydev = is_device_ptr(y);
    double2* ys = ydev ? reinterpret_cast<double2*>(y) : c->d_y;
    op_apply(c, m, nb, xs, nullptr, nullptr, 1.0, nullptr, ys);
    if (!ydev) AIM_CUDA(cudaMemcpyAsync(y, ys, n * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    AIM_CUDA(cudaStreamSynchronize(c->stream));
    return AIM_OK;
  });
}

int aim_rhs(aim_ctx* c, int32_t l, int32_t nb, const aim_c128* hist, aim_c128* rhs) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (!hist || !rhs || nb < 1 || nb > c->batch_max || l < 1)
      throw AimError{AIM_ERR_ARG, "aim_rhs: bad step, batch or pointer"};
    const int ng = c->n_delays;
    const size_t n = (size_t)nb * c->ns;
    const double2* hs = stage_in(c, hist, (size_t)ng * n, c->d_hist);
    ensure_ring(c);
    const size_t slab = op_slab_bytes(c, c->batch_max);
    SlabList sl{};
    NearList nl{};
    for (int m = 1; m <= ng; ++m) {
      if (l - m < 1) continue;
      const double2* I = hs + (size_t)(m - 1) * n;
      void* dst = (char*)c->d_ring + (size_t)(m - 1) * slab;
      op_forward_slab(c, nb, I, dst);
      sl.p[sl.n] = dst;
      sl.m[sl.n] = m;
      sl.n++;
      if (c->nnz > 0) {
        nl.val[nl.n] = c->d_near + (size_t)m * c->nnz;
        nl.x[nl.n] = I;
        nl.n++;
      }
    }
    const bool ydev = is_device_ptr(rhs);
    double2* ys = ydev ? reinterpret_cast<double2*>(rhs) : c->d_y;
    op_apply_rhs(c, nb, sl, nl, nullptr, 1.0, ys);
    if (!ydev) AIM_CUDA(cudaMemcpyAsync(rhs, ys, n * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    int h_err = 0;
    AIM_CUDA(cudaMemcpyAsync(&h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    AIM_CUDA(cudaStreamSynchronize(c->stream));
    if (h_err) {
      AIM_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
      throw AimError{AIM_ERR_TIMEOUT, "aim_rhs: a bounded wait of the delayed-sum kernel gave up"};
    }
    return AIM_OK;
  });
}

int aim_excitation_vector(aim_ctx* c, const aim_excitation* exc, int32_t l, aim_c128* out) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (!out) throw AimError{AIM_ERR_ARG, "aim_excitation_vector: null output"};
    upload_waves(c, exc);
    const size_t n = (size_t)exc->nb * c->ns;
    const bool dev = is_device_ptr(out);
    double2* o = dev ? reinterpret_cast<double2*>(out) : c->d_y;
    op_excitation(c, exc->nb, c->d_exc, exc->sigma, exc->t_d, l, o);
    if (!dev) AIM_CUDA(cudaMemcpyAsync(out, o, n * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    AIM_CUDA(cudaStreamSynchronize(c->stream));
    return AIM_OK;
  });
}

int aim_march(aim_ctx* c, const aim_excitation* exc, int32_t n_steps, double tol, aim_c128* currents,
              aim_stats* stats) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (!currents || n_steps < 1 || !(tol > 0)) throw AimError{AIM_ERR_ARG, "aim_march: bad arguments"};
    upload_waves(c, exc);
    AIM_CUDA(cudaMemsetAsync(c->d_x, 0, (size_t)exc->nb * c->ns * sizeof(double2), c->stream));
    c->l_done = 0;
    c->march_nb = exc->nb;
    StepIO io;
    io.exc = exc;
    io.nb = exc->nb;
    io.out = currents;
    return march_steps(c, io, n_steps, tol, stats);
  });
}

int aim_march_continue(aim_ctx* c, const aim_excitation* exc, int32_t n_steps, double tol, aim_c128* currents,
                       aim_stats* stats) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (!currents || n_steps < 1 || !(tol > 0)) throw AimError{AIM_ERR_ARG, "aim_march_continue: bad arguments"};
    if (c->march_nb < 1 || !exc || exc->nb != c->march_nb)
      throw AimError{AIM_ERR_ARG, "aim_march_continue: no march with this batch was started on the context"};
    upload_waves(c, exc);
    StepIO io;
    io.exc = exc;
    io.nb = exc->nb;
    io.out = currents;
    return march_steps(c, io, n_steps, tol, stats);
  });
}

int aim_profile(aim_ctx* c, int32_t enable) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    AIM_CUDA(cudaStreamSynchronize(c->stream));
    prof_flush(c);
    for (int i = 0; i < AIM_K_COUNT; ++i) {
      c->prof.ms[i] = 0;
      c->prof.n[i] = 0;
    }
    c->prof.launches = 0;
    c->prof.on = enable != 0;
    return AIM_OK;
  });
}

int aim_get_profile(aim_ctx* c, int64_t* launches, double* ms, int64_t* total) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    AIM_CUDA(cudaStreamSynchronize(c->stream));
    prof_flush(c);
    for (int i = 0; i < AIM_K_COUNT; ++i) {
      if (launches) launches[i] = c->prof.n[i];
      if (ms) ms[i] = c->prof.ms[i];
    }
    if (total) *total = c->prof.launches;
    return AIM_OK;
  });
}

const char* aim_kernel_name(int32_t id) {
  static const char* names[AIM_K_COUNT] = {"anterp_xfft", "yfft_fwd", "zconv", "zrhs", "yfft_inv", "xfft_inv",
                                          "interp_near", "excitation", "gmres_dot", "gmres_update", "gmres_small", "prep",
                                          "zfwd", "block_square", "zinv_pending"};
  return id >= 0 && id < AIM_K_COUNT ? names[id] : "?";
}

int aim_march_source(aim_ctx* c, int32_t transpose, int32_t nb, int32_t n_steps, const aim_c128* src, double tol,
                     aim_c128* currents, aim_stats* stats) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (!src || !currents || n_steps < 1 || nb < 1 || nb > c->batch_max || !(tol > 0))
      throw AimError{AIM_ERR_ARG, "aim_march_source: bad arguments"};
    std::unique_ptr<TransposeNear> tn(transpose ? new TransposeNear(c) : nullptr);
    AIM_CUDA(cudaMemsetAsync(c->d_x, 0, (size_t)nb * c->ns * sizeof(double2), c->stream));
    c->l_done = 0;
    c->march_nb = 0;  // a source march cannot be continued with aim_march_continue
    StepIO io;
    io.nb = nb;
    io.src = src;
    io.out = currents;
    return march_steps(c, io, n_steps, tol, stats);
  });
}

namespace {
// host or device array of n doubles -> device pointer (staged through a scratch buffer)
const double2* dev_in(aim_ctx* c, const aim_c128* p, size_t n, double2* staging) {
  if (is_device_ptr(p)) return reinterpret_cast<const double2*>(p);
  AIM_CUDA(cudaMemcpyAsync(staging, p, n * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
  return staging;
}
double2* scratch(aim_ctx* c, size_t n, int slot) {
  if (c->adj_cap[slot] < n) {
    c->adj_buf[slot] = (double2*)aim_alloc(c, n * sizeof(double2));
    c->adj_cap[slot] = n;
  }
  return c->adj_buf[slot];
}
void finish_out(aim_ctx* c, aim_c128* out, const double2* d, size_t n, bool dev) {
  if (!dev) AIM_CUDA(cudaMemcpyAsync(out, d, n * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
  AIM_CUDA(cudaStreamSynchronize(c->stream));
}
const double* upload_dirs(aim_ctx* c, int nd, const double* rhat, const double* e1, const double* e2) {
  std::vector<double> h((size_t)9 * nd);
  for (int i = 0; i < 3 * nd; ++i) {
    h[i] = rhat[i];
    h[3 * nd + i] = e1[i];
    h[6 * nd + i] = e2[i];
  }
  double* d = reinterpret_cast<double*>(scratch(c, (size_t)(9 * nd + 1) / 2 + 1, 4));
  AIM_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  return d;
}
}  // namespace

int aim_excitation_samples(aim_ctx* c, const double* khat, const double* phat, int32_t i0, int32_t n_samp,
                           const aim_c128* a, int32_t n_steps, aim_c128* V) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (!khat || !phat || !a || !V || n_samp < 1 || n_steps < 1)
      throw AimError{AIM_ERR_ARG, "aim_excitation_samples: bad arguments"};
    const size_t n = (size_t)n_steps * c->ns;
    const double2* da = dev_in(c, a, n_samp, scratch(c, n_samp, 0));
    const bool dev = is_device_ptr(V);
    double2* out = dev ? reinterpret_cast<double2*>(V) : scratch(c, n, 1);
    adj_excitation_samples(c, khat, phat, i0, n_samp, da, 1, n_steps, out);
    finish_out(c, V, out, n, dev);
    return AIM_OK;
  });
}

int aim_excitation_samples_adjoint(aim_ctx* c, const double* khat, const double* phat, int32_t i0, int32_t n_samp,
                                   int32_t n_steps, const aim_c128* lam, aim_c128* grad) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (!khat || !phat || !lam || !grad || n_samp < 1 || n_steps < 1)
      throw AimError{AIM_ERR_ARG, "aim_excitation_samples_adjoint: bad arguments"};
    const size_t n = (size_t)n_steps * c->ns;
    const double2* dl = dev_in(c, lam, n, scratch(c, n, 1));
    const bool dev = is_device_ptr(grad);
    double2* out = dev ? reinterpret_cast<double2*>(grad) : scratch(c, n_samp, 0);
    adj_excitation_samples_adjoint(c, khat, phat, i0, n_samp, 1, n_steps, dl, false, false, out);
    finish_out(c, grad, out, n_samp, dev);
    return AIM_OK;
  });
}

int aim_farfield(aim_ctx* c, int32_t nd, const double* rhat, const double* e1, const double* e2, int32_t n_steps,
                 const aim_c128* I, int32_t n0, int32_t n_out, aim_c128* F) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (nd < 1 || !rhat || !e1 || !e2 || !I || !F || n_steps < 1 || n_out < 1)
      throw AimError{AIM_ERR_ARG, "aim_farfield: bad arguments"};
    const size_t n = (size_t)n_steps * c->ns, nf = (size_t)n_out * nd * 2;
    const double* dd = upload_dirs(c, nd, rhat, e1, e2);
    const double2* dI = dev_in(c, I, n, scratch(c, n, 1));
    const bool dev = is_device_ptr(F);
    double2* out = dev ? reinterpret_cast<double2*>(F) : scratch(c, nf, 2);
    adj_farfield(c, nd, dd, 1, n_steps, dI, n0, n_out, false, out);
    finish_out(c, F, out, nf, dev);
    return AIM_OK;
  });
}

int aim_farfield_adjoint(aim_ctx* c, int32_t nd, const double* rhat, const double* e1, const double* e2,
                         int32_t n_steps, int32_t n0, int32_t n_out, const aim_c128* F, aim_c128* G) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (nd < 1 || !rhat || !e1 || !e2 || !F || !G || n_steps < 1 || n_out < 1)
      throw AimError{AIM_ERR_ARG, "aim_farfield_adjoint: bad arguments"};
    const size_t n = (size_t)n_steps * c->ns, nf = (size_t)n_out * nd * 2;
    const double* dd = upload_dirs(c, nd, rhat, e1, e2);
    const double2* dF = dev_in(c, F, nf, scratch(c, nf, 2));
    const bool dev = is_device_ptr(G);
    double2* out = dev ? reinterpret_cast<double2*>(G) : scratch(c, n, 3);
    adj_farfield_adjoint(c, nd, dd, 1, n_steps, n0, n_out, dF, false, out);
    finish_out(c, G, out, n, dev);
    return AIM_OK;
  });
}

int aim_march_adjoint(aim_ctx* c, int32_t nb, int32_t n_steps, const aim_c128* G, double tol, aim_c128* lam,
                      aim_stats* stats) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (!G || !lam || n_steps < 1 || nb < 1 || nb > c->batch_max || !(tol > 0))
      throw AimError{AIM_ERR_ARG, "aim_march_adjoint: bad arguments"};
    TransposeNear tn(c);
    AIM_CUDA(cudaMemsetAsync(c->d_x, 0, (size_t)nb * c->ns * sizeof(double2), c->stream));
    c->l_done = 0;
    c->march_nb = 0;
    StepIO io;
    io.nb = nb;
    io.src = G;
    io.out = lam;
    io.rev = true;
    return march_steps(c, io, n_steps, tol, stats);
  });
}

int aim_march_farfield(aim_ctx* c, const double* khat, const double* phat, int32_t i0, int32_t n_samp,
                       const aim_c128* a, int32_t n_steps, double tol, int32_t nd, const double* rhat,
                       const double* e1, const double* e2, int32_t n0, int32_t n_out, aim_c128* F,
                       aim_stats* stats) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (!khat || !phat || !a || n_samp < 1 || n_steps < 1 || !(tol > 0) || nd < 1 || !rhat || !e1 || !e2 ||
        n_out < 1 || !F)
      throw AimError{AIM_ERR_ARG, "aim_march_farfield: bad arguments"};
    const size_t nf = (size_t)n_out * nd * 2;
    const double* dd = upload_dirs(c, nd, rhat, e1, e2);
    const double2* da = dev_in(c, a, n_samp, scratch(c, n_samp, 0));
    const bool dev = is_device_ptr(F);
    double2* Fd = dev ? reinterpret_cast<double2*>(F) : scratch(c, nf, 2);
    AIM_CUDA(cudaMemsetAsync(Fd, 0, nf * sizeof(double2), c->stream));
    AIM_CUDA(cudaMemsetAsync(c->d_x, 0, (size_t)c->ns * sizeof(double2), c->stream));
    c->l_done = 0;
    c->march_nb = 0;
    StepIO io;
    io.nb = 1;
    io.make_src = [&](int j, double2* b) { adj_excitation_samples(c, khat, phat, i0, n_samp, da, j, 1, b); };
    io.commit = [&](int j, const double2* x) { adj_farfield(c, nd, dd, j, 1, x, n0, n_out, true, Fd); };
    const int rc = march_steps(c, io, n_steps, tol, stats);
    finish_out(c, F, Fd, nf, dev);
    return rc;
  });
}

int aim_march_spectrum(aim_ctx* c, const aim_excitation* exc, int32_t n_steps, double tol, int32_t n_freq,
                       const double* freqs, aim_c128* spec, aim_stats* stats) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (!spec || !freqs || n_steps < 1 || !(tol > 0) || n_freq < 1 || n_freq > kMaxRcsFreq)
      throw AimError{AIM_ERR_ARG, "aim_march_spectrum: bad arguments (1 <= n_freq <= 64)"};
    for (int f = 0; f < n_freq; ++f)
      if (!(freqs[f] > 0)) throw AimError{AIM_ERR_ARG, "aim_march_spectrum: frequencies must be > 0"};
    upload_waves(c, exc);
    const int nb = exc->nb;
    const size_t n = (size_t)n_freq * nb * c->ns;
    std::vector<double> omega(n_freq);
    for (int f = 0; f < n_freq; ++f) omega[f] = 2.0 * aimc::kPi * (freqs[f] - c->f_c);
    const bool dev = is_device_ptr(spec);
    double2* acc = dev ? reinterpret_cast<double2*>(spec) : scratch(c, n, 3);
    AIM_CUDA(cudaMemsetAsync(acc, 0, n * sizeof(double2), c->stream));
    AIM_CUDA(cudaMemsetAsync(c->d_x, 0, (size_t)nb * c->ns * sizeof(double2), c->stream));
    c->l_done = 0;
    c->march_nb = 0;  // no current history to continue from
    StepIO io;
    io.exc = exc;
    io.nb = nb;
    io.commit = [&](int j, const double2* x) { rcs_dft_accum(c, nb, j, n_freq, omega.data(), x, acc); };
    const int rc = march_steps(c, io, n_steps, tol, stats);
    // dt That(Omega dt) / E~(Omega): the interpolated envelope over the unit incident pulse
    RcsPhases sc{};
    sc.n = n_freq;
    for (int f = 0; f < n_freq; ++f) {
      const double W = omega[f];
      const std::complex<double> E = exc->sigma * std::sqrt(2.0 * aimc::kPi) *
                                     std::exp(-0.5 * exc->sigma * exc->sigma * W * W) *
                                     std::exp(std::complex<double>(0.0, -(c->wc + W) * exc->t_d));
      const std::complex<double> v = c->dt * basis_spectrum(c->tb, W * c->dt) / E;
      sc.w[f] = make_double2(v.real(), v.imag());
    }
    rcs_scale(c, nb, sc, acc);
    finish_out(c, spec, acc, n, dev);
    return rc;
  });
}

int aim_rcs(aim_ctx* c, int32_t n_freq, const double* freqs, int32_t nb, const aim_c128* spec, int32_t nd,
            const double* rhat, const double* pol, double* sigma) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (!freqs || !spec || !rhat || !pol || !sigma || n_freq < 1 || nb < 1 || nd < 1 || nd > 65535 || nb > 65535 ||
        n_freq > 65535)
      throw AimError{AIM_ERR_ARG, "aim_rcs: bad arguments"};
    const size_t n = (size_t)n_freq * nb * c->ns, no = (size_t)n_freq * nb * nd;
    std::vector<double> h((size_t)6 * nd + 2 * n_freq);
    for (int d = 0; d < nd; ++d)
      for (int x = 0; x < 3; ++x) {
        h[6 * d + x] = rhat[3 * d + x];
        h[6 * d + 3 + x] = pol[3 * d + x];
      }
    for (int f = 0; f < n_freq; ++f) {
      if (!(freqs[f] > 0)) throw AimError{AIM_ERR_ARG, "aim_rcs: frequencies must be > 0"};
      const double w = 2.0 * aimc::kPi * freqs[f];
      const double a = w * c->mu_med / (4.0 * aimc::kPi);
      h[6 * nd + 2 * f] = w / c->c_med;
      h[6 * nd + 2 * f + 1] = 4.0 * aimc::kPi * a * a;
    }
    double* dd = reinterpret_cast<double*>(scratch(c, h.size() / 2 + 1, 4));
    AIM_CUDA(cudaMemcpyAsync(dd, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    const double2* ds = dev_in(c, spec, n, scratch(c, n, 1));
    const bool dev = is_device_ptr(sigma);
    double* out = dev ? sigma : reinterpret_cast<double*>(scratch(c, no / 2 + 1, 2));
    rcs_farfield(c, n_freq, nb, ds, nd, dd, dd + 6 * nd, out);
    if (!dev) AIM_CUDA(cudaMemcpyAsync(sigma, out, no * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    AIM_CUDA(cudaStreamSynchronize(c->stream));
    return AIM_OK;
  });
}

int aim_march_adjoint_farfield(aim_ctx* c, const double* khat, const double* phat, int32_t i0, int32_t n_samp,
                               int32_t n_steps, double tol, int32_t nd, const double* rhat, const double* e1,
                               const double* e2, int32_t n0, int32_t n_out, const aim_c128* F, aim_c128* grad,
                               aim_stats* stats) {
  if (!c) return AIM_ERR_ARG;
  return guard(c, [&] {
    if (!khat || !phat || !grad || n_samp < 1 || n_steps < 1 || !(tol > 0) || nd < 1 || !rhat || !e1 || !e2 ||
        n_out < 1 || !F)
      throw AimError{AIM_ERR_ARG, "aim_march_adjoint_farfield: bad arguments"};
    const size_t nf = (size_t)n_out * nd * 2;
    const double* dd = upload_dirs(c, nd, rhat, e1, e2);
    const double2* dF = dev_in(c, F, nf, scratch(c, nf, 2));
    const bool dev = is_device_ptr(grad);
    double2* gd = dev ? reinterpret_cast<double2*>(grad) : scratch(c, n_samp, 0);
    AIM_CUDA(cudaMemsetAsync(gd, 0, (size_t)n_samp * sizeof(double2), c->stream));
    TransposeNear tn(c);
    AIM_CUDA(cudaMemsetAsync(c->d_x, 0, (size_t)c->ns * sizeof(double2), c->stream));
    c->l_done = 0;
    c->march_nb = 0;
    StepIO io;
    io.nb = 1;
    // step j of the transposed march is time step l = n_steps + 1 - j: source conj(G_l),
    // and its solution u gives lam_l = conj(u)
    io.make_src = [&](int j, double2* b) {
      adj_farfield_adjoint(c, nd, dd, n_steps + 1 - j, 1, n0, n_out, dF, true, b);
    };
    io.commit = [&](int j, const double2* u) {
      adj_excitation_samples_adjoint(c, khat, phat, i0, n_samp, n_steps + 1 - j, 1, u, true, true, gd);
    };
    const int rc = march_steps(c, io, n_steps, tol, stats);
    finish_out(c, grad, gd, n_samp, dev);
    return rc;
  });
}

int aim_get_anterp(const aim_ctx* c, int32_t* anchor, double* lam) {
  if (!c) return AIM_ERR_ARG;
  return guard(const_cast<aim_ctx*>(c), [&] {
    if (anchor)
      AIM_CUDA(cudaMemcpy(anchor, c->d_anchor, (size_t)c->ns * 3 * sizeof(int), cudaMemcpyDeviceToHost));
    if (lam) AIM_CUDA(cudaMemcpy(lam, c->d_lam, (size_t)c->ns * 256 * sizeof(double), cudaMemcpyDeviceToHost));
    return AIM_OK;
  });
}

int aim_get_near(const aim_ctx* c, int32_t* rowptr, int32_t* col, aim_c128* val) {
  if (!c) return AIM_ERR_ARG;
  return guard(const_cast<aim_ctx*>(c), [&] {
    if (rowptr) std::memcpy(rowptr, c->h_rowptr.data(), (c->ns + 1) * sizeof(int));
    if (col && c->nnz) AIM_CUDA(cudaMemcpy(col, c->d_col, c->nnz * sizeof(int), cudaMemcpyDeviceToHost));
    if (val && c->nnz)
      AIM_CUDA(cudaMemcpy(val, c->d_near, (size_t)(c->n_delays + 1) * c->nnz * sizeof(double2),
                          cudaMemcpyDeviceToHost));
    return AIM_OK;
  });
}

int aim_get_preconditioner(const aim_ctx* c, int32_t* rowptr, int32_t* col, aim_c128* val) {
  if (!c) return AIM_ERR_ARG;
  return guard(const_cast<aim_ctx*>(c), [&] {
    if (c->d_sai) {
      if (rowptr) std::memcpy(rowptr, c->h_srowptr.data(), (c->ns + 1) * sizeof(int));
      if (col) AIM_CUDA(cudaMemcpy(col, c->d_scol, c->snnz * sizeof(int), cudaMemcpyDeviceToHost));
      if (val) AIM_CUDA(cudaMemcpy(val, c->d_sai, c->snnz * sizeof(double2), cudaMemcpyDeviceToHost));
    } else {
      for (int k = 0; k <= c->ns; ++k)
        if (rowptr) rowptr[k] = k;
      for (int k = 0; k < c->ns; ++k)
        if (col) col[k] = k;
      if (val) AIM_CUDA(cudaMemcpy(val, c->d_dinv, c->ns * sizeof(double2), cudaMemcpyDeviceToHost));
    }
    return AIM_OK;
  });
}

int aim_get_kernel_spectrum(const aim_ctx* c, int32_t m, int32_t kind, aim_c128* out) {
  if (!c) return AIM_ERR_ARG;
  return guard(const_cast<aim_ctx*>(c), [&] {
    if (!out || m < 0 || m > c->n_delays || kind < 0 || kind > 1)
      throw AimError{AIM_ERR_ARG, "aim_get_kernel_spectrum: bad delay or kind"};
    const size_t oct = (size_t)(c->N + 1) * (c->N + 1) * (c->LZ / 2 + 1);
    AIM_CUDA(cudaMemcpy(out, c->d_kspec + ((size_t)m * 2 + kind) * oct, oct * sizeof(double2),
                        cudaMemcpyDeviceToHost));
    return AIM_OK;
  });
}

}  // extern "C"

// FP64 refinement of the immediate solve just enqueued (complex64 path): the GMRES with
// the complex64 operator has run to tol on the stream (synchronised by the caller).
// Then, with every grid stage of the residual in FP64,
//   r = b - Z_0 x;  while |r| > tol |b| (any RHS) and corrections remain:
//     solve Z_0 d = r with the complex64 operator from zero to kCorrTol;  x += d;  r = b - Z_0 x.
// The complex64 operator's error (relative ~1e-7) limits each correction, not the
// result: the error of the corrected x is that of the FP64 operator plus tol.
// Returns AIM_OK or AIM_ERR_NOCONV; its = GMRES iterations of all solves of the step,
// res = final FP64 relative residuals, n_corr = correction solves.
static int refine_solution(aim_ctx* c, int nb, double tol, std::vector<int>& its, std::vector<double>& res,
                           int& n_corr) {
  constexpr double kCorrTol = 1e-2;
  cudaStream_t st = c->stream;
  const size_t n = (size_t)nb * c->ns;
  std::vector<int> it(nb);
  std::vector<double> rr(nb);
  int rc = gmres_collect(c, it.data(), rr.data());
  for (int b = 0; b < nb; ++b) its[b] += it[b];
  res.assign(nb, 0.0);
  n_corr = 0;
  for (int k = 0;; ++k) {
    op_apply_f64(c, 0, nb, c->d_x, c->d_b, -1.0, c->d_r);  // r = b - Z_0 x, FP64 grid stages
    gmres_norms(c, nb, c->d_r, c->d_rn);
    gmres_norms(c, nb, c->d_b, c->d_rn + nb);
    AIM_CUDA(cudaMemcpyAsync(c->h_rn, c->d_rn, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    AIM_CUDA(cudaStreamSynchronize(st));
    bool ok = true;
    for (int b = 0; b < nb; ++b) {
      res[b] = c->h_rn[nb + b] > 0 ? c->h_rn[b] / c->h_rn[nb + b] : 0.0;
      ok = ok && res[b] <= tol;
    }
    if (ok) return AIM_OK;
    if (rc != AIM_OK || k == c->refine) return AIM_ERR_NOCONV;
    AIM_CUDA(cudaMemsetAsync(c->d_w, 0, n * sizeof(double2), st));
    gmres_solve_async(c, nb, c->d_r, c->d_w, kCorrTol, true);
    gmres_axpy(c, nb, c->d_w, c->d_x);
    AIM_CUDA(cudaStreamSynchronize(st));
    rc = gmres_collect(c, it.data(), rr.data());
    for (int b = 0; b < nb; ++b) its[b] += it[b];
    ++n_corr;
  }
}

static int march_steps(aim_ctx* c, const StepIO& io, int n_steps, double tol, aim_stats* stats) {
  cudaStream_t st = c->stream;
  const int nb = io.nb, ns = c->ns, ng = c->n_delays, B = c->batch_max;
  const aim_c128* src = io.src;
  aim_c128* currents = io.out;
  const bool src_dev = src && is_device_ptr(src);
  const size_t n = (size_t)nb * ns;
  const size_t slab = op_slab_bytes(c, B);
  const bool dev_out = currents && is_device_ptr(currents);
  ensure_ring(c);
  cudaEvent_t ev[3];
  for (auto& e : ev) AIM_CUDA(cudaEventCreate(&e));
  std::vector<int> its(nb);
  std::vector<double> res(nb), norms;
  double* d_nrm = c->gs.nrm;
  std::vector<double> h_nrm(nb);
  if (stats) {
    stats->last_step = 0;
    stats->total_iters = 0;
    stats->max_iters = 0;
    stats->max_rel_res = 0;
    stats->rhs_ms = 0;
    stats->solve_ms = 0;
    stats->refine_corrections = 0;
    stats->refine_checks = 0;
  }
  int rc = AIM_OK;
  const int l0 = c->l_done;
  const int nsrc = c->rhs_blocked ? 1 << c->blk_P : ng;  // source slots of the ring
  if (c->rhs_blocked && l0 == 0)  // a march from rest: nothing pending
    AIM_CUDA(cudaMemsetAsync(c->d_pend, 0, ((size_t)2 << c->blk_P) * slab, st));
  for (int l = l0 + 1; l <= l0 + n_steps; ++l) {
    AIM_CUDA(cudaEventRecord(ev[0], st));
    const int j = l - l0;                                       // step within this call
    const size_t jo = (size_t)(io.rev ? n_steps - j : j - 1);  // its slot in src / currents
    if (io.make_src) {
      io.make_src(j, c->d_b);
    } else if (src) {  // explicit right-hand side samples S_l
      AIM_CUDA(cudaMemcpyAsync(c->d_b, src + jo * n, n * sizeof(double2),
                               src_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
      if (io.rev) conj_copy(c, n, c->d_b, c->d_b);
    } else {
      op_excitation(c, nb, c->d_exc, io.exc->sigma, io.exc->t_d, l, c->d_b);
    }
    SlabList sl{};
    NearList nl{};
    for (int m = 1; m <= ng; ++m) {
      if (l - m < 1) continue;
      const int s = (l - m) % ng;
      if (!c->rhs_blocked) {
        sl.p[sl.n] = (char*)c->d_ring + (size_t)s * slab;
        sl.m[sl.n] = m;
        sl.n++;
      }
      if (c->nnz > 0) {
        nl.val[nl.n] = c->d_near + (size_t)m * c->nnz;
        nl.x[nl.n] = c->d_iring + (size_t)s * B * ns;
        nl.n++;
      }
    }
    if (c->rhs_blocked && l > 1)  // the grid part was gathered by the squares of earlier steps
      op_apply_rhs_pending(c, nb, (char*)c->d_pend + (size_t)(l % (2 * nsrc)) * slab, nl, c->d_b, -1.0, c->d_b);
    else
      op_apply_rhs(c, nb, sl, nl, c->d_b, -1.0, c->d_b);  // b = V_l - sum_m Z_m I_{l-m}
    AIM_CUDA(cudaEventRecord(ev[1], st));
    if (c->zero_start) AIM_CUDA(cudaMemsetAsync(c->d_x, 0, n * sizeof(double2), st));
    const bool refining = c->refine > 0 && l % c->refine_every == 0;
    // a checked step solves to half the tolerance, so that the FP64 residual (the
    // complex64 one plus the complex64 operator's error) usually passes without a
    // correction solve
    gmres_solve_async(c, nb, c->d_b, c->d_x, refining ? 0.5 * tol : tol);
    int r_ref = AIM_OK, n_corr = 0;
    std::vector<int> its_ref(nb, 0);
    std::vector<double> res_ref;
    if (refining) {
      AIM_CUDA(cudaStreamSynchronize(st));
      r_ref = refine_solution(c, nb, tol, its_ref, res_ref, n_corr);
    }
    AIM_CUDA(cudaEventRecord(ev[2], st));
    // commit I_l: RWG-space history and its forward slab
    const int s = l % ng;
    AIM_CUDA(cudaMemcpyAsync(c->d_iring + (size_t)s * B * ns, c->d_x, n * sizeof(double2),
                             cudaMemcpyDeviceToDevice, st));
    op_forward_slab(c, nb, c->d_x, (char*)c->d_ring + (size_t)(l % nsrc) * slab);
    if (c->rhs_blocked) {
      // the square of the last b = 2^min(ctz(l), P) steps radiated to the next b steps,
      // as sub-squares of at most 16 steps (source block u, observer block v: delays
      // from 1 + bs (v - u - 1) + 1 ... ; blocks whose delays all exceed N_g are skipped)
      int p = 0;
      while (p < c->blk_P && ((l >> p) & 1) == 0) ++p;
      const int b = 1 << p, bs = std::min(b, 16), nblk = b / bs;
      for (int u = 0; u < nblk; ++u)
        for (int v = 0; v < nblk; ++v) {
          BlockSquare sq{};
          sq.b = bs;
          sq.toff = b + (v - u) * bs;  // delay of (observer i, source j) = toff + i - j
          if (sq.toff - bs + 1 > ng || sq.toff + bs - 1 < 1) continue;
          for (int j = 0; j < bs; ++j) {
            sq.src[j] = (char*)c->d_ring + (size_t)((l - b + 1 + u * bs + j) % nsrc) * slab;
            sq.dst[j] = (char*)c->d_pend + (size_t)((l + 1 + v * bs + j) % (2 * nsrc)) * slab;
          }
          op_block_square(c, nb, sq);
        }
    }
    if (currents) {
      const double2* xo = c->d_x;
      if (io.rev) {
        conj_copy(c, n, c->d_x, c->d_y);
        xo = c->d_y;
      }
      AIM_CUDA(cudaMemcpyAsync(currents + jo * n, xo, n * sizeof(double2),
                               dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    if (io.commit) io.commit(j, c->d_x);
    gmres_norms(c, nb, c->d_x, d_nrm);
    AIM_CUDA(cudaMemcpyAsync(h_nrm.data(), d_nrm, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    int h_err = 0;
    AIM_CUDA(cudaMemcpyAsync(&h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    AIM_CUDA(cudaStreamSynchronize(st));
    if (h_err) {
      AIM_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
      throw AimError{AIM_ERR_TIMEOUT, "a bounded wait of the delayed-sum kernel gave up at step " + std::to_string(l)};
    }
    int r;
    if (refining) {  // statistics gathered by the refinement (solves and FP64 residuals)
      r = r_ref;
      its = its_ref;
      res = res_ref;
    } else {
      r = gmres_collect(c, its.data(), res.data());
    }
    double mx = 0;
    for (int b = 0; b < nb; ++b) mx = std::max(mx, h_nrm[b]);
    norms.push_back(mx);
    if (stats) {
      float a = 0, b2 = 0;
      cudaEventElapsedTime(&a, ev[0], ev[1]);
      cudaEventElapsedTime(&b2, ev[1], ev[2]);
      stats->rhs_ms += a;
      stats->solve_ms += b2;
      for (int b = 0; b < nb; ++b) {
        stats->total_iters += its[b];
        stats->max_iters = std::max(stats->max_iters, its[b]);
        stats->max_rel_res = std::max(stats->max_rel_res, res[b]);
        if (stats->iters) stats->iters[(size_t)(l - l0 - 1) * nb + b] = its[b];
      }
      stats->last_step = l;
      stats->refine_corrections += n_corr;
      stats->refine_checks += refining ? 1 : 0;
    }
    c->l_done = l;
    prof_flush(c);
    if (r != AIM_OK) {
      if (stats) stats->last_step = l - 1;
      c->err = (refining ? "GMRES reached its iteration cap or the FP64 refinement did not reach tol at step "
                               : "GMRES reached its iteration cap at step ") +
               std::to_string(l);
      rc = r;
      break;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (rc == AIM_OK && norms.size() >= 4) {
    double early = 0;
    for (size_t i = 0; i < norms.size() / 2; ++i) early = std::max(early, norms[i]);
    if (norms.back() > 1e3 * early) rc = AIM_WARN_UNSTABLE;
  }
  return rc;
}
