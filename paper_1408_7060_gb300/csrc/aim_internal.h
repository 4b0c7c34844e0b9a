// Internal state of an ET-AIM context and the helpers shared by the translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/aim.h"

// free-space constants (Sec. 2.1: homogeneous medium, here vacuum)
namespace aimc {
constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4.0e-7 * kPi;
constexpr double kEps0 = 1.0 / (kMu0 * kC0 * kC0);
constexpr int kMaxDelays = 32;   // N_g + 1 <= kMaxDelays
constexpr int kMaxOrder = 4;     // CPPIF order
constexpr int kMaxHalfWidth = 5; // BLIF half-width M
}  // namespace aimc

struct AimError {
  int code;
  std::string msg;
};

#define AIM_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      throw AimError{AIM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};  \
  } while (0)

#define AIM_CHECK_LAUNCH() AIM_CUDA(cudaGetLastError())

// programmatic dependent launch: wait for the previous kernel's results (a no-op when the
// kernel was launched without the attribute) / let the next kernel start launching
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with programmatic dependent launch allowed: the kernel may be scheduled while
// the previous kernel in the stream finishes; it must execute pdl_wait() before touching
// that kernel's results (every kernel launched this way does so first).
template <typename... P, typename... A>
inline void launch_pdl(cudaStream_t st, dim3 grid, dim3 block, size_t smem, void (*kern)(P...), A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  AIM_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...));
}

// one profiled kernel launch: AIM_KLAUNCH(ctx, AIM_K_..., kernel<<<...>>>(...))
#define AIM_KLAUNCH(ctx, kid, ...)   \
  do {                               \
    KScope ks_(ctx, kid);            \
    __VA_ARGS__;                     \
    AIM_CHECK_LAUNCH();              \
  } while (0)

// Temporal basis.  CPPIF (kind AIM_CPPIF): T on the piece (j-1, j] is sum_p coef[j][p] u^p
// (Horner on device), support (-1, Q].  BLIF (kind AIM_BLIF): T(u) = sinc(u) w(u) on |u| < M,
// w(u) = G(M^2 - u^2) / G(M^2), G(s) = sinh(b sqrt s) / sqrt s, b the guard band, and the
// sample l+p (p = 1..M-1) extrapolated as sum_q ext[p][q] I_{l-q}, q = 0..M-1.
struct TBasis {
  int kind;
  int Q;         // upper end of the support in steps: the CPPIF order Q or the BLIF half-width M
  double coef[aimc::kMaxOrder + 1][aimc::kMaxOrder + 1];
  double b, invG0;
  double ext[aimc::kMaxHalfWidth][aimc::kMaxHalfWidth];
};

// Sum over the lanes of a warp of a complex value, in 5 FP64 additions instead of 10:
// the first exchange pairs lane l with l ^ 16, the lower half keeping the real and the
// upper half the imaginary part, then both halves reduce their part in 4 more steps.
// (A double-precision instruction holds its sub-partition's FP64 pipe for the whole
// warp whatever the number of active lanes, so the instruction count is the cost.)
__device__ __forceinline__ double2 warp_sum_c(double2 v) {
  const int lane = threadIdx.x & 31;
  const bool hi = lane & 16;
  double keep = hi ? v.y : v.x;
  const double send = hi ? v.x : v.y;
  keep += __shfl_xor_sync(0xffffffffu, send, 16);
  for (int o = 8; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
  return make_double2(__shfl_sync(0xffffffffu, keep, 0), __shfl_sync(0xffffffffu, keep, 16));
}

// Raw Krylov dots formed by the interpolation kernel of an Arnoldi step's operator:
// d[b][i] = conj(vt_i) . y_b for i <= *jdev, y the kernel's output (Krylov slot j+1);
// partials per block of 32 rows, summed by the last block of each RHS.
struct DotFuse {
  const double2* V = nullptr;  // Krylov basis; null: no dots
  long long vstride = 0;
  const int* jdev = nullptr;
  double2* pd = nullptr;       // partials [B][64][P]
  double2* d = nullptr;        // sums [B][64]
  unsigned* ucnt = nullptr;    // [B] block arrivals per RHS
  int P = 0;                   // interpolation blocks per RHS
};

// GMRES small state, one row of 64 per right-hand side (restart <= 63)
struct GmresState {
  double2* H = nullptr;      // [B][64][64] Hessenberg columns, unrotated (upper triangle)
  double2* rd = nullptr;     // [B][64] diagonal of the rotated triangle R
  double2* rho = nullptr;    // [B][64] row j of the accumulated Givens rotation
  unsigned* fin = nullptr;   // [2] column-finish arrivals, any RHS still iterating
  double2* g = nullptr;      // [B][64]
  double2* sn = nullptr;     // [B][64]
  double* cs = nullptr;      // [B][64]
  double2* y = nullptr;      // [B][64]
  double2* h1 = nullptr;     // [B][64] first CGS pass
  double2* h2 = nullptr;     // [B][64] second CGS pass
  double* sig = nullptr;     // [B][64] scales of the stored Krylov vectors
  double* bn = nullptr;      // [B] ||b||
  double* relres = nullptr;  // [B]
  int* act = nullptr;        // [B] taking Arnoldi steps
  int* done = nullptr;       // [B] 1 converged, 2 iteration cap
  int* jc = nullptr;         // [B] columns in the current cycle
  int* its = nullptr;        // [B] iterations of this solve
  int* jdev = nullptr;       // current Arnoldi column (shared by the batch)
  int* flag = nullptr;       // [3] any active at cycle start / after a step / a stop without convergence
  int* cnt = nullptr;        // [2] cycles and Arnoldi steps executed (launch accounting)
  double2* pd = nullptr;     // raw dot partials of the new Krylov vector [B][64][cgs_P]
  double2* d1 = nullptr;     // their sums: the first CGS pass's dots [B][64]
  double2* pdi = nullptr;    // the same partials formed by the interpolation kernel [B][64][P_i]
  int interp_P = 0;          // interpolation blocks per RHS when it forms the dots (0: it does not)
  double* pu = nullptr;      // |w|^2 partials [B][cgs_P]
  double2* pd2 = nullptr;    // raw dot partials of the first CGS update [B][64][cgs_P]
  double2* d2 = nullptr;     // their sums: the second pass's dots [B][64]
  unsigned* ucnt = nullptr;  // [B] CGS update blocks arrived per RHS
  int cgs_E = 0, cgs_P = 0;  // elements per CGS update block, blocks per RHS
  double* pr = nullptr;      // |r|^2 partials [B][P]
  double* pbn = nullptr;     // |b|^2 partials [B][P]
  double* nrm = nullptr;     // [B] norms for the march's growth check
  int* h_flag = nullptr;     // pinned host mirrors
  int* h_its = nullptr;
  double* h_res = nullptr;
  int* h_done = nullptr;
  int* h_cnt = nullptr;
  // captured solves (one graph with conditional loops each), rebuilt when their inputs
  // change: slot 0 for solves warm-started from x, slot 1 for solves from zero (the
  // correction solves of the FP64 refinement, or every solve with zero_start)
  struct SolveGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int nb = 0;
    double tol = 0;
    const void* b = nullptr;
    const void* x = nullptr;
    const void* near = nullptr;
  } graphs[2];
  bool graph_failed = false;
  bool last_graphed = false;  // the last enqueued solve ran as a graph
  bool last_zs = false;       // ... and started from zero
  int last_nb = 0;
};

// Launch shapes of the grid passes (tile widths and rows per block).  Zero fields take
// the built-in defaults; aim_opts.autotune fills them by timing the candidates on the
// context's own buffers at setup (or from the plan cache).
struct KPlan {
  int zw = 0;      // z pass (fused convolution): columns per tile
  int cw = 0;      // y passes: columns per tile
  int rp = 0;      // inverse x pass: rows per block
  int ypb = 0;     // anterpolation + forward x pass: grid rows per block
  int source = 0;  // AIM_PLAN_DEFAULT, AIM_PLAN_MEASURED or AIM_PLAN_CACHED
};

// per-kernel event timing (aim_profile / aim_get_profile); ids match AIM_K_* in aim.h
struct ProfState {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  struct Rec { int id; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  double ms[AIM_K_COUNT] = {0};
  long long n[AIM_K_COUNT] = {0};
  long long launches = 0;
};

struct aim_ctx;
// elements of the grid work buffers for nb right-hand sides (layouts above d_A, d_Bf, d_P)
size_t grid_a_elems(const aim_ctx* c, int nb);
size_t grid_bf_elems(const aim_ctx* c, int nb);
size_t grid_p_elems(const aim_ctx* c, int nb);

struct aim_ctx {
  // problem
  int ns = 0, nt = 0, nv = 0;
  int N = 0, L = 0;            // grid nodes per axis, padded length 2N
  int box_lo[3] = {0, 0, 0};   // active box: the nodes (x, y, z) some stencil touches lie in
  int box_hi[3] = {0, 0, 0};   // [box_lo, box_hi] per axis (inclusive); the FFT passes prune to it
  int NZ = 0;                  // z-planes held by the grid buffers: the box's, box_lo[2] .. box_hi[2]
  int LZ = 0;                  // z transform length: the shortest supported length >= 2 NZ
  double h = 0, origin[3] = {0, 0, 0};
  double dt = 0, f_c = 0, wc = 0, kc = 0, near_radius = 0;
  double c_med = 0, mu_med = 0, eps_med = 0;  // light speed, permeability, permittivity of the medium
  TBasis tb{};
  int precision = AIM_C64;
  int batch_max = 1, restart = 50, max_iter = 500;
  int n_delays = 0, n_active = 0;
  long long nnz = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;

  // host copies of the RWG table (for aim_rwg_table)
  std::vector<int> h_edge, h_tri, h_free;
  std::vector<int> h_rowptr, h_col;

  // ---- device tables (FP64 unless noted) ----
  double* d_v = nullptr;       // [nv][3]
  int* d_tri = nullptr;        // [nt][3]
  int* d_rtri = nullptr;       // [ns][2]  T+, T-
  int* d_rfree = nullptr;      // [ns][2]
  double* d_len = nullptr;     // [ns]
  double* d_area = nullptr;    // [nt]
  int* d_tbk = nullptr;        // [nt][3] rwg of each edge slot of a face
  double* d_tbs = nullptr;     // [nt][3] sign
  int* d_tbf = nullptr;        // [nt][3] free vertex
  double* d_qp = nullptr;      // [nt][7][3] cubature points
  double* d_qw = nullptr;      // [nt][7] weights * area
  double* d_cent = nullptr;    // [nt][3]
  double mean_edge = 0;
  double rmax = 0;             // largest vertex distance from the origin (bounds the time reach
                               // r.u / (c dt) of every cubature point)

  int* d_anchor = nullptr;     // [ns][3]
  int* d_order = nullptr;      // [ns] RWGs in Morton order of their anchors (interpolation visit order)
  double* d_lam = nullptr;     // [ns][4][64]  FP64 anterpolation rows
  float* d_lamf = nullptr;     // [ns][4][64]  FP32 copy (C64 path)
  int* d_nptr = nullptr;       // [N^3 + 1]    node-major CSR of the transpose
  int* d_nidx = nullptr;       // [64 ns]
  double4_32a* d_ncoef = nullptr;  // [64 ns]  (x, y, z, div) coefficients
  float4* d_ncoeff = nullptr;  // [64 ns]  FP32 copy

  double2* d_kspec = nullptr;  // [(N_g+1)][2][LZ/2+1][N+1][N+1] kernel spectra octant (FP64)
  float2* d_kspecf = nullptr;  // FP32 copy
  double2* d_tw = nullptr;     // [L] twiddles W_L^t (FP64)
  float2* d_twf = nullptr;     // [L] FP32
  double2* d_twz = nullptr;    // [LZ] twiddles W_LZ^t of the z transform (FP64)
  float2* d_twzf = nullptr;    // [LZ] FP32

  int* d_rowptr = nullptr;     // [ns+1] near CSR
  int* d_col = nullptr;        // [nnz]
  double2* d_near = nullptr;   // [(N_g+1)][nnz]
  double2* d_dinv = nullptr;   // [ns] 1 / Z_0[k,k]
  int precond = 0;             // AIM_PRECOND_*
  double precond_radius = 0;   // SAI pattern radius (m)
  bool zero_start = false;     // GMRES initial guess 0 instead of the previous currents
  KPlan plan;                   // launch shapes of the grid passes
  int refine = 0;              // complex64 path: FP64-operator refinement sweeps per step (0: off)
  int refine_every = 1;        // FP64 residual checked at every k-th step
  bool rhs_blocked = false;    // multilevel blocked delayed sums (Sec. 4 stage ii)
  int blk_P = 0;               // top level: 2^P >= N_g source steps held
  void* d_pend = nullptr;      // [2^(P+1)] pending z-spectra of future steps (blocked sums)
  int ref_nb = 0;              // right-hand sides per FP64 residual product (its buffers' batch)
  void* d_A64 = nullptr;       // FP64 grid work buffers of the refinement residual ([ref_nb] x the
  void* d_Bf64 = nullptr;      // layouts of d_A, d_Bf, d_P), and its FP64 operator input
  void* d_P64 = nullptr;
  void* d_xs64 = nullptr;
  double* d_rn = nullptr;      // [2][B] |r| and |b| of the refinement check
  double* h_rn = nullptr;      // pinned host copy
  double2* d_sai = nullptr;    // [snnz] SAI values on its CSR pattern (AIM_PRECOND_NEAR_SAI)
  float2* d_saif = nullptr;    // the same rounded to complex64 (applied by the complex64 path)
  int* d_srowptr = nullptr;    // SAI pattern (the near-zone CSR when the radii agree)
  int* d_scol = nullptr;
  long long snnz = 0;
  std::vector<int> h_srowptr;
  double2* d_u = nullptr;      // [B][ns] Krylov combination before the preconditioner (SAI)
  double2* d_nearT = nullptr;  // [(N_g+1)][nnz] values of the transposed near matrices (lazy)

  // ---- work buffers (sized for batch_max) ----
  void* d_A = nullptr;         // [B][4][NZ][N][L]  after the x pass
  void* d_Bf = nullptr;        // [B][4][NZ][L][L]  after the y pass (the slab)
  void* d_P = nullptr;         // [B][4][NZ][N][N]  potentials on the grid
  void* d_ring = nullptr;      // [N_g][B][4][Z][L][L] history slabs: z-spectra (Z = LZ, power-of-two
                               // LZ) or x/y-transformed grids (Z = NZ)
  CUtensorMap ring_map;        // TMA view of the ring [slot][B*4*LZ][L][L] (complex64, power-of-two LZ)
  bool ring_tma = false;
  int* d_err = nullptr;        // device error flag (a bounded wait gave up)
  void* d_xs = nullptr;        // [B][ns] prepared operator input, grid precision
  double2* d_xd = nullptr;     // [B][ns] prepared operator input, FP64 (near zone)
  DotFuse dotfuse;             // set by the Arnoldi step around its operator application
  float2* d_vf = nullptr;      // [B][ns] complex64 copy of the Krylov vector the next SAI application
                               // reads (complex64 path; written by the kernel that finishes it)
  double2* d_iring = nullptr;  // [N_g][B][ns] current history (RWG space)
  double2* d_x = nullptr;      // [B][ns] staging / solution
  double2* d_y = nullptr;      // [B][ns]
  double2* d_b = nullptr;      // [B][ns]
  double2* d_r = nullptr;      // [B][ns]
  double2* d_w = nullptr;      // [B][ns]
  double2* d_V = nullptr;      // [restart+1][B][ns] Krylov basis
  double2* d_hist = nullptr;   // [N_g][B][ns] staging for aim_rhs
  double2* d_small = nullptr;  // GMRES small state (see gmres.cu)
  double* d_partial = nullptr; // reduction partials
  unsigned* d_counter = nullptr;
  int* d_status = nullptr;
  double* d_exc = nullptr;     // excitation parameters
  size_t device_bytes = 0;

  GmresState gs;
  double2* adj_buf[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // adjoint-helper staging
  size_t adj_cap[5] = {0, 0, 0, 0, 0};
  ProfState prof;
  int l_done = 0, march_nb = 0;   // march state for aim_march_continue
  bool use_graphs = true;
  std::string graph_error;
  std::vector<void*> allocs;
};

// helpers implemented in api.cu
void* aim_alloc(aim_ctx* c, size_t bytes);

// records events around one kernel launch when profiling is on; counts launches always
struct KScope {
  aim_ctx* c;
  int id;
  cudaEvent_t a = nullptr;
  KScope(aim_ctx* c_, int id_);
  ~KScope();
};
void prof_flush(aim_ctx* c);   // after a stream synchronisation
