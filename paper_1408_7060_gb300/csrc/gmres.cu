// Batched, restarted GMRES with a right preconditioner (the diagonal of Sec. 5.1, or the
// near-zone SAI) for the immediate system of Eq. 5 (Sec. 5.1: preconditioned GMRES, warm
// start from the previous step).  Krylov basis, Hessenberg matrix, Givens rotations and
// residuals are FP64; the operator is the ET-AIM matvec in the context's precision.
//
// Layout: the Krylov vectors are stored unnormalised, v_i = sig_i * vt_i, with the
// scales sig [B][64] kept beside the Hessenberg matrix.  The operator reads vt_j
// (times sig_j and the preconditioner) and writes A v_j straight into slot j+1, which
// classical Gram-Schmidt applied twice (CGS2) then orthogonalises in place -- no
// copies, no normalisation pass.  Reductions are two-stage with a fixed summation
// order (bitwise reproducible): partials per block, summed by the last block of each
// right-hand side to arrive (a fenced atomic counter, no waiting).  An Arnoldi step is
// the operator (whose interpolation kernel also forms the first pass's dots) and two
// update kernels (the second also finishes the column).  The column index j lives in
// device memory, so a whole solve is one CUDA graph: an outer conditional WHILE over
// restart cycles and an inner one over Arnoldi steps; kernels set the loop conditions.
#include <algorithm>
#include <cmath>
#include <functional>
#include <vector>

#include "aim_internal.h"
#include "gmres.h"
#include "operator.h"

namespace {

constexpr int kThreads = 256;
constexpr int kUpdN = 32;        // elements per update block (x 8 column groups)
constexpr int kNormChunk = 256;  // elements per norm-partial block

__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial sums of |v_b|^2 over chunks of kNormChunk: grid (P, nb); with vf non-null
// also the complex64 copy of v
__global__ void __launch_bounds__(kThreads) k_normpart(const double2* __restrict__ v, int ns,
                                                       double* __restrict__ pn, float2* __restrict__ vf) {
  const int b = blockIdx.y;
  const int n = blockIdx.x * kNormChunk + threadIdx.x;
  double a = 0;
  if (n < ns) {
    double2 x = v[(size_t)b * ns + n];
    a = x.x * x.x + x.y * x.y;
    if (vf) vf[(size_t)b * ns + n] = make_float2((float)x.x, (float)x.y);
  }
  __shared__ double red[kThreads / 32];
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int q = 0; q < kThreads / 32; ++q) s += red[q];
    pn[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
}

// sum of P partials of row b by one warp in a fixed order
__device__ __forceinline__ double warp_row_sum(const double* __restrict__ p, int P) {
  const int lane = threadIdx.x & 31;
  double s = 0;
  for (int q0 = 0; q0 < P; q0 += 256) {  // 8 loads per lane in flight, summed in order
    double v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int q = q0 + 32 * t + lane;
      v[t] = q < P ? p[q] : 0.0;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) s += v[t];
  }
  return warp_sum(s);
}

struct CycleArgs {
  int nb, restart, max_iter;
  double tol;
  const double* pb;   // partials of |b|^2   [nb][Pn]
  const double* pr;   // partials of |r|^2   [nb][Pn]
  int Pn;
  int use_cond;
  cudaGraphConditionalHandle outer, inner;
  int use_resid;                       // zero start: later cycles need the explicit residual
  cudaGraphConditionalHandle resid;
};

// cycle start: beta = |r| (explicit residual in slot 0), sig_0 = 1/beta, g = (beta, 0..),
// activity, j = 0, and both loop conditions.  One block, one warp per right-hand side.
__global__ void __launch_bounds__(kThreads) k_cycle_start(CycleArgs a, GmresState s) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int b = warp; b < a.nb; b += nw) {
    const double bn = sqrt(warp_row_sum(a.pb + (size_t)b * a.Pn, a.Pn));
    const double beta = sqrt(warp_row_sum(a.pr + (size_t)b * a.Pn, a.Pn));
    if (lane == 0) {
      s.bn[b] = bn;
      s.relres[b] = bn > 0 ? beta / bn : 0.0;
      const bool conv = !(bn > 0) || beta <= a.tol * bn;
      const bool cap = s.its[b] >= a.max_iter;
      s.done[b] = conv ? 1 : (cap ? 2 : 0);
      s.act[b] = s.done[b] == 0;
      s.jc[b] = 0;
      s.sig[b * 64] = beta > 0 ? 1.0 / beta : 0.0;
      s.g[b * 64] = make_double2(beta, 0.0);
      s.rho[b * 64] = make_double2(1.0, 0.0);
      if (s.act[b]) atomicOr(&any, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *s.jdev = 0;
    s.fin[0] = 0u;
    s.fin[1] = 0u;
    s.cnt[0] += 1;
    s.flag[0] = any;
    s.flag[1] = any;
    s.flag[2] = 0;
    if (a.use_cond) {
      cudaGraphSetConditional(a.outer, any ? 1u : 0u);
      cudaGraphSetConditional(a.inner, any ? 1u : 0u);
      if (a.use_resid) cudaGraphSetConditional(a.resid, 1u);
    }
  }
}

struct FinishArgs {
  int nb, restart, max_iter;
  double tol;
  int use_cond;
  cudaGraphConditionalHandle inner, outer;
};

// ---------------------------------------------------------------- CGS2 updates and column finish

// the same as warp_row_sum over partials that other blocks of the running kernel wrote
// (read through L2)
__device__ __forceinline__ double warp_row_sum_cg(const double* p, int P) {
  const int lane = threadIdx.x & 31;
  double s = 0;
  for (int q0 = 0; q0 < P; q0 += 256) {
    double v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int q = q0 + 32 * t + lane;
      v[t] = q < P ? __ldcg(p + q) : 0.0;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) s += v[t];
  }
  return warp_sum(s);
}

// complex partials p[0 .. P) summed by one warp in a fixed order (ld.cg when cg)
template <bool CG>
__device__ __forceinline__ double2 warp_row_sum_c(const double2* p, int P) {
  const int lane = threadIdx.x & 31;
  double2 t = make_double2(0, 0);
  for (int q = lane; q < P; q += 32) {
    const double2 v = CG ? __ldcg(p + q) : p[q];
    t.x += v.x;
    t.y += v.y;
  }
  return warp_sum_c(t);
}

// Column j of one RHS, by the warps 0 and 1 of the calling block (every thread calls it;
// hn2 = |w|^2 on thread 0).  The column h = h1 + h2 (entries 0..j) is stored unrotated in
// H[.][j]; the Givens rotations G_0..G_{j-1} reach it only through
//   p_j = (G_{j-1} ... G_0 h)_j = rho_j . h,
// where rho_j is row j of the accumulated rotation, kept from step to step by
// rho_{j+1} = (-conj(s_j) rho_j, c_j), rho_0 = (1).  With |w| the new rotation is
// c_j = |p|/r, s_j = (p/|p|) |w|/r, r^2 = |p|^2 + |w|^2, and R[j][j] = p r/|p|,
// g_{j+1} = -conj(s_j) g_j, g_j <- c_j g_j, the residual estimate
// |g_{j+1}|/|b| = relres_j |w|/r and sig_{j+1} = 1/|w| -- three reciprocal square roots
// and no division.  The rotated entries above the diagonal are formed once per cycle, in
// k_cycle_solve.  Returns (on every thread) whether the RHS takes another step.
__device__ bool finish_rhs(const FinishArgs& a, GmresState& s, int b, int j, double hn2) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ double sh_p2, sh_rp, sh_c;
  __shared__ double2 sh_p, sh_s;
  __shared__ int cont;
  double2 gj = make_double2(0, 0);
  double rel = 0, rhn = 0;
  int its = 0;
  if (tid == 0) {
    rhn = hn2 > 0 ? rsqrt(hn2) : 0.0;
    gj = s.g[b * 64 + j];
    rel = s.relres[b];
    its = s.its[b];
  } else if (warp == 1) {
    double2* H = s.H + (size_t)b * 64 * 64;  // H[i][k] at i*64 + k
    double2 acc = make_double2(0, 0);
    for (int i = lane; i <= j; i += 32) {
      const double2 x = __ldcg(s.h1 + b * 64 + i), y = __ldcg(s.h2 + b * 64 + i);
      const double2 h = make_double2(x.x + y.x, x.y + y.y);
      H[i * 64 + j] = h;
      const double2 r = s.rho[b * 64 + i];
      acc.x += r.x * h.x - r.y * h.y;
      acc.y += r.x * h.y + r.y * h.x;
    }
    const double2 pj = warp_sum_c(acc);
    if (lane == 0) {
      const double p2 = pj.x * pj.x + pj.y * pj.y;
      sh_p = pj;
      sh_p2 = p2;
      sh_rp = p2 > 0 ? rsqrt(p2) : 0.0;
    }
  }
  __syncthreads();
  if (tid == 0) {
    const double p2 = sh_p2, r2 = hn2 + p2;
    const double hn = hn2 * rhn;  // |w| (0 when |w| = 0)
    const double rr = r2 > 0 ? rsqrt(r2) : 0.0;
    const double2 pj = sh_p;
    double c;
    double2 sv, rjj;
    if (!(r2 > 0)) {
      c = 1.0;
      sv = make_double2(0, 0);
      rjj = make_double2(0, 0);
    } else if (!(p2 > 0)) {
      c = 0.0;
      sv = make_double2(1.0, 0.0);
      rjj = make_double2(hn, 0.0);
    } else {
      const double inv = rr * sh_rp;  // 1 / (|p| r)
      c = p2 * inv;
      const double q = hn * inv, t = r2 * inv;
      sv = make_double2(pj.x * q, pj.y * q);
      rjj = make_double2(pj.x * t, pj.y * t);
    }
    sh_s = sv;
    sh_c = c;
    s.cs[b * 64 + j] = c;
    s.sn[b * 64 + j] = sv;
    s.rd[b * 64 + j] = rjj;
    s.g[b * 64 + j] = make_double2(c * gj.x, c * gj.y);
    s.g[b * 64 + j + 1] = make_double2(-(sv.x * gj.x + sv.y * gj.y), -(sv.x * gj.y - sv.y * gj.x));
    rel *= hn * rr;  // |s_j| = |w| / r
    s.relres[b] = rel;
    s.jc[b] = j + 1;
    s.its[b] = its + 1;
    s.sig[b * 64 + j + 1] = rhn;
    const bool conv = rel <= a.tol || !(hn > 0);
    const bool stop = conv || its + 1 >= a.max_iter || j + 1 >= a.restart;
    if (conv) s.done[b] = 1;       // converged by the Arnoldi residual estimate
    else if (stop) s.flag[2] = 1;  // stopped by the cap or the restart length
    if (stop) s.act[b] = 0;
    cont = !stop;
  }
  __syncthreads();
  if (warp == 1) {  // rho_{j+1}
    const double2 sv = sh_s;
    for (int i = lane; i <= j + 1 && i < 64; i += 32) {
      double2 r;
      if (i <= j) {
        const double2 o = s.rho[b * 64 + i];
        r = make_double2(-(sv.x * o.x + sv.y * o.y), -(sv.x * o.y - sv.y * o.x));
      } else {
        r = make_double2(sh_c, 0.0);
      }
      s.rho[b * 64 + i] = r;
    }
  }
  return cont != 0;
}

// Thread 0 of the block that finished one RHS (or of block 0 of an inactive one): the
// last of the nb arrivals advances j and sets the loop conditions.
__device__ void finish_arrive(const FinishArgs& a, GmresState& s, int j, bool cont) {
  if (cont) atomicOr(s.fin + 1, 1u);
  __threadfence();
  if (atomicAdd(s.fin, 1u) != (unsigned)a.nb - 1) return;
  __threadfence();
  const bool any = atomicExch(s.fin + 1, 0u) != 0;
  atomicExch(s.fin, 0u);
  *s.jdev = j + 1;
  s.cnt[1] += 1;
  s.flag[1] = any;
  if (a.use_cond) cudaGraphSetConditional(a.inner, any ? 1u : 0u);
  // every RHS of this cycle converged by its estimate: no explicit residual and no
  // further cycle (the epilogue still applies the update)
  if (!any && !*(volatile int*)(s.flag + 2) && a.use_cond) cudaGraphSetConditional(a.outer, 0u);
}

constexpr int kCgsSub = 64;       // elements per sub-chunk: 64 lanes x 4 groups of basis vectors
constexpr int kCgsMaxE = 2048;    // elements per block at most
constexpr int kCgsTargetP = 256;  // blocks per RHS aimed at (the chunk grows beyond)

struct CgsArgs {
  double2* V;
  long long vstride;
  int ns, E, P;          // RHS length, elements per block (multiple of kCgsSub), blocks per RHS
  double2* pd1;          // raw dot partials of w (k_cgs_dots) [B][64][P]
  double2* d1;           // their sums: the first pass's dots [B][64]
  double2* pd2;          // first pass: raw dot partials of the updated w [B][64][P]
  double2* d2;           // their sums, by the last block of each RHS [B][64]
  double* pn;            // second pass: |w|^2 partials [B][P]
  unsigned* ucnt;        // [B] block arrivals per RHS
  float2* wf;            // second pass: complex64 copy of w (or null)
};

// Raw dots d_i = conj(vt_i) . w of the new vector w = slot j+1 with vt_0..vt_j, the
// first CGS pass's d, grid (P, nb) over the same element blocks as k_cgs: warp y takes
// i = y, y + 8, ... over the block's elements; the last block of each RHS sums the P
// partials in a fixed order into d1.
__global__ void __launch_bounds__(kThreads) k_cgs_dots(CgsArgs a, GmresState s) {
  pdl_wait();
  const int b = blockIdx.y, blk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (!s.act[b]) return;
  const int j = *s.jdev, J = j + 1;
  __shared__ int last;
  const double2* Vb = a.V + (size_t)b * a.ns;
  const double2* w = a.V + (size_t)J * a.vstride + (size_t)b * a.ns;
  const int n0 = blk * a.E, cnt = min(a.ns, n0 + a.E) - n0;
  for (int i = warp; i < J; i += kThreads / 32) {
    const double2* vi = Vb + i * a.vstride + n0;
    double2 t = make_double2(0, 0);
    for (int q = lane; q < cnt; q += 32) {
      const double2 p = cmulc(vi[q], w[n0 + q]);
      t.x += p.x;
      t.y += p.y;
    }
    t = warp_sum_c(t);
    if (lane == 0) a.pd1[((size_t)b * 64 + i) * a.P + blk] = t;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    last = atomicAdd(a.ucnt + b, 1u) == (unsigned)a.P - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    if (tid == 0) a.ucnt[b] = 0u;
    for (int i = warp; i < J; i += kThreads / 32) {
      const double2 d = warp_row_sum_c<true>(a.pd1 + ((size_t)b * 64 + i) * a.P, a.P);
      if (lane == 0) a.d1[b * 64 + i] = d;
    }
  }
  pdl_trigger();
}

// One classical Gram-Schmidt pass on slot j+1 of every active RHS, grid (P, nb):
//   h_i = sig_i d_i (d_i = sum of the raw dots conj(vt_i) . w, block 0 stores h),
//   w -= sum_i vt_i (sig_i h_i) on the block's E elements (64 at a time: 4 groups of
//   threads take every 4th basis vector, group 0 sums and writes),
// then for the first pass the raw dots of the updated w over the block's elements (warp y
// takes i = y, y + 8, ...), summed over the P blocks by the last block of the RHS into
// d2 -- the second pass's d; for the second pass |w|^2 over the block, summed by the last
// block, which then finishes column j (finish_rhs) and arrives at the step's counter.
template <int PASS>
__global__ void __launch_bounds__(kThreads) k_cgs(CgsArgs a, FinishArgs f, GmresState s) {
  pdl_wait();
  const int b = blockIdx.y, blk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int j = *s.jdev, J = j + 1;
  if (!s.act[b]) {
    if (PASS == 1 && blk == 0 && tid == 0) finish_arrive(f, s, j, false);
    return;
  }
  __shared__ double2 coef[64];
  __shared__ double2 red[4][kCgsSub];
  __shared__ double2 wsm[kCgsMaxE];
  __shared__ double nrd[kThreads / 32];
  __shared__ int last;
  // coefficients: warp y sums the raw dots of i = y, y + 8, ...
  for (int i = warp; i < J; i += kThreads / 32) {
    const double2 d = PASS == 0 ? a.d1[b * 64 + i] : a.d2[b * 64 + i];
    if (lane == 0) {
      const double sg = s.sig[b * 64 + i];
      const double2 h = make_double2(sg * d.x, sg * d.y);
      if (blk == 0) (PASS == 0 ? s.h1 : s.h2)[b * 64 + i] = h;
      coef[i] = make_double2(sg * h.x, sg * h.y);  // sig_i h_i multiplies vt_i
    }
  }
  __syncthreads();
  const double2* Vb = a.V + (size_t)b * a.ns;
  double2* w = a.V + (size_t)J * a.vstride + (size_t)b * a.ns;
  const int n0 = blk * a.E, cnt = min(a.ns, n0 + a.E) - n0;
  const int e = tid & (kCgsSub - 1), grp = tid / kCgsSub;
  for (int s0 = 0; s0 < cnt; s0 += kCgsSub) {
    const int n = n0 + s0 + e;
    const bool in = s0 + e < cnt;
    double2 pv = make_double2(0, 0);
    if (in)
      for (int i = grp; i < J; i += 4) {
        const double2 v = cmul(Vb[i * a.vstride + n], coef[i]);
        pv.x += v.x;
        pv.y += v.y;
      }
    red[grp][e] = pv;
    __syncthreads();
    if (grp == 0 && in) {
      double2 wv = w[n];
      wv.x -= (red[0][e].x + red[1][e].x) + (red[2][e].x + red[3][e].x);
      wv.y -= (red[0][e].y + red[1][e].y) + (red[2][e].y + red[3][e].y);
      w[n] = wv;
      if (PASS == 1 && a.wf) a.wf[(size_t)b * a.ns + n] = make_float2((float)wv.x, (float)wv.y);
      wsm[s0 + e] = wv;
    }
    __syncthreads();
  }
  if (PASS == 0) {
    for (int i = warp; i < J; i += kThreads / 32) {
      const double2* vi = Vb + i * a.vstride + n0;
      double2 t = make_double2(0, 0);
      for (int q = lane; q < cnt; q += 32) {
        const double2 p = cmulc(vi[q], wsm[q]);
        t.x += p.x;
        t.y += p.y;
      }
      t = warp_sum_c(t);
      if (lane == 0) a.pd2[((size_t)b * 64 + i) * a.P + blk] = t;
    }
  } else {
    double t = 0;
    for (int q = tid; q < cnt; q += kThreads) t += wsm[q].x * wsm[q].x + wsm[q].y * wsm[q].y;
    t = warp_sum(t);
    if (lane == 0) nrd[warp] = t;
    __syncthreads();
    if (tid == 0) {
      double u = 0;
      for (int q = 0; q < kThreads / 32; ++q) u += nrd[q];
      a.pn[(size_t)b * a.P + blk] = u;
    }
  }
  // the last block of this RHS to arrive sums the P partials
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    last = atomicAdd(a.ucnt + b, 1u) == (unsigned)a.P - 1;
  }
  __syncthreads();
  if (!last) {
    pdl_trigger();
    return;
  }
  __threadfence();
  if (tid == 0) a.ucnt[b] = 0u;
  if (PASS == 0) {
    for (int i = warp; i < J; i += kThreads / 32) {
      const double2 d = warp_row_sum_c<true>(a.pd2 + ((size_t)b * 64 + i) * a.P, a.P);
      if (lane == 0) a.d2[b * 64 + i] = d;
    }
  } else {
    double hn2 = 0;
    if (warp == 0) hn2 = warp_row_sum_cg(a.pn + (size_t)b * a.P, a.P);
    const bool cont = finish_rhs(f, s, b, j, hn2);
    if (tid == 0) finish_arrive(f, s, j, cont);
  }
  pdl_trigger();
}

// End of a cycle, one block per RHS: the rotated triangle R from the unrotated columns
// (G_0, G_1, ... applied in turn to every later column at once, one column per lane,
// with R[k][k] from the step that made the rotation), then R y = g by back substitution
// with the reciprocals of the diagonal taken up front; y is stored as sig_i y_i.
__global__ void __launch_bounds__(kThreads) k_cycle_solve(int nb, GmresState s) {
  extern __shared__ double2 hs[];  // [64][64]
  __shared__ double2 ys[64], dinv[64];
  const int b = blockIdx.x;
  const int n = s.jc[b];
  if (n == 0) return;
  const double2* H = s.H + (size_t)b * 64 * 64;
  for (int t = threadIdx.x; t < n * 64; t += blockDim.x) hs[t] = H[t];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = 0; i < n; ++i) {
      const double c = s.cs[b * 64 + i];
      const double2 sn = s.sn[b * 64 + i];
      for (int k = lane; k < n; k += 32) {
        if (k > i) {
          const double2 u = hs[i * 64 + k], v = hs[(i + 1) * 64 + k];
          hs[i * 64 + k] = make_double2(c * u.x + sn.x * v.x - sn.y * v.y, c * u.y + sn.x * v.y + sn.y * v.x);
          hs[(i + 1) * 64 + k] = make_double2(c * v.x - sn.x * u.x - sn.y * u.y, c * v.y - sn.x * u.y + sn.y * u.x);
        } else if (k == i) {
          hs[i * 64 + i] = s.rd[b * 64 + i];
        }
      }
      __syncwarp();
    }
    for (int i = lane; i < n; i += 32) {
      const double2 d = hs[i * 64 + i];
      const double dd = d.x * d.x + d.y * d.y;
      const double r = dd > 0 ? 1.0 / dd : 0.0;
      dinv[i] = make_double2(d.x * r, -d.y * r);
    }
    __syncwarp();
    for (int i = n - 1; i >= 0; --i) {
      double2 acc = make_double2(0, 0);
      for (int k = i + 1 + lane; k < n; k += 32) {
        const double2 p = cmul(hs[i * 64 + k], ys[k]);
        acc.x += p.x;
        acc.y += p.y;
      }
      acc = warp_sum_c(acc);
      if (lane == 0) {
        const double2 g = s.g[b * 64 + i];
        ys[i] = cmul(make_double2(g.x - acc.x, g.y - acc.y), dinv[i]);
      }
      __syncwarp();
    }
    for (int i = lane; i < n; i += 32) {
      const double sg = s.sig[b * 64 + i];
      s.y[b * 64 + i] = make_double2(sg * ys[i].x, sg * ys[i].y);
    }
  }
}

// x += dinv .* sum_i vt_i (sig_i y_i);  grid (ceil(ns/32), nb), block (32, 8)
// (with u non-null: u = sum_i vt_i (sig_i y_i) is stored instead, for the SAI below,
// and with uf non-null its complex64 copy as well)
__global__ void __launch_bounds__(kThreads) k_xupdate(const double2* __restrict__ V, long long vstride, int ns,
                                                      const double2* __restrict__ dinv, GmresState s,
                                                      double2* __restrict__ x, double2* __restrict__ u_out,
                                                      float2* __restrict__ uf) {
  const int b = blockIdx.y;
  const int J = s.jc[b];
  if (J == 0) return;
  __shared__ double2 red[8][kUpdN];
  const int n = blockIdx.x * kUpdN + threadIdx.x;
  double2 u = make_double2(0, 0);
  if (n < ns)
    for (int i = threadIdx.y; i < J; i += 8) {
      double2 p = cmul(V[i * vstride + (size_t)b * ns + n], s.y[b * 64 + i]);
      u.x += p.x;
      u.y += p.y;
    }
  red[threadIdx.y][threadIdx.x] = u;
  __syncthreads();
  if (threadIdx.y == 0 && n < ns) {
    double2 t = make_double2(0, 0);
    for (int q = 0; q < 8; ++q) {
      t.x += red[q][threadIdx.x].x;
      t.y += red[q][threadIdx.x].y;
    }
    if (u_out) {
      u_out[(size_t)b * ns + n] = t;
      if (uf) uf[(size_t)b * ns + n] = make_float2((float)t.x, (float)t.y);
      return;
    }
    const double2 du = cmul(dinv[n], t);
    double2 xv = x[(size_t)b * ns + n];
    x[(size_t)b * ns + n] = make_double2(xv.x + du.x, xv.y + du.y);
  }
}

// x_b += M u_b with the near-zone SAI (one warp per row, fixed-order warp sum); RHS with
// an empty cycle (jc = 0) are left alone.
__global__ void __launch_bounds__(kThreads) k_sai_xupdate(const double2* __restrict__ sai,
                                                          const int* __restrict__ rowptr,
                                                          const int* __restrict__ col, const double2* __restrict__ u,
                                                          int ns, int nb, GmresState s, double2* __restrict__ x) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (long long)nb * ns) return;
  const int b = (int)(w / ns), k = (int)(w % ns);
  if (s.jc[b] == 0) return;
  const double2* ub = u + (size_t)b * ns;
  double2 t = make_double2(0, 0);
  for (int e = rowptr[k] + lane; e < rowptr[k + 1]; e += 32) {
    const double2 p = cmul(sai[e], ub[col[e]]);
    t.x += p.x;
    t.y += p.y;
  }
  t = make_double2(warp_sum(t.x), warp_sum(t.y));
  if (lane == 0) {
    double2 xv = x[(size_t)b * ns + k];
    x[(size_t)b * ns + k] = make_double2(xv.x + t.x, xv.y + t.y);
  }
}

// The same on the complex64 path with the complex64 SAI (the M the Arnoldi process
// applied): 16 lanes per row, up to 9 entries per lane, FP32 products and butterfly sum,
// the sum added to x in FP64.
__global__ void __launch_bounds__(kThreads) k_sai_xupdate_c64(const float2* __restrict__ sai,
                                                              const int* __restrict__ rowptr,
                                                              const int* __restrict__ col,
                                                              const float2* __restrict__ uf, int ns, int nb,
                                                              GmresState s, double2* __restrict__ x) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 4;
  const int lane = threadIdx.x & 15;
  const bool valid = w < (long long)nb * ns;  // both rows of a warp join the shuffles
  const int b = valid ? (int)(w / ns) : 0, k = valid ? (int)(w % ns) : 0;
  const bool on = valid && s.jc[b] != 0;
  float tr = 0, ti = 0;
  if (on) {
    const float2* ub = uf + (size_t)b * ns;
    const int e0 = rowptr[k] + lane, e1 = rowptr[k + 1];
    int j[9];
    float2 m[9], u[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const int e = e0 + 16 * q;
      j[q] = e < e1 ? col[e] : -1;
      m[q] = e < e1 ? sai[e] : make_float2(0, 0);
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) u[q] = j[q] >= 0 ? ub[j[q]] : make_float2(0, 0);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      tr += m[q].x * u[q].x - m[q].y * u[q].y;
      ti += m[q].x * u[q].y + m[q].y * u[q].x;
    }
  }
  for (int o = 8; o > 0; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    ti += __shfl_xor_sync(0xffffffffu, ti, o);
  }
  if (on && lane == 0) {
    double2 xv = x[(size_t)b * ns + k];
    x[(size_t)b * ns + k] = make_double2(xv.x + (double)tr, xv.y + (double)ti);
  }
}

// |v_b| for every b into out[b]
__global__ void __launch_bounds__(kThreads) k_norm_finish(int nb, const double* __restrict__ pn, int P, double* __restrict__ out) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = warp; b < nb; b += nw) {
    double v = sqrt(warp_row_sum(pn + (size_t)b * P, P));
    if ((threadIdx.x & 31) == 0) out[b] = v;
  }
}

int n_upd_blocks(int ns) { return (ns + kUpdN - 1) / kUpdN; }
int n_norm_blocks(int ns) { return (ns + kNormChunk - 1) / kNormChunk; }

// ---------------------------------------------------------------- launch sequences

// explicit residual into slot 0 and the cycle start
// explicit residual into slot 0 (slot 0 = b - Z_0 x); with a zero start, the first
// cycle's residual is b itself (the caller copies it and skips this)
void cycle_residual(aim_ctx* c, int nb, const double2* b, double2* x) {
  op_apply(c, 0, nb, x, nullptr, b, -1.0, nullptr, c->d_V);
}

void copy_b_to_slot0(aim_ctx* c, int nb, const double2* b) {
  AIM_CUDA(cudaMemcpyAsync(c->d_V, b, (size_t)nb * c->ns * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
}

// the complex64 copy of the Krylov vector that the SAI application of the complex64 path
// gathers from (null when that path is not in use)
float2* krylov_c64(aim_ctx* c) { return c->d_sai && c->precision == AIM_C64 ? c->d_vf : nullptr; }

// |r|^2 of slot 0 and the cycle start
void cycle_start(aim_ctx* c, int nb, double tol, bool use_cond, cudaGraphConditionalHandle outer,
                 cudaGraphConditionalHandle inner, cudaGraphConditionalHandle resid, bool zs) {
  GmresState& s = c->gs;
  cudaStream_t st = c->stream;
  const int ns = c->ns;
  AIM_KLAUNCH(c, AIM_K_GMRES_UPDATE,
              k_normpart<<<dim3(n_norm_blocks(ns), nb), kThreads, 0, st>>>(c->d_V, ns, s.pr, krylov_c64(c)));
  CycleArgs a{nb, c->restart, c->max_iter, tol, s.pbn, s.pr, n_norm_blocks(ns), use_cond ? 1 : 0, outer, inner,
              (use_cond && zs) ? 1 : 0, resid};
  AIM_KLAUNCH(c, AIM_K_GMRES_SMALL, k_cycle_start<<<1, kThreads, 0, st>>>(a, s));
}

// slot j+1 = Z_0 (dinv .* v_j) for every active RHS (column j from device memory)
void arnoldi_operator(aim_ctx* c, int nb) {
  GmresState& s = c->gs;
  const int ns = c->ns;
  const long long vstride = (long long)c->batch_max * ns;
  VecSel vin;
  vin.sel = s.jdev;
  vin.stride = vstride;
  vin.off = 0;
  vin.scale = s.sig;
  VecSel vout;
  vout.sel = s.jdev;
  vout.stride = vstride;
  vout.off = 1;
  if (s.interp_P > 0) {  // the interpolation kernel also forms the first pass's dots
    c->dotfuse.V = c->d_V;
    c->dotfuse.vstride = vstride;
    c->dotfuse.jdev = s.jdev;
    c->dotfuse.pd = s.pdi;
    c->dotfuse.d = s.d1;
    c->dotfuse.ucnt = s.ucnt;
    c->dotfuse.P = s.interp_P;
  }
  try {
    op_apply(c, 0, nb, c->d_V, c->d_dinv, nullptr, 1.0, s.act, c->d_V, vin, vout);
  } catch (...) {
    c->dotfuse = DotFuse();
    throw;
  }
  c->dotfuse = DotFuse();
}

// one Arnoldi step for every active RHS: operator into slot j+1, CGS2, column finish
void arnoldi_step(aim_ctx* c, int nb, double tol, bool use_cond, cudaGraphConditionalHandle inner,
                  cudaGraphConditionalHandle outer) {
  GmresState& s = c->gs;
  cudaStream_t st = c->stream;
  const int ns = c->ns;
  const long long vstride = (long long)c->batch_max * ns;
  arnoldi_operator(c, nb);
  FinishArgs f{nb, c->restart, c->max_iter, tol, use_cond ? 1 : 0, inner, outer};
  CgsArgs a{c->d_V, vstride, ns, s.cgs_E, s.cgs_P, s.pd, s.d1, s.pd2, s.d2, s.pu, s.ucnt, krylov_c64(c)};
  if (s.interp_P == 0)
    AIM_KLAUNCH(c, AIM_K_GMRES_DOT, launch_pdl(st, dim3(s.cgs_P, nb), dim3(kThreads), 0, k_cgs_dots, a, s));
  AIM_KLAUNCH(c, AIM_K_GMRES_UPDATE,
              launch_pdl(st, dim3(s.cgs_P, nb), dim3(kThreads), 0, k_cgs<0>, a, f, s));
  AIM_KLAUNCH(c, AIM_K_GMRES_UPDATE,
              launch_pdl(st, dim3(s.cgs_P, nb), dim3(kThreads), 0, k_cgs<1>, a, f, s));
}

void cycle_epilogue(aim_ctx* c, int nb, double2* x) {
  GmresState& s = c->gs;
  cudaStream_t st = c->stream;
  const int ns = c->ns;
  const long long vstride = (long long)c->batch_max * ns;
  AIM_KLAUNCH(c, AIM_K_GMRES_SMALL, k_cycle_solve<<<nb, kThreads, 64 * 64 * sizeof(double2), st>>>(nb, s));
  AIM_KLAUNCH(c, AIM_K_GMRES_SMALL,
              k_xupdate<<<dim3(n_upd_blocks(ns), nb), dim3(kUpdN, 8), 0, st>>>(c->d_V, vstride, ns, c->d_dinv, s, x,
                                                                                c->d_sai ? c->d_u : nullptr,
                                                                                krylov_c64(c)));
  if (krylov_c64(c)) {
    const long long rows = (long long)nb * ns;
    AIM_KLAUNCH(c, AIM_K_GMRES_SMALL,
                k_sai_xupdate_c64<<<(int)((rows * 16 + kThreads - 1) / kThreads), kThreads, 0, st>>>(
                    c->d_saif, c->d_srowptr, c->d_scol, krylov_c64(c), ns, nb, s, x));
  } else if (c->d_sai) {
    const long long warps = (long long)nb * ns;
    AIM_KLAUNCH(c, AIM_K_GMRES_SMALL,
                k_sai_xupdate<<<(int)((warps * 32 + kThreads - 1) / kThreads), kThreads, 0, st>>>(
                    c->d_sai, c->d_srowptr, c->d_scol, c->d_u, ns, nb, s, x));
  }
}

// ---------------------------------------------------------------- graph of one solve

cudaGraphNode_t leaf_of(cudaGraph_t g) {
  size_t n = 0;
  AIM_CUDA(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  AIM_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
  for (auto nd : nodes) {
    size_t out = 0;
    AIM_CUDA(cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &out));
    if (out == 0) return nd;
  }
  throw AimError{AIM_ERR_CUDA, "graph without a leaf node"};
}

void capture_into(aim_ctx* c, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                  const std::function<void()>& body) {
  AIM_CUDA(cudaStreamBeginCaptureToGraph(c->stream, g, deps, nullptr, ndeps, cudaStreamCaptureModeThreadLocal));
  try {
    body();
  } catch (...) {
    cudaGraph_t dummy;
    cudaStreamEndCapture(c->stream, &dummy);
    cudaGetLastError();
    throw;
  }
  cudaGraph_t out;
  AIM_CUDA(cudaStreamEndCapture(c->stream, &out));
}

cudaGraphNode_t add_cond(cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps, cudaGraphConditionalHandle h,
                         cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  AIM_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &p));
  *body = p.conditional.phGraph_out[0];
  return node;
}

void build_solve_graph(aim_ctx* c, int nb, const double2* b, double2* x, double tol, bool zs) {
  GmresState& s = c->gs;
  GmresState::SolveGraph& sg = s.graphs[zs ? 1 : 0];
  cudaGraph_t g;
  AIM_CUDA(cudaGraphCreate(&g, 0));
  const ProfState saved = c->prof;  // capture-time launches are not executions
  c->prof.on = false;                // no event records inside a captured graph
  try {
    // |b|^2 partials, then WHILE(cycles) { prologue; WHILE(arnoldi) { step }; epilogue }
    capture_into(c, g, nullptr, 0, [&] {
      AIM_KLAUNCH(c, AIM_K_GMRES_UPDATE,
                  k_normpart<<<dim3(n_norm_blocks(c->ns), nb), kThreads, 0, c->stream>>>(b, c->ns, s.pbn, nullptr));
    });
    cudaGraphNode_t pre = leaf_of(g);
    cudaGraphConditionalHandle outer, inner, resid = 0;
    AIM_CUDA(cudaGraphConditionalHandleCreate(&outer, g, 1, cudaGraphCondAssignDefault));
    if (zs)  // 0 for the first cycle of every launch; the cycle start sets it to 1
      AIM_CUDA(cudaGraphConditionalHandleCreate(&resid, g, 0, cudaGraphCondAssignDefault));
    cudaGraph_t obody;
    add_cond(g, &pre, 1, outer, cudaGraphCondTypeWhile, &obody);
    AIM_CUDA(cudaGraphConditionalHandleCreate(&inner, obody, 0, cudaGraphCondAssignDefault));
    if (zs) {
      // slot 0 = b; IF(resid) { slot 0 = b - Z_0 x }; |r|^2 and the cycle start
      capture_into(c, obody, nullptr, 0, [&] { copy_b_to_slot0(c, nb, b); });
      cudaGraphNode_t cp = leaf_of(obody);
      cudaGraph_t rbody;
      cudaGraphNode_t rn = add_cond(obody, &cp, 1, resid, cudaGraphCondTypeIf, &rbody);
      capture_into(c, rbody, nullptr, 0, [&] { cycle_residual(c, nb, b, x); });
      capture_into(c, obody, &rn, 1, [&] { cycle_start(c, nb, tol, true, outer, inner, resid, zs); });
    } else {
      capture_into(c, obody, nullptr, 0, [&] {
        cycle_residual(c, nb, b, x);
        cycle_start(c, nb, tol, true, outer, inner, resid, zs);
      });
    }
    cudaGraphNode_t pro = leaf_of(obody);
    cudaGraph_t ibody;
    cudaGraphNode_t wn = add_cond(obody, &pro, 1, inner, cudaGraphCondTypeWhile, &ibody);
    capture_into(c, ibody, nullptr, 0, [&] { arnoldi_step(c, nb, tol, true, inner, outer); });
    capture_into(c, obody, &wn, 1, [&] { cycle_epilogue(c, nb, x); });
    cudaGraphExec_t ex;
    AIM_CUDA(cudaGraphInstantiate(&ex, g, 0));
    if (sg.exec) cudaGraphExecDestroy(sg.exec);
    if (sg.graph) cudaGraphDestroy(sg.graph);
    sg.graph = g;
    sg.exec = ex;
    sg.nb = nb;
    sg.tol = tol;
    sg.b = b;
    sg.x = x;
    sg.near = c->d_near;
  } catch (...) {
    c->prof = saved;
    cudaGraphDestroy(g);
    throw;
  }
  c->prof = saved;
}

}  // namespace

void gmres_alloc(aim_ctx* c) {
  const int B = c->batch_max, ns = c->ns;
  GmresState& s = c->gs;
  s.H = (double2*)aim_alloc(c, (size_t)B * 64 * 64 * sizeof(double2));
  s.rd = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  s.rho = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  s.fin = (unsigned*)aim_alloc(c, 2 * sizeof(unsigned));
  AIM_CUDA(cudaMemset(s.fin, 0, 2 * sizeof(unsigned)));
  s.g = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  s.sn = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  s.cs = (double*)aim_alloc(c, (size_t)B * 64 * sizeof(double));
  s.y = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  s.h1 = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  s.h2 = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  s.sig = (double*)aim_alloc(c, (size_t)B * 64 * sizeof(double));
  s.bn = (double*)aim_alloc(c, B * sizeof(double));
  s.relres = (double*)aim_alloc(c, B * sizeof(double));
  s.act = (int*)aim_alloc(c, B * sizeof(int));
  s.done = (int*)aim_alloc(c, B * sizeof(int));
  s.jc = (int*)aim_alloc(c, B * sizeof(int));
  s.its = (int*)aim_alloc(c, B * sizeof(int));
  s.jdev = (int*)aim_alloc(c, sizeof(int));
  s.flag = (int*)aim_alloc(c, 3 * sizeof(int));
  // CGS update blocks: E elements each (a multiple of 64), about kCgsTargetP per RHS
  s.cgs_E = std::min(kCgsMaxE, std::max(kCgsSub, ((ns + kCgsTargetP - 1) / kCgsTargetP + kCgsSub - 1) / kCgsSub * kCgsSub));
  s.cgs_P = (ns + s.cgs_E - 1) / s.cgs_E;
  s.pu = (double*)aim_alloc(c, (size_t)B * s.cgs_P * sizeof(double));
  s.pd = (double2*)aim_alloc(c, (size_t)B * 64 * s.cgs_P * sizeof(double2));
  s.d1 = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  // the interpolation kernel forms the first pass's dots when its blocks of 32 rows are
  // few enough for one block to sum their partials
  const int pi = (ns + 31) / 32;
  s.interp_P = pi <= 1024 ? pi : 0;
  if (s.interp_P) s.pdi = (double2*)aim_alloc(c, (size_t)B * 64 * s.interp_P * sizeof(double2));
  s.pd2 = (double2*)aim_alloc(c, (size_t)B * 64 * s.cgs_P * sizeof(double2));
  s.d2 = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  s.ucnt = (unsigned*)aim_alloc(c, (size_t)B * sizeof(unsigned));
  AIM_CUDA(cudaMemset(s.ucnt, 0, (size_t)B * sizeof(unsigned)));
  s.pr = (double*)aim_alloc(c, (size_t)B * n_norm_blocks(ns) * sizeof(double));
  s.pbn = (double*)aim_alloc(c, (size_t)B * n_norm_blocks(ns) * sizeof(double));
  s.nrm = (double*)aim_alloc(c, B * sizeof(double));
  s.cnt = (int*)aim_alloc(c, 2 * sizeof(int));
  AIM_CUDA(cudaMallocHost(&s.h_cnt, 2 * sizeof(int)));
  AIM_CUDA(cudaFuncSetAttribute(k_cycle_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(64 * 64 * sizeof(double2))));
  AIM_CUDA(cudaMallocHost(&s.h_flag, 3 * sizeof(int)));
  AIM_CUDA(cudaMallocHost(&s.h_its, B * sizeof(int)));
  AIM_CUDA(cudaMallocHost(&s.h_res, B * sizeof(double)));
  AIM_CUDA(cudaMallocHost(&s.h_done, B * sizeof(int)));
}

void gmres_free_host(aim_ctx* c) {
  GmresState& s = c->gs;
  for (auto& sg : s.graphs) {
    if (sg.exec) cudaGraphExecDestroy(sg.exec);
    if (sg.graph) cudaGraphDestroy(sg.graph);
    sg.exec = nullptr;
    sg.graph = nullptr;
  }
  if (s.h_flag) cudaFreeHost(s.h_flag);
  if (s.h_its) cudaFreeHost(s.h_its);
  if (s.h_res) cudaFreeHost(s.h_res);
  if (s.h_done) cudaFreeHost(s.h_done);
  if (s.h_cnt) cudaFreeHost(s.h_cnt);
  s.h_cnt = nullptr;
  s.h_flag = nullptr;
  s.h_its = nullptr;
  s.h_res = nullptr;
  s.h_done = nullptr;
}

// Solve Z_0 x = b for nb right-hand sides; x holds the initial guess on entry.
// Returns AIM_OK or AIM_ERR_NOCONV; per-RHS iteration counts and final relative
// residuals land in iters / relres (host arrays, may be null).
// Enqueue the solve and the copies of its statistics to pinned host memory; they are read
// by gmres_collect once the caller has synchronised the stream (the host-driven mode
// synchronises inside).
void gmres_solve_async(aim_ctx* c, int nb, const double2* b, double2* x, double tol) {
  gmres_solve_async(c, nb, b, x, tol, c->zero_start);
}

// zs: start from zero (x must hold zeros; the first residual is b itself, no operator
// product) instead of the guess in x
void gmres_solve_async(aim_ctx* c, int nb, const double2* b, double2* x, double tol, bool zs) {
  GmresState& s = c->gs;
  cudaStream_t st = c->stream;
  AIM_CUDA(cudaMemsetAsync(s.its, 0, nb * sizeof(int), st));
  AIM_CUDA(cudaMemsetAsync(s.cnt, 0, 2 * sizeof(int), st));
  bool graphed = false;
  // per-kernel event timing needs host-side launches: profiling runs the host-driven loop
  if (c->use_graphs && !s.graph_failed && !c->prof.on) {
    try {
      const GmresState::SolveGraph& sg = s.graphs[zs ? 1 : 0];
      if (!sg.exec || sg.nb != nb || sg.tol != tol || sg.b != b || sg.x != x || sg.near != c->d_near)
        build_solve_graph(c, nb, b, x, tol, zs);
      AIM_CUDA(cudaGraphLaunch(sg.exec, st));
      graphed = true;
    } catch (const AimError& e) {
      s.graph_failed = true;
      c->graph_error = e.msg;
      cudaGetLastError();
    }
  }
  if (!graphed) {
    // the same kernels driven from the host (one synchronisation per Arnoldi step)
    AIM_KLAUNCH(c, AIM_K_GMRES_UPDATE,
                k_normpart<<<dim3(n_norm_blocks(c->ns), nb), kThreads, 0, st>>>(b, c->ns, s.pbn, nullptr));
    for (int cycle = 0;; ++cycle) {
      if (zs && cycle == 0) copy_b_to_slot0(c, nb, b);
      else cycle_residual(c, nb, b, x);
      cycle_start(c, nb, tol, false, 0, 0, 0, zs);
      AIM_CUDA(cudaMemcpyAsync(s.h_flag, s.flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
      AIM_CUDA(cudaStreamSynchronize(st));
      if (!s.h_flag[0]) break;
      for (;;) {
        arnoldi_step(c, nb, tol, false, 0, 0);
        AIM_CUDA(cudaMemcpyAsync(s.h_flag, s.flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
        AIM_CUDA(cudaStreamSynchronize(st));
        if (!s.h_flag[1]) break;
      }
      cycle_epilogue(c, nb, x);
      AIM_CUDA(cudaMemcpyAsync(s.h_flag, s.flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
      AIM_CUDA(cudaStreamSynchronize(st));
      if (!s.h_flag[2]) break;  // every RHS converged by its estimate (as in the graph)
      if (cycle > 4 * (c->max_iter / std::max(1, c->restart) + 2)) break;
    }
  }
  AIM_CUDA(cudaMemcpyAsync(s.h_its, s.its, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
  AIM_CUDA(cudaMemcpyAsync(s.h_res, s.relres, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  AIM_CUDA(cudaMemcpyAsync(s.h_done, s.done, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
  AIM_CUDA(cudaMemcpyAsync(s.h_cnt, s.cnt, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  s.last_graphed = graphed;
  s.last_zs = zs;
  s.last_nb = nb;
}

int gmres_collect(aim_ctx* c, int* iters, double* relres) {
  GmresState& s = c->gs;
  const int nb = s.last_nb;
  if (s.last_graphed) {
    // kernels the graph executed: 1 + cycles * (prologue: operator + 2, epilogue 2, + 1
    // with the SAI) + steps * (operator + dots + 2 updates, the dots inside the operator's
    // interpolation kernel when it forms them); a zero start skips
    // the operator of the first cycle
    const long long op = op_kernel_count(c);
    const long long krylov = s.interp_P > 0 ? 2 : 3;
    c->prof.launches += 1 + (op + 4 + (c->d_sai ? 1 : 0)) * s.h_cnt[0] + (op + krylov) * s.h_cnt[1] -
                        (s.last_zs && s.h_cnt[0] > 0 ? op : 0);
  }
  int rc = AIM_OK;
  for (int i = 0; i < nb; ++i) {
    if (iters) iters[i] = s.h_its[i];
    if (relres) relres[i] = s.h_res[i];
    if (s.h_done[i] != 1) rc = AIM_ERR_NOCONV;
  }
  return rc;
}

int gmres_solve(aim_ctx* c, int nb, const double2* b, double2* x, double tol, int* iters, double* relres) {
  gmres_solve_async(c, nb, b, x, tol);
  AIM_CUDA(cudaStreamSynchronize(c->stream));
  return gmres_collect(c, iters, relres);
}

int gmres_blocks(int ns) { return n_norm_blocks(ns); }

namespace {
__global__ void __launch_bounds__(kThreads) k_axpy(long long n, const double2* __restrict__ a, double2* __restrict__ x) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) {
    const double2 u = a[i], v = x[i];
    x[i] = make_double2(v.x + u.x, v.y + u.y);
  }
}
}  // namespace

void gmres_axpy(aim_ctx* c, int nb, const double2* a, double2* x) {
  const long long n = (long long)nb * c->ns;
  AIM_KLAUNCH(c, AIM_K_GMRES_SMALL, k_axpy<<<(int)((n + kThreads - 1) / kThreads), kThreads, 0, c->stream>>>(n, a, x));
}

void gmres_norms(aim_ctx* c, int nb, const double2* v, double* d_out) {
  const int P = n_norm_blocks(c->ns);
  AIM_KLAUNCH(c, AIM_K_GMRES_UPDATE, k_normpart<<<dim3(P, nb), kThreads, 0, c->stream>>>(v, c->ns, c->gs.pr, nullptr));
  AIM_KLAUNCH(c, AIM_K_GMRES_SMALL, k_norm_finish<<<1, kThreads, 0, c->stream>>>(nb, c->gs.pr, P, d_out));
}
