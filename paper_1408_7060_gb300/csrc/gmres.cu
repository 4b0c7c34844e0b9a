// Batched, restarted GMRES with right diagonal preconditioning for the immediate
// system of Eq. 5 (Sec. 5.1: diagonally preconditioned GMRES, warm start from the
// previous step).  Krylov basis, Hessenberg matrix, Givens rotations and residuals
// are FP64; the operator is the ET-AIM matvec in the context's precision.
// Orthogonalisation is classical Gram-Schmidt applied twice (CGS2), so each
// Arnoldi step needs two multi-vector reductions instead of j sequential ones.
// Every reduction is two-stage with a fixed summation order (bitwise reproducible).
#include <algorithm>
#include <cmath>
#include <vector>

#include "aim_internal.h"
#include "gmres.h"
#include "operator.h"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// h[b][i] = sum_n conj(V_i[b][n]) w[b][n], i < J.  grid (nblk, nb).
__global__ void k_dots(const double2* __restrict__ V, size_t vstride, int J, const double2* __restrict__ w, int ns,
                       int nb, const int* __restrict__ act, double2* __restrict__ partial, unsigned* __restrict__ counter,
                       double2* __restrict__ h) {
  const int b = blockIdx.y;
  if (!act[b]) return;
  __shared__ double2 red[64][kThreads / 32];
  __shared__ bool last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double2* wb = w + (size_t)b * ns;
  for (int i = 0; i < J; ++i) {
    const double2* vb = V + i * vstride + (size_t)b * ns;
    double2 acc = make_double2(0, 0);
    for (int n = blockIdx.x * kThreads + threadIdx.x; n < ns; n += gridDim.x * kThreads) {
      double2 p = cmulc(vb[n], wb[n]);
      acc.x += p.x;
      acc.y += p.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) red[i][warp] = acc;
  }
  __syncthreads();
  double2* pb = partial + ((size_t)b * gridDim.x + blockIdx.x) * 64;
  if (threadIdx.x < J) {
    double2 s = make_double2(0, 0);
    for (int q = 0; q < kThreads / 32; ++q) {
      s.x += red[threadIdx.x][q].x;
      s.y += red[threadIdx.x][q].y;
    }
    pb[threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&counter[b], 1u) == gridDim.x - 1;
  __syncthreads();
  if (last) {
    if (threadIdx.x < J) {
      double2 s = make_double2(0, 0);
      for (int q = 0; q < (int)gridDim.x; ++q) {
        double2 v = __ldcg(&partial[((size_t)b * gridDim.x + q) * 64 + threadIdx.x]);
        s.x += v.x;
        s.y += v.y;
      }
      h[(size_t)b * 64 + threadIdx.x] = s;
    }
    if (threadIdx.x == 0) counter[b] = 0;
  }
}

// w -= sum_{i<J} V_i h_i ; optionally ||w||^2 -> nrm[b] (two-stage).  grid (nblk, nb).
__global__ void k_update(const double2* __restrict__ V, size_t vstride, int J, const double2* __restrict__ h,
                         double2* __restrict__ w, int ns, const int* __restrict__ act, bool want_norm,
                         double* __restrict__ partial, unsigned* __restrict__ counter, double* __restrict__ nrm) {
  const int b = blockIdx.y;
  if (!act[b]) return;
  __shared__ double hs[2 * 64];
  __shared__ double red[kThreads / 32];
  __shared__ bool last;
  for (int i = threadIdx.x; i < J; i += kThreads) {
    hs[2 * i] = h[(size_t)b * 64 + i].x;
    hs[2 * i + 1] = h[(size_t)b * 64 + i].y;
  }
  __syncthreads();
  double acc = 0;
  double2* wb = w + (size_t)b * ns;
  for (int n = blockIdx.x * kThreads + threadIdx.x; n < ns; n += gridDim.x * kThreads) {
    double2 s = wb[n];
    for (int i = 0; i < J; ++i) {
      double2 v = V[i * vstride + (size_t)b * ns + n];
      double2 p = cmul(v, make_double2(hs[2 * i], hs[2 * i + 1]));
      s.x -= p.x;
      s.y -= p.y;
    }
    wb[n] = s;
    acc += s.x * s.x + s.y * s.y;
  }
  if (!want_norm) return;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int q = 0; q < kThreads / 32; ++q) s += red[q];
    partial[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&counter[b], 1u) == gridDim.x - 1;
  __syncthreads();
  if (last && threadIdx.x == 0) {
    double s = 0;
    for (int q = 0; q < (int)gridDim.x; ++q) s += __ldcg(&partial[(size_t)b * gridDim.x + q]);
    nrm[b] = sqrt(s);
    counter[b] = 0;
  }
}

// ||v_b|| for every b (two-stage).  grid (nblk, nb).
__global__ void k_norms(const double2* __restrict__ v, int ns, double* __restrict__ partial,
                        unsigned* __restrict__ counter, double* __restrict__ nrm) {
  const int b = blockIdx.y;
  __shared__ double red[kThreads / 32];
  __shared__ bool last;
  double acc = 0;
  const double2* vb = v + (size_t)b * ns;
  for (int n = blockIdx.x * kThreads + threadIdx.x; n < ns; n += gridDim.x * kThreads) {
    double2 s = vb[n];
    acc += s.x * s.x + s.y * s.y;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int q = 0; q < kThreads / 32; ++q) s += red[q];
    partial[(size_t)b * gridDim.x + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&counter[b], 1u) == gridDim.x - 1;
  __syncthreads();
  if (last && threadIdx.x == 0) {
    double s = 0;
    for (int q = 0; q < (int)gridDim.x; ++q) s += __ldcg(&partial[(size_t)b * gridDim.x + q]);
    nrm[b] = sqrt(s);
    counter[b] = 0;
  }
}

// start of a cycle: beta = ||r||, V_0 = r/beta, g = (beta, 0, ...), activity from the
// explicit residual.  One thread per b (small state only); scaling in k_scale.
__global__ void k_cycle_start(int nb, int restart, double tol, int max_iter, const double* __restrict__ rn,
                              const double* __restrict__ bn, GmresState s) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const double beta = rn[b];
  s.relres[b] = bn[b] > 0 ? beta / bn[b] : 0.0;
  const bool conv = !(bn[b] > 0) || beta <= tol * bn[b];
  const bool cap = s.its[b] >= max_iter;
  s.done[b] = conv ? 1 : (cap ? 2 : 0);
  s.act[b] = s.done[b] == 0;
  s.jc[b] = 0;
  s.scale[b] = beta > 0 ? 1.0 / beta : 0.0;
  for (int i = 0; i <= restart; ++i) s.g[(size_t)b * 64 + i] = make_double2(i == 0 ? beta : 0.0, 0.0);
}

// v_out[b] = v_in[b] * scale[b] for active b.  grid (nblk, nb).
__global__ void k_scale(const double2* __restrict__ in, double2* __restrict__ out, int ns,
                        const int* __restrict__ act, const double* __restrict__ scale) {
  const int b = blockIdx.y;
  if (!act[b]) return;
  const double sc = scale[b];
  for (int n = blockIdx.x * kThreads + threadIdx.x; n < ns; n += gridDim.x * kThreads) {
    double2 v = in[(size_t)b * ns + n];
    out[(size_t)b * ns + n] = make_double2(sc * v.x, sc * v.y);
  }
}

// Arnoldi column j: H[0..j][j] = h1 + h2, H[j+1][j] = ||w||; previous rotations,
// a new complex Givens rotation, residual estimate |g_{j+1}|, convergence / cap.
__global__ void k_arnoldi_finish(int nb, int j, int restart, double tol, int max_iter, const double2* __restrict__ h1,
                                 const double2* __restrict__ h2, const double* __restrict__ hn,
                                 const double* __restrict__ bn, GmresState s) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || !s.act[b]) return;
  double2* H = s.H + (size_t)b * 64 * 64;  // H[i][j] at i*64 + j
  double2 col[65];
  for (int i = 0; i <= j; ++i) {
    double2 a = h1[(size_t)b * 64 + i], c = h2[(size_t)b * 64 + i];
    col[i] = make_double2(a.x + c.x, a.y + c.y);
  }
  col[j + 1] = make_double2(hn[b], 0.0);
  for (int i = 0; i < j; ++i) {  // apply G_i: [c s; -conj(s) c]
    double c = s.cs[(size_t)b * 64 + i];
    double2 sn = s.sn[(size_t)b * 64 + i];
    double2 a = col[i], d = col[i + 1];
    double2 sd = cmul(sn, d);
    double2 csa = make_double2(sn.x * a.x + sn.y * a.y, sn.x * a.y - sn.y * a.x);  // conj(sn) a
    col[i] = make_double2(c * a.x + sd.x, c * a.y + sd.y);
    col[i + 1] = make_double2(c * d.x - csa.x, c * d.y - csa.y);
  }
  double2 a = col[j], d = col[j + 1];
  double na = sqrt(a.x * a.x + a.y * a.y), nd = sqrt(d.x * d.x + d.y * d.y);
  double r = sqrt(na * na + nd * nd);
  double c;
  double2 sn;
  if (r == 0.0) {
    c = 1.0;
    sn = make_double2(0, 0);
  } else if (na == 0.0) {
    c = 0.0;
    sn = make_double2(d.x / nd, -d.y / nd);
  } else {
    c = na / r;
    double2 ph = make_double2(a.x / na, a.y / na);
    sn = cmul(ph, make_double2(d.x / r, -d.y / r));  // (a/|a|) conj(d)/r
  }
  s.cs[(size_t)b * 64 + j] = c;
  s.sn[(size_t)b * 64 + j] = sn;
  col[j] = make_double2(c * a.x + (sn.x * d.x - sn.y * d.y), c * a.y + (sn.x * d.y + sn.y * d.x));
  col[j + 1] = make_double2(0, 0);
  for (int i = 0; i <= j; ++i) H[i * 64 + j] = col[i];
  double2 gj = s.g[(size_t)b * 64 + j];
  s.g[(size_t)b * 64 + j] = make_double2(c * gj.x, c * gj.y);
  double2 gn = make_double2(-(sn.x * gj.x + sn.y * gj.y), -(sn.x * gj.y - sn.y * gj.x));  // -conj(sn) g_j
  s.g[(size_t)b * 64 + j + 1] = gn;
  s.jc[b] = j + 1;
  s.its[b] += 1;
  const double res = sqrt(gn.x * gn.x + gn.y * gn.y);
  s.relres[b] = res / bn[b];
  s.scale[b] = hn[b] > 0 ? 1.0 / hn[b] : 0.0;
  if (res <= tol * bn[b] || !(hn[b] > 0) || s.its[b] >= max_iter || j + 1 >= restart) s.act[b] = 0;
}

// y = H^{-1} g on the jc x jc triangle, per b
__global__ void k_cycle_solve(int nb, GmresState s) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int n = s.jc[b];
  const double2* H = s.H + (size_t)b * 64 * 64;
  double2* y = s.y + (size_t)b * 64;
  for (int i = n - 1; i >= 0; --i) {
    double2 t = s.g[(size_t)b * 64 + i];
    for (int k = i + 1; k < n; ++k) {
      double2 p = cmul(H[i * 64 + k], y[k]);
      t.x -= p.x;
      t.y -= p.y;
    }
    double2 d = H[i * 64 + i];
    double dd = d.x * d.x + d.y * d.y;
    y[i] = dd > 0 ? make_double2((t.x * d.x + t.y * d.y) / dd, (t.y * d.x - t.x * d.y) / dd) : make_double2(0, 0);
  }
}

// x += dinv .* (V y)
__global__ void k_xupdate(const double2* __restrict__ V, size_t vstride, int ns, const double2* __restrict__ dinv,
                          GmresState s, double2* __restrict__ x) {
  const int b = blockIdx.y;
  const int n_cols = s.jc[b];
  if (n_cols == 0) return;
  for (int n = blockIdx.x * kThreads + threadIdx.x; n < ns; n += gridDim.x * kThreads) {
    double2 u = make_double2(0, 0);
    for (int i = 0; i < n_cols; ++i) {
      double2 p = cmul(V[i * vstride + (size_t)b * ns + n], s.y[(size_t)b * 64 + i]);
      u.x += p.x;
      u.y += p.y;
    }
    double2 d = dinv[n];
    double2 du = cmul(d, u);
    double2 xv = x[(size_t)b * ns + n];
    x[(size_t)b * ns + n] = make_double2(xv.x + du.x, xv.y + du.y);
  }
}

__global__ void k_any(int nb, const int* __restrict__ act, int* __restrict__ flag) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int a = 0;
    for (int b = 0; b < nb; ++b) a |= act[b];
    *flag = a;
  }
}

}  // namespace

int gmres_blocks(int ns) { return std::max(1, std::min(64, (ns + kThreads * 4 - 1) / (kThreads * 4))); }

void gmres_alloc(aim_ctx* c) {
  const int B = c->batch_max;
  GmresState& s = c->gs;
  const size_t nblk = gmres_blocks(c->ns);
  s.H = (double2*)aim_alloc(c, (size_t)B * 64 * 64 * sizeof(double2));
  s.g = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  s.sn = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  s.cs = (double*)aim_alloc(c, (size_t)B * 64 * sizeof(double));
  s.y = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  s.h1 = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  s.h2 = (double2*)aim_alloc(c, (size_t)B * 64 * sizeof(double2));
  s.hn = (double*)aim_alloc(c, B * sizeof(double));
  s.bn = (double*)aim_alloc(c, B * sizeof(double));
  s.rn = (double*)aim_alloc(c, B * sizeof(double));
  s.scale = (double*)aim_alloc(c, B * sizeof(double));
  s.relres = (double*)aim_alloc(c, B * sizeof(double));
  s.act = (int*)aim_alloc(c, B * sizeof(int));
  s.done = (int*)aim_alloc(c, B * sizeof(int));
  s.jc = (int*)aim_alloc(c, B * sizeof(int));
  s.its = (int*)aim_alloc(c, B * sizeof(int));
  s.flag = (int*)aim_alloc(c, sizeof(int));
  s.pc = (double2*)aim_alloc(c, (size_t)B * nblk * 64 * sizeof(double2));
  s.pr = (double*)aim_alloc(c, (size_t)B * nblk * sizeof(double));
  s.counter = (unsigned*)aim_alloc(c, B * sizeof(unsigned));
  AIM_CUDA(cudaMemsetAsync(s.counter, 0, B * sizeof(unsigned), c->stream));
  AIM_CUDA(cudaMallocHost(&s.h_flag, sizeof(int)));
  AIM_CUDA(cudaMallocHost(&s.h_its, B * sizeof(int)));
  AIM_CUDA(cudaMallocHost(&s.h_res, B * sizeof(double)));
  AIM_CUDA(cudaMallocHost(&s.h_done, B * sizeof(int)));
}

void gmres_free_host(aim_ctx* c) {
  GmresState& s = c->gs;
  if (s.h_flag) cudaFreeHost(s.h_flag);
  if (s.h_its) cudaFreeHost(s.h_its);
  if (s.h_res) cudaFreeHost(s.h_res);
  if (s.h_done) cudaFreeHost(s.h_done);
  s.h_flag = nullptr;
  s.h_its = nullptr;
  s.h_res = nullptr;
  s.h_done = nullptr;
}

// Solve Z_0 x = b for nb right-hand sides; x holds the initial guess on entry.
// Returns AIM_OK or AIM_ERR_NOCONV; per-RHS iteration counts and final relative
// residuals land in iters / relres (host arrays, may be null).
int gmres_solve(aim_ctx* c, int nb, const double2* b, double2* x, double tol, int* iters, double* relres) {
  GmresState& s = c->gs;
  cudaStream_t st = c->stream;
  const int ns = c->ns, R = c->restart;
  const int nblk = gmres_blocks(ns);
  const size_t vstride = (size_t)c->batch_max * ns;
  dim3 vg(nblk, nb);
  const int sb = (nb + 63) / 64;
  AIM_CUDA(cudaMemsetAsync(s.its, 0, nb * sizeof(int), st));
  AIM_KLAUNCH(c, AIM_K_GMRES_UPDATE, k_norms<<<vg, kThreads, 0, st>>>(b, ns, s.pr, s.counter, s.bn));
  for (int cycle = 0;; ++cycle) {
    // explicit residual r = b - Z_0 x (FP64 vectors; operator in the context precision)
    op_apply(c, 0, nb, x, nullptr, b, -1.0, nullptr, c->d_r);
    AIM_KLAUNCH(c, AIM_K_GMRES_UPDATE, k_norms<<<vg, kThreads, 0, st>>>(c->d_r, ns, s.pr, s.counter, s.rn));
    AIM_KLAUNCH(c, AIM_K_GMRES_SMALL, k_cycle_start<<<sb, 64, 0, st>>>(nb, R, tol, c->max_iter, s.rn, s.bn, s));
    AIM_KLAUNCH(c, AIM_K_GMRES_SMALL, k_scale<<<vg, kThreads, 0, st>>>(c->d_r, c->d_V, ns, s.act, s.scale));
    AIM_KLAUNCH(c, AIM_K_GMRES_SMALL, k_any<<<1, 32, 0, st>>>(nb, s.act, s.flag));
    AIM_CUDA(cudaMemcpyAsync(s.h_flag, s.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    AIM_CUDA(cudaStreamSynchronize(st));
    if (!*s.h_flag) break;
    for (int j = 0; j < R; ++j) {
      double2* vj = c->d_V + (size_t)j * vstride;
      double2* vn = c->d_V + (size_t)(j + 1) * vstride;
      // w = Z_0 (dinv .* v_j), then CGS2 against v_0..v_j
      op_apply(c, 0, nb, vj, c->d_dinv, nullptr, 1.0, s.act, c->d_w);
      AIM_KLAUNCH(c, AIM_K_GMRES_DOT,
                  k_dots<<<vg, kThreads, 0, st>>>(c->d_V, vstride, j + 1, c->d_w, ns, nb, s.act, s.pc, s.counter, s.h1));
      AIM_KLAUNCH(c, AIM_K_GMRES_UPDATE,
                  k_update<<<vg, kThreads, 0, st>>>(c->d_V, vstride, j + 1, s.h1, c->d_w, ns, s.act, false, s.pr,
                                                    s.counter, s.hn));
      AIM_KLAUNCH(c, AIM_K_GMRES_DOT,
                  k_dots<<<vg, kThreads, 0, st>>>(c->d_V, vstride, j + 1, c->d_w, ns, nb, s.act, s.pc, s.counter, s.h2));
      AIM_KLAUNCH(c, AIM_K_GMRES_UPDATE,
                  k_update<<<vg, kThreads, 0, st>>>(c->d_V, vstride, j + 1, s.h2, c->d_w, ns, s.act, true, s.pr,
                                                    s.counter, s.hn));
      AIM_KLAUNCH(c, AIM_K_GMRES_SMALL,
                  k_arnoldi_finish<<<sb, 64, 0, st>>>(nb, j, R, tol, c->max_iter, s.h1, s.h2, s.hn, s.bn, s));
      AIM_KLAUNCH(c, AIM_K_GMRES_SMALL, k_scale<<<vg, kThreads, 0, st>>>(c->d_w, vn, ns, s.act, s.scale));
      AIM_KLAUNCH(c, AIM_K_GMRES_SMALL, k_any<<<1, 32, 0, st>>>(nb, s.act, s.flag));
      AIM_CUDA(cudaMemcpyAsync(s.h_flag, s.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
      AIM_CUDA(cudaStreamSynchronize(st));
      if (!*s.h_flag) break;
    }
    AIM_KLAUNCH(c, AIM_K_GMRES_SMALL, k_cycle_solve<<<sb, 64, 0, st>>>(nb, s));
    AIM_KLAUNCH(c, AIM_K_GMRES_SMALL, k_xupdate<<<vg, kThreads, 0, st>>>(c->d_V, vstride, ns, c->d_dinv, s, x));
    if (cycle > 4 * (c->max_iter / std::max(1, R) + 2)) break;
  }
  AIM_CUDA(cudaMemcpyAsync(s.h_its, s.its, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
  AIM_CUDA(cudaMemcpyAsync(s.h_res, s.relres, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  AIM_CUDA(cudaMemcpyAsync(s.h_done, s.done, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
  AIM_CUDA(cudaStreamSynchronize(st));
  int rc = AIM_OK;
  for (int i = 0; i < nb; ++i) {
    if (iters) iters[i] = s.h_its[i];
    if (relres) relres[i] = s.h_res[i];
    if (s.h_done[i] != 1) rc = AIM_ERR_NOCONV;
  }
  return rc;
}

void gmres_norms(aim_ctx* c, int nb, const double2* v, double* d_out) {
  dim3 vg(gmres_blocks(c->ns), nb);
  AIM_KLAUNCH(c, AIM_K_GMRES_UPDATE, k_norms<<<vg, kThreads, 0, c->stream>>>(v, c->ns, c->gs.pr, c->gs.counter, d_out));
}
