// The ET-AIM operator on the device (Eq. 5, Sec. 4 stages i-iv), templated on the
// complex type of the grid stages (float2: complex64 path, double2: plain path).
//
// Data layout per right-hand side b and component c (x, y, z, div), with L = 2N and the
// nz z-planes z0 .. z0 + nz - 1 of the active box (the nodes some stencil touches):
//   A  [b][c][nz][y<N][x<L]   after anterpolation + forward x-FFT
//   Bf [b][c][nz][y<L][x<L]   after the forward y-FFT (the slab)
//   P  [b][c][nz][y<N][x<N]   potentials after the inverse passes
// The forward z-FFT (length LZ >= 2 nz), the pointwise kernel product and the inverse
// z-FFT are one kernel per column (k_zconv / k_zrhs), so no 3-D spectrum reaches
// memory.  Zero padding is pruned in every pass: forward passes read only the non-zero
// inputs, inverse passes write only the needed outputs.
#pragma once
#include <algorithm>
#include <functional>
#include <type_traits>
#include <vector>

#include "aim_internal.h"
#include "fft_kernels.cuh"
#include "operator.h"
#include "tma.cuh"

template <class C> struct Real;
template <> struct Real<float2> { using T = float; using F4 = float4; };
template <> struct Real<double2> { using T = double; using F4 = double4_32a; };

template <class C> __device__ __forceinline__ C cvt(double2 a);
template <> __device__ __forceinline__ float2 cvt<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __device__ __forceinline__ double2 cvt<double2>(double2 a) { return a; }

// ---------------------------------------------------------------- stage i + x pass
// S_c[n] = sum_k L_c[n,k] x_k gathered node by node (the transpose of the
// interpolation rows), then the forward x-FFT of each grid row.  One block holds
// the 4 components of ypb consecutive rows (z, y); grid (nb, rows / ypb, nz) with the
// right-hand side fastest, so the CSR rows a block gathers serve the other right-hand
// sides from L2.
template <int L, class C>
__global__ void __launch_bounds__(256) k_anterp_rows(const int* __restrict__ nptr, const int* __restrict__ nidx,
                                                     const typename Real<C>::F4* __restrict__ ncoef,
                                                     const C* __restrict__ xs, const int* __restrict__ active,
                                                     int ns, int N, int ypb, C* __restrict__ A,
                                                     const C* __restrict__ twg, int ylo, int yhi, int zlo, int nz) {
  pdl_wait();
  using R = typename Real<C>::T;
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  C* tw = reinterpret_cast<C*>(aim_smem);
  C* b0 = tw + L;
  C* b1 = b0 + 4 * ypb * L;
  load_twiddles(tw, twg, L);
  const int z = zlo + blockIdx.z, y0 = ylo + blockIdx.y * ypb;  // rows of the active box
  const C* vb = xs + (size_t)b * ns;
  // gather the N nodes of each row (all threads busy), zero the padding half
  for (int t = threadIdx.x; t < ypb * N; t += blockDim.x) {
    const int yy = t / N, x = t % N, y = y0 + yy;
    C a0{}, a1{}, a2{}, a3{};
    if (y <= yhi) {
      const size_t n = ((size_t)z * N + y) * N + x;
      int e = nptr[n];
      const int e1 = nptr[n + 1];
      // eight entries at a time: their index and coefficient loads, then their gathers of
      // x, are independent and in flight together (the sums keep the entry order)
      for (; e + 8 <= e1; e += 8) {
        int k[8];
        typename Real<C>::F4 w[8];
        C xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          k[u] = nidx[e + u];
          w[u] = ncoef[e + u];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) xv[u] = vb[k[u]];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          a0 += (R)w[u].x * xv[u];
          a1 += (R)w[u].y * xv[u];
          a2 += (R)w[u].z * xv[u];
          a3 += (R)w[u].w * xv[u];
        }
      }
      if (e + 4 <= e1) {  // then four
        int k[4];
        typename Real<C>::F4 w[4];
        C xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          k[u] = nidx[e + u];
          w[u] = ncoef[e + u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = vb[k[u]];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a0 += (R)w[u].x * xv[u];
          a1 += (R)w[u].y * xv[u];
          a2 += (R)w[u].z * xv[u];
          a3 += (R)w[u].w * xv[u];
        }
        e += 4;
      }
      for (; e < e1; ++e) {
        const int k = nidx[e];
        const typename Real<C>::F4 w = ncoef[e];
        const C xv = vb[k];
        a0 += (R)w.x * xv;
        a1 += (R)w.y * xv;
        a2 += (R)w.z * xv;
        a3 += (R)w.w * xv;
      }
    }
    b0[(0 * ypb + yy) * L + x] = a0;
    b0[(1 * ypb + yy) * L + x] = a1;
    b0[(2 * ypb + yy) * L + x] = a2;
    b0[(3 * ypb + yy) * L + x] = a3;
  }
  C* res;
  if constexpr (two_step_len(L)) {  // the padding half is never read
    __syncthreads();
    row_fft2<L, false, C, true>(b0, b1, 4 * ypb, tw);
    res = b0;
  } else {
    for (int t = threadIdx.x; t < 4 * ypb * (L - N); t += blockDim.x) {
      const int row = t / (L - N), x = N + t % (L - N);
      b0[row * L + x] = C{};
    }
    __syncthreads();
    res = line_fft_rows<L, false, C>(b0, b1, 4 * ypb, tw);
  }
  for (int t = threadIdx.x; t < 4 * ypb * L; t += blockDim.x) {
    const int row = t / L, x = t % L, c = row / ypb, y = y0 + row % ypb;
    if (y <= yhi) A[((((size_t)b * 4 + c) * nz + blockIdx.z) * N + y) * L + x] = res[t];
  }
  pdl_trigger();
}

// Operator input: x_b = scale_b(j) * dinv .* v_b (selection, Krylov scale and
// preconditioner applied once), in the grid precision for the anterpolation gather
// and in FP64 for the near-zone product.
template <class C>
__global__ void __launch_bounds__(256) k_prep(const double2* __restrict__ v, const double2* __restrict__ dinv,
                                              VecSel vs, const int* __restrict__ active, int ns, int nb,
                                              C* __restrict__ xs, double2* __restrict__ xd) {
  pdl_wait();
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)nb * ns) return;
  const int b = (int)(idx / ns), k = (int)(idx % ns);
  if (active && !active[b]) return;
  double sc = 1.0;
  if (vs.sel) {
    const int j = *vs.sel + vs.off;
    v += j * vs.stride;
    if (vs.scale) sc = vs.scale[b * 64 + j];
  }
  double2 x = v[idx];
  x = make_double2(sc * x.x, sc * x.y);
  if (dinv) {
    const double2 d = dinv[k];
    x = make_double2(x.x * d.x - x.y * d.y, x.x * d.y + x.y * d.x);
  }
  xs[idx] = cvt<C>(x);
  if (xd) xd[idx] = x;
  pdl_trigger();
}

// The same with the SAI as the preconditioner: x_b[k] = scale_b(j) *
// sum_e M[k, col_e] v_b[col_e] over row k of its CSR pattern (at most 144 entries).  16
// lanes per row (two rows per warp), fixed-order butterfly sum over the 16 lanes.  M is
// applied in the grid precision: complex64 (M rounded to FP32, products and sums in FP32,
// like the grid stages it feeds) or complex128 (FP64).
template <class C>
__global__ void __launch_bounds__(256) k_prep_sai(const double2* __restrict__ v, const float2* __restrict__ vf,
                                                  const C* __restrict__ sai, const int* __restrict__ rowptr,
                                                  const int* __restrict__ col, VecSel vs,
                                                  const int* __restrict__ active, int ns, int nb,
                                                  C* __restrict__ xs, double2* __restrict__ xd) {
  pdl_wait();
  using R = typename Real<C>::T;
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 4;
  const int lane = threadIdx.x & 15;
  const bool valid = w < (long long)nb * ns;  // both rows of a warp join the shuffles
  const int b = valid ? (int)(w / ns) : 0, k = valid ? (int)(w % ns) : 0;
  const bool on = valid && !(active && !active[b]);
  double sc = 1.0;
  if (vs.sel) {
    const int j = *vs.sel + vs.off;
    v += j * vs.stride;
    if (vs.scale) sc = vs.scale[b * 64 + j];
  }
  const double2* vb = v + (size_t)b * ns;
  R xr = 0, xi = 0;
  if (on) {
    // up to 9 entries per lane: indices and values first, then the gathered vector
    // entries, then the products in entry order
    const int e0 = rowptr[k] + lane, e1 = rowptr[k + 1];
    int j[9];
    C m[9];
    double2 u[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const int e = e0 + 16 * q;
      j[q] = e < e1 ? col[e] : -1;
      m[q] = e < e1 ? sai[e] : C{};
    }
    if (vf) {  // complex64 copy of v_j: no FP64 -> FP32 conversion per gathered entry
      const float2* vfb = vf + (size_t)b * ns;
      float2 uf[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) uf[q] = j[q] >= 0 ? vfb[j[q]] : make_float2(0, 0);
#pragma unroll
      for (int q = 0; q < 9; ++q)
        if (j[q] >= 0) {
          const R ur = (R)uf[q].x, ui = (R)uf[q].y;
          xr += m[q].x * ur - m[q].y * ui;
          xi += m[q].x * ui + m[q].y * ur;
        }
    } else {
#pragma unroll
      for (int q = 0; q < 9; ++q) u[q] = j[q] >= 0 ? vb[j[q]] : make_double2(0, 0);
#pragma unroll
      for (int q = 0; q < 9; ++q)
        if (j[q] >= 0) {
          const R ur = (R)u[q].x, ui = (R)u[q].y;
          xr += m[q].x * ur - m[q].y * ui;
          xi += m[q].x * ui + m[q].y * ur;
        }
    }
  }
  for (int o = 8; o > 0; o >>= 1) {
    xr += __shfl_xor_sync(0xffffffffu, xr, o);
    xi += __shfl_xor_sync(0xffffffffu, xi, o);
  }
  if (on && lane == 0) {
    const double2 x = make_double2(sc * (double)xr, sc * (double)xi);
    const size_t idx = (size_t)b * ns + k;
    xs[idx] = cvt<C>(x);
    if (xd) xd[idx] = x;
  }
  pdl_trigger();
}

// ---------------------------------------------------------------- z pass with the kernel
__device__ __forceinline__ int fold(int k, int N) { return k <= N ? k : 2 * N - k; }

// Geometry of a z pass.  The slab holds the nz z-planes of the active box (plane p is grid
// z = box_lo + p), each an L x L plane of x/y spectra.  The z transform length LZ (a
// template parameter) is at least 2 nz: the linear convolution of nz planes with the
// kernel needs offsets |dz| < nz only, so a circular convolution of any length >= 2 nz - 1
// gives the same values on the nz output planes as the 2N-point padding.  The kernel
// spectrum octant is [LZ/2 + 1][N + 1][N + 1] (z, y, x).
struct ZGeom {
  int L;   // x/y padded length 2N
  int N;   // L / 2 (x/y fold of the kernel octant)
  int nz;  // z planes of the slab: input samples 0 .. nz-1, outputs kept 0 .. nz-1
};

// Two-step LZ = R1 * R2, one tile of W adjacent z-columns per block, a single
// shared exchange tile t[(k1 R2 + n2) W + l]:
//   A  thread (l, n2): the nz <= LZ/2 nonzero samples p = R2 n1 + n2 (n1 < R1/2) come
//      straight from memory, radix-R1 butterfly, twiddle W_LZ^{n2 k1}, into t;
//   B  thread (l, k1): its R2 values of t, radix-R2 butterfly -> X[k1 + R1 k2] in
//      registers; product with the kernel spectrum; inverse radix-R2 butterfly,
//      twiddle W_LZ^{-k1 n2}, back into the same slots of t (a thread reads and writes
//      only its own (k1, l) slice, so B needs no barrier inside);
//   C  thread (l, n2): inverse radix-R1 butterfly over k1, the outputs
//      p = n2 + R2 n1 < nz stored straight to memory.
// A column's data cross shared memory twice instead of once per pass.
// radix split of the z pass: for LZ = 128 the 16 x 8 split keeps the step-B registers
// (operands and spectrum slice) at 8 complex values each
template <int LZ>
constexpr int zsplit_r1() {
  return LZ == 128 ? 16 : split_r1(LZ);
}
template <int LZ, class C>
constexpr int zcol_width() {
  return (int)sizeof(C) == 8 ? (LZ < 32 ? LZ : LZ >= 512 ? 16 : 32) : (LZ < 16 ? LZ : LZ >= 512 ? 8 : 16);
}
constexpr int kZThreads = 256;

template <int LZ, int W, class C>
__device__ __forceinline__ void zcol_step_a(const C* __restrict__ col, long long es, C* t, const C* tw, int nz) {
  constexpr int R1 = zsplit_r1<LZ>(), R2 = LZ / R1;
  for (int u = threadIdx.x; u < W * R2; u += kZThreads) {
    const int l = u % W, n2 = u / W;
    C v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const int p = R2 * n1 + n2;
      v[n1] = n1 < R1 / 2 && p < nz ? col[(long long)p * es + l] : C{};
    }
    dft_half_in<R1, LZ, false, C>(v, tw);  // samples p >= LZ/2 are the zero padding
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      C x = v[k1];
      if (k1 && n2) x = x * tw[n2 * k1];
      t[(k1 * R2 + n2) * W + l] = x;
    }
  }
}

// the spectrum X[k1 + R1 k2] of column l from t (after step A and a barrier)
template <int LZ, int W, class C>
__device__ __forceinline__ void zcol_step_b_fwd(const C* t, const C* tw, int k1, int l,
                                                C (&v)[LZ / zsplit_r1<LZ>()]) {
  constexpr int R1 = zsplit_r1<LZ>(), R2 = LZ / R1;
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) v[n2] = t[(k1 * R2 + n2) * W + l];
  DFTL<R2, LZ, false, C>::run(v, tw);
  (void)R1;
}

// inverse radix-R2 butterfly of a spectrum slice, twiddled back into t
template <int LZ, int W, class C>
__device__ __forceinline__ void zcol_step_b_inv(C* t, const C* tw, int k1, int l, C (&v)[LZ / zsplit_r1<LZ>()]) {
  constexpr int R1 = zsplit_r1<LZ>(), R2 = LZ / R1;
  DFTL<R2, LZ, true, C>::run(v, tw);
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    C x = v[n2];
    if (k1 && n2) x = x * conjc(tw[n2 * k1]);
    t[(k1 * R2 + n2) * W + l] = x;
  }
  (void)R1;
}

template <int LZ, int W, class C>
__device__ __forceinline__ void zcol_step_c(const C* t, const C* tw, C* __restrict__ col, long long es, int nz) {
  constexpr int R1 = zsplit_r1<LZ>(), R2 = LZ / R1;
  for (int u = threadIdx.x; u < W * R2; u += kZThreads) {
    const int l = u % W, n2 = u / W;
    C v[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) v[k1] = t[(k1 * R2 + n2) * W + l];
    dft_half_out<R1, LZ, true, C>(v, tw);  // only the outputs p < LZ/2 are formed
#pragma unroll
    for (int n1 = 0; n1 < R1 / 2; ++n1) {
      const int p = n2 + R2 * n1;
      if (p < nz) col[(long long)p * es + l] = v[n1];
    }
  }
}

// Grid order of the z-pass blocks: (right-hand side, component) fastest, then the x
// tile, then the row y taken in mirror pairs (0, N, 1, L-1, 2, L-2, ...).  Every block
// reads the kernel-spectrum octant at (fold(kz), fold(y), fold(x)); the octant of a large
// grid does not fit in L2, and this order keeps the blocks that read the same entries
// (all right-hand sides and components of one kernel kind, the rows y and L-y) close in
// time, so the octant comes from DRAM about once per launch.
__device__ __forceinline__ int zpass_row(int j, int N) {
  if (j < 2) return j * N;
  const int k = ((j - 2) >> 1) + 1;
  return (j & 1) ? 2 * N - k : k;
}

// the kernel-spectrum column of kind `kind` at (x, y): entry kz at [fold(kz, LZ/2) * n1^2]
template <int LZ, class C>
__device__ __forceinline__ const C* kcol(const C* kspec, const ZGeom& g, int kind, int x, int y) {
  const size_t n1 = (size_t)g.N + 1;
  return kspec + (size_t)kind * n1 * n1 * (LZ / 2 + 1) + (size_t)fold(y, g.N) * n1 + fold(x, g.N);
}

// Forward z-FFT of the slab column, product with the kernel spectrum of delay m
// (G^A for c = x,y,z; G^phi for c = div; even-symmetric octant), inverse z-FFT,
// the nz outputs written back in place.  Grid (nb * 4, L / W, L) in the order above.
template <int LZ, int W, class C>
__global__ void __launch_bounds__(kZThreads) k_zconv_p2(C* __restrict__ Bf, const C* __restrict__ kspec, ZGeom g,
                                                        const int* __restrict__ active,
                                                        const C* __restrict__ twg) {
  pdl_wait();
  constexpr int R1 = zsplit_r1<LZ>(), R2 = LZ / R1;
  const int bc = blockIdx.x;
  if (active && !active[bc >> 2]) return;
  C* tw = reinterpret_cast<C*>(aim_smem);
  C* t = tw + LZ;
  load_twiddles(tw, twg, LZ);
  __syncthreads();
  const int y = zpass_row(blockIdx.z, g.N), x0 = blockIdx.y * W;
  const long long es = (long long)g.L * g.L;
  C* col = Bf + (size_t)bc * g.nz * es + (size_t)y * g.L + x0;
  const size_t nn = (size_t)(g.N + 1) * (g.N + 1);
  zcol_step_a<LZ, W, C>(col, es, t, tw, g.nz);
  __syncthreads();
  for (int u = threadIdx.x; u < W * R1; u += kZThreads) {
    const int l = u % W, k1 = u / W;
    const C* G = kcol<LZ>(kspec, g, (bc & 3) == 3 ? 1 : 0, x0 + l, y);
    C gk[R2], v[R2];
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) gk[k2] = __ldg(G + (size_t)fold(k1 + R1 * k2, LZ / 2) * nn);
    zcol_step_b_fwd<LZ, W, C>(t, tw, k1, l, v);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k2] = v[k2] * gk[k2];
    zcol_step_b_inv<LZ, W, C>(t, tw, k1, l, v);
  }
  __syncthreads();
  zcol_step_c<LZ, W, C>(t, tw, col, es, g.nz);
  pdl_trigger();
}

// History slabs of power-of-two z length are kept z-transformed: S[bc][kz][y][x], all LZ
// frequencies kz of every (x, y) line (LZ / nz times the bytes of the x/y-transformed
// slab).  The delay sum of the right-hand side is then a multiply-accumulate streamed
// over the N_g spectra and one inverse z-FFT, instead of N_g forward z-FFTs recomputed
// at every step.
//
// k_zfwd_spec: the forward z-FFT (steps A and B of the z pass) of the slab in Bf into the
// spectral layout; thread (l, k1) of step B stores X[k1 + R1 k2] for all k2.
template <int LZ, int W, class C>
__global__ void __launch_bounds__(kZThreads) k_zfwd_spec(const C* __restrict__ Bf, C* __restrict__ S, ZGeom g,
                                                         const C* __restrict__ twg) {
  constexpr int R1 = zsplit_r1<LZ>(), R2 = LZ / R1;
  C* tw = reinterpret_cast<C*>(aim_smem);
  C* t = tw + LZ;
  load_twiddles(tw, twg, LZ);
  __syncthreads();
  const int bc = blockIdx.z, y = blockIdx.y, x0 = blockIdx.x * W;
  const long long es = (long long)g.L * g.L;
  zcol_step_a<LZ, W, C>(Bf + (size_t)bc * g.nz * es + (size_t)y * g.L + x0, es, t, tw, g.nz);
  __syncthreads();
  C* out = S + (size_t)bc * LZ * es + (size_t)y * g.L + x0;
  for (int u = threadIdx.x; u < W * R1; u += kZThreads) {
    const int l = u % W, k1 = u / W;
    C v[R2];
    zcol_step_b_fwd<LZ, W, C>(t, tw, k1, l, v);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) out[(long long)(k1 + R1 * k2) * es + l] = v[k2];
  }
}

// Delay sum of the right-hand side in the spectral domain:
//   P^_col = sum_i G^_{m_i} . S_i(col), then one inverse z-FFT (steps B inverse and C),
// the sum kept in the registers of the step-B threads (thread (l, k1) owns the
// frequencies k1 + R1 k2).
template <int LZ, int W, class C>
__global__ void __launch_bounds__(kZThreads, 3) k_zrhs_spec(SlabList sl, const C* __restrict__ kspec_all, ZGeom g,
                                                         C* __restrict__ Bf, const C* __restrict__ twg) {
  constexpr int R1 = zsplit_r1<LZ>(), R2 = LZ / R1, U = (W * R1 + kZThreads - 1) / kZThreads;
  C* tw = reinterpret_cast<C*>(aim_smem);
  C* t = tw + LZ;
  load_twiddles(tw, twg, LZ);
  __syncthreads();
  const int bc = blockIdx.z, y = blockIdx.y, x0 = blockIdx.x * W;
  const long long es = (long long)g.L * g.L;
  const size_t nn = (size_t)(g.N + 1) * (g.N + 1), oct = nn * (LZ / 2 + 1);
  const int kind = (bc & 3) == 3 ? 1 : 0;
  C acc[U][R2];
#pragma unroll
  for (int j = 0; j < U; ++j)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) acc[j][k2] = C{};
  for (int s = 0; s < sl.n; ++s) {
    const C* Sc = reinterpret_cast<const C*>(sl.p[s]) + (size_t)bc * LZ * es + (size_t)y * g.L + x0;
    const C* Gm = kspec_all + (size_t)sl.m[s] * 2 * oct;
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int u = threadIdx.x + j * kZThreads;
      if (u < W * R1) {
        const int l = u % W, k1 = u / W;
        const C* G = kcol<LZ>(Gm, g, kind, x0 + l, y);
        C gk[R2], v[R2];
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const int kz = k1 + R1 * k2;
          v[k2] = Sc[(long long)kz * es + l];
          gk[k2] = __ldg(G + (size_t)fold(kz, LZ / 2) * nn);
        }
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) acc[j][k2] += v[k2] * gk[k2];
      }
    }
  }
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const int u = threadIdx.x + j * kZThreads;
    if (u < W * R1) zcol_step_b_inv<LZ, W, C>(t, tw, u / W, u % W, acc[j]);
  }
  __syncthreads();
  zcol_step_c<LZ, W, C>(t, tw, Bf + (size_t)bc * g.nz * es + (size_t)y * g.L + x0, es, g.nz);
}

// The same with the spectra streamed by TMA (complex64): the LZ x W tile of each spectrum
// is a 4-D box of the ring tensor [slot][B*4*LZ][L][L], loaded into one of two 128-byte
// aligned shared buffers by cp.async.bulk.tensor and signalled on an mbarrier, so
// spectrum s + 2 streams in while spectrum s + 1 is accumulated.  Waits are bounded.  A
// wait that gives up sets *err (the host reports AIM_ERR_TIMEOUT) and a block-wide flag;
// the block then issues no further load, drains the loads it has in flight with one more
// bounded wait each and returns without writing its output (which is undefined whenever
// *err is set).
template <int LZ, int W>
__global__ void __launch_bounds__(kZThreads, 3) k_zrhs_spec_tma(const __grid_constant__ CUtensorMap ring,
                                                                SlabRing sr, const float2* __restrict__ kspec_all,
                                                                ZGeom g, float2* __restrict__ Bf,
                                                                const float2* __restrict__ twg, int* __restrict__ err) {
  using C = float2;
  constexpr int R1 = zsplit_r1<LZ>(), R2 = LZ / R1, U = (W * R1 + kZThreads - 1) / kZThreads;
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int gave_up[2];  // by iteration parity: a write in iteration s + 1 cannot reach a
                              // thread still reading the flag of iteration s
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(aim_smem) + 127) & ~static_cast<uintptr_t>(127));
  C* in0 = reinterpret_cast<C*>(base);  // [2][LZ][W]
  C* tw = in0 + 2 * LZ * W;
  C* t = tw + LZ;
  const int bc = blockIdx.z, y = blockIdx.y, x0 = blockIdx.x * W;
  const unsigned bytes = (unsigned)(LZ * W * sizeof(C));
  if (threadIdx.x == 0) {
    gave_up[0] = gave_up[1] = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  load_twiddles(tw, twg, LZ);
  __syncthreads();
  if (threadIdx.x == 0)
    for (int s = 0; s < 2 && s < sr.n; ++s) {
      mbar_arrive_expect_tx(&bar[s], bytes);
      tma_load_4d(in0 + s * LZ * W, &ring, &bar[s], x0, y, bc * LZ, sr.slot[s]);
    }
  const long long es = (long long)g.L * g.L;
  const size_t nn = (size_t)(g.N + 1) * (g.N + 1), oct = nn * (LZ / 2 + 1);
  const int kind = (bc & 3) == 3 ? 1 : 0;
  C acc[U][R2];
#pragma unroll
  for (int j = 0; j < U; ++j)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) acc[j][k2] = C{};
  for (int s = 0; s < sr.n; ++s) {
    const int buf = s & 1;
    const C* Gm = kspec_all + (size_t)sr.m[s] * 2 * oct;
    C gk[U][R2];
#pragma unroll
    for (int j = 0; j < U; ++j) {  // the kernel spectrum while the tile streams in
      const int u = threadIdx.x + j * kZThreads;
      if (u < W * R1) {
        const C* G = kcol<LZ>(Gm, g, kind, x0 + u % W, y);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) gk[j][k2] = __ldg(G + (size_t)fold(u / W + R1 * k2, LZ / 2) * nn);
      }
    }
    const bool ok = mbar_wait_bounded(&bar[buf], (unsigned)((s >> 1) & 1));
    if (!ok) {
      atomicExch(err, 1);
      gave_up[s & 1] = 1;
    }
    const C* tile = in0 + buf * LZ * W;  // [kz][l]
    if (ok) {
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int u = threadIdx.x + j * kZThreads;
        if (u < W * R1) {
          const int l = u % W, k1 = u / W;
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) acc[j][k2] += tile[(k1 + R1 * k2) * W + l] * gk[j][k2];
        }
      }
    }
    __syncthreads();  // the tile is consumed: it may be refilled (gave_up[s & 1] is block-uniform)
    if (gave_up[s & 1]) {
      // loads in flight: spectrum s (the wait that gave up, for some thread) and s + 1
      if (threadIdx.x == 0) {
        mbar_wait_bounded(&bar[buf], (unsigned)((s >> 1) & 1));
        if (s + 1 < sr.n) mbar_wait_bounded(&bar[buf ^ 1], (unsigned)(((s + 1) >> 1) & 1));
      }
      __syncthreads();
      return;
    }
    if (threadIdx.x == 0 && s + 2 < sr.n) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bar[buf], bytes);
      tma_load_4d(in0 + buf * LZ * W, &ring, &bar[buf], x0, y, bc * LZ, sr.slot[s + 2]);
    }
  }
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const int u = threadIdx.x + j * kZThreads;
    if (u < W * R1) zcol_step_b_inv<LZ, W, C>(t, tw, u / W, u % W, acc[j]);
  }
  __syncthreads();
  zcol_step_c<LZ, W, C>(t, tw, Bf + (size_t)bc * g.nz * es + (size_t)y * g.L + x0, es, g.nz);
}

// Blocked right-hand side (Sec. 4 stage ii), power-of-two z lengths.  The pending
// accumulator of a step holds the z-spectra P^ of its delayed grid sum, built by the
// squares of earlier steps; k_zinv_pending turns it into the slab of potentials (inverse
// z-FFT, steps B^-1 and C) and clears it for reuse.
template <int LZ, int W, class C>
__global__ void __launch_bounds__(kZThreads) k_zinv_pending(C* __restrict__ S, ZGeom g, C* __restrict__ Bf,
                                                            const C* __restrict__ twg) {
  constexpr int R1 = zsplit_r1<LZ>(), R2 = LZ / R1;
  C* tw = reinterpret_cast<C*>(aim_smem);
  C* t = tw + LZ;
  load_twiddles(tw, twg, LZ);
  __syncthreads();
  const int bc = blockIdx.z, y = blockIdx.y, x0 = blockIdx.x * W;
  const long long es = (long long)g.L * g.L;
  C* Sc = S + (size_t)bc * LZ * es + (size_t)y * g.L + x0;
  for (int u = threadIdx.x; u < W * R1; u += kZThreads) {
    const int l = u % W, k1 = u / W;
    C v[R2];
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      C* e = Sc + (long long)(k1 + R1 * k2) * es + l;
      v[k2] = *e;
      *e = C{};
    }
    zcol_step_b_inv<LZ, W, C>(t, tw, k1, l, v);
  }
  __syncthreads();
  zcol_step_c<LZ, W, C>(t, tw, Bf + (size_t)bc * g.nz * es + (size_t)y * g.L + x0, es, g.nz);
}

// One square: every element q of the z-spectra ([bc][kz][y][x], nb * 4 * LZ * L * L of
// them) gathers its kernel taps G^_m, m = toff - B + 1 .. toff + B - 1 within 1 .. N_g,
// from the octant, its B sources, and adds the B Toeplitz products into the pending
// accumulators.  Each source and accumulator element is read (and written) once per
// square; at B <= 16 the direct product (8 B^2 flops per element) costs no more than
// temporal FFTs of length 2B would.
template <int B, class C>
__global__ void __launch_bounds__(256) k_block_square(BlockSquare sq, const C* __restrict__ kspec, ZGeom g, int LZ,
                                                      int ng, long long n) {
  const size_t nn = (size_t)(g.N + 1) * (g.N + 1), oct = nn * (LZ / 2 + 1);
  const long long plane = (long long)g.L * g.L, per_bc = plane * LZ;
  const int m0 = sq.toff - B + 1;  // tap[t] = G^_{m0 + t}
  for (long long q = blockIdx.x * 256LL + threadIdx.x; q < n; q += (long long)gridDim.x * 256) {
    const int x = (int)(q % g.L), y = (int)((q / g.L) % g.L), kz = (int)((q / plane) % LZ);
    const int bc = (int)(q / per_bc), kind = (bc & 3) == 3 ? 1 : 0;
    const size_t go = (size_t)kind * oct + ((size_t)fold(kz, LZ / 2) * (g.N + 1) + fold(y, g.N)) * (g.N + 1) +
                      fold(x, g.N);
    C tap[2 * B - 1];
#pragma unroll
    for (int t = 0; t < 2 * B - 1; ++t) {
      const int m = m0 + t;
      tap[t] = (m >= 1 && m <= ng) ? __ldg(kspec + (size_t)m * 2 * oct + go) : C{};
    }
    C s[B];
#pragma unroll
    for (int j = 0; j < B; ++j) s[j] = reinterpret_cast<const C*>(sq.src[j])[q];
#pragma unroll
    for (int i = 0; i < B; ++i) {
      C acc{};
#pragma unroll
      for (int j = 0; j < B; ++j) acc += tap[B - 1 + i - j] * s[j];
      C* d = reinterpret_cast<C*>(sq.dst[i]) + q;
      *d = *d + acc;
    }
  }
}

// z lengths with a factor 3 keep x/y-transformed history slabs: the delay sum recomputes
// each slab's forward z-transform (steps A and B of the z pass), multiplies it by its
// delay's kernel spectrum and accumulates in the registers of the step-B threads; then one
// inverse z-FFT (steps B^-1 and C), the nz outputs written to Bf.
template <int LZ, int W, class C>
__global__ void __launch_bounds__(kZThreads) k_zrhs_2s(SlabList sl, const C* __restrict__ kspec_all, ZGeom g,
                                                       C* __restrict__ Bf, const C* __restrict__ twg) {
  constexpr int R1 = zsplit_r1<LZ>(), R2 = LZ / R1, U = (W * R1 + kZThreads - 1) / kZThreads;
  C* tw = reinterpret_cast<C*>(aim_smem);
  C* t = tw + LZ;
  load_twiddles(tw, twg, LZ);
  __syncthreads();
  const int bc = blockIdx.x, y = zpass_row(blockIdx.z, g.N), x0 = blockIdx.y * W;  // z-pass grid order
  const long long es = (long long)g.L * g.L;
  const size_t nn = (size_t)(g.N + 1) * (g.N + 1), oct = nn * (LZ / 2 + 1);
  const int kind = (bc & 3) == 3 ? 1 : 0;
  C acc[U][R2];
#pragma unroll
  for (int j = 0; j < U; ++j)
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) acc[j][k2] = C{};
  for (int s = 0; s < sl.n; ++s) {
    const C* col = reinterpret_cast<const C*>(sl.p[s]) + (size_t)bc * g.nz * es + (size_t)y * g.L + x0;
    const C* Gm = kspec_all + (size_t)sl.m[s] * 2 * oct;
    if (s) __syncthreads();  // the previous delay's step B has read t
    zcol_step_a<LZ, W, C>(col, es, t, tw, g.nz);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int u = threadIdx.x + j * kZThreads;
      if (u < W * R1) {
        const int l = u % W, k1 = u / W;
        const C* G = kcol<LZ>(Gm, g, kind, x0 + l, y);
        C v[R2];
        zcol_step_b_fwd<LZ, W, C>(t, tw, k1, l, v);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) acc[j][k2] += v[k2] * __ldg(G + (size_t)fold(k1 + R1 * k2, LZ / 2) * nn);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const int u = threadIdx.x + j * kZThreads;
    if (u < W * R1) zcol_step_b_inv<LZ, W, C>(t, tw, u / W, u % W, acc[j]);
  }
  __syncthreads();
  zcol_step_c<LZ, W, C>(t, tw, Bf + (size_t)bc * g.nz * es + (size_t)y * g.L + x0, es, g.nz);
}

// ---------------------------------------------------------------- stage iii + iv
// y_k = sign * ( sum_c sum_{n in stencil(k)} L_c[n,k] P_c[n]  +  sum_terms Z~near_m x_m ) + base_k
// Grid (nb, ceil(ns / 32)): a block takes 32 rows of one RHS, one warp per kInterpRows
// consecutive rows.  Grid part: the whole warp per row, accumulated in the grid precision.
// Near part: 8 lanes per row, all rows at once, in FP64 -- the warp's FP64 instructions
// (each holds the sub-partition's FP64 pipe for the whole warp) serve kInterpRows rows
// instead of one.  With df.V set (the operator of an Arnoldi step, y = Krylov slot j+1)
// the block also forms the raw dots conj(vt_i) . y over its 32 rows for i <= j, and the
// last block of the RHS sums them into df.d.
constexpr int kInterpRows = 4;
constexpr int kInterpBlockRows = 8 * kInterpRows;  // 256 threads

template <class C>
__global__ void __launch_bounds__(256, 3) k_interp_near(const C* __restrict__ P, const int* __restrict__ anchor,
                                                     const int* __restrict__ order,
                                                     const typename Real<C>::T* __restrict__ lam, int N, int nz,
                                                     int zlo, int ns,
                                                     int nb, const int* __restrict__ rowptr,
                                                     const int* __restrict__ col, NearList nl,
                                                     const double2* __restrict__ base, double sign,
                                                     const int* __restrict__ active, double2* __restrict__ y,
                                                     VecSel ys, DotFuse df) {
  pdl_wait();
  using R = typename Real<C>::T;
  // the right-hand side is the fastest grid index: the blocks of all right-hand sides
  // for one set of rows run together and share that set's near-zone rows through L2
  const int b = blockIdx.x, rb = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (active && !active[b]) return;
  const int k0 = rb * kInterpBlockRows + warp * kInterpRows;  // the warp's first position
  // grid part, row by row; lane group r (lanes 8r .. 8r+7) keeps row r's sum
  C mine{};
  if (P) {
    const size_t N3 = (size_t)nz * N * N;  // the box planes z0 .. z0 + nz - 1
    // the warp's RWGs and their stencil origins first, so that the potential gathers of
    // all kInterpRows RWGs depend on no further load and can be in flight together
    int kr[kInterpRows];
    size_t org[kInterpRows];
#pragma unroll
    for (int r = 0; r < kInterpRows; ++r) kr[r] = k0 + r < ns ? order[k0 + r] : -1;
#pragma unroll
    for (int r = 0; r < kInterpRows; ++r) {
      const int k = kr[r] < 0 ? 0 : kr[r];
      org[r] = ((size_t)(anchor[3 * k + 2] - zlo) * N + anchor[3 * k + 1]) * N + anchor[3 * k];
    }
#pragma unroll
    for (int r = 0; r < kInterpRows; ++r) {
      C g{};
      if (kr[r] >= 0) {
        const int k = kr[r];
        // 4 lanes per stencil row: lane -> (row of 8, dx); the 256 (component, node)
        // terms of an RWG take 8 warp loads of 8 rows x 32 B each
        const C* Pb = P + (size_t)b * 4 * N3 + org[r] + (lane & 3);
        const R* lk = lam + (size_t)k * 256 + lane;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const int q = it * 8 + (lane >> 2);  // (component, row) pair, 0..63
          const int c = q >> 4, row = q & 15;
          const int dz = row >> 2, dy = row & 3;
          g += lk[it * 32] * Pb[c * N3 + ((size_t)dz * N + dy) * N];
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        g.x += __shfl_xor_sync(0xffffffffu, g.x, o);
        g.y += __shfl_xor_sync(0xffffffffu, g.y, o);
      }
      if ((lane >> 3) == r) mine = g;
    }
  }
  // near part: lane group r, sub-lane sl
  const int r = lane >> 3, sl = lane & 7;
  const bool on = k0 + r < ns;
  const int k = on ? order[k0 + r] : 0;
  long long xoff = 0;
  double xscale = 1.0;
  if (nl.xsel.sel) {
    const int jj = *nl.xsel.sel + nl.xsel.off;
    xoff = jj * nl.xsel.stride;
    if (nl.xsel.scale) xscale = nl.xsel.scale[b * 64 + jj];
  }
  double2 nr = make_double2(0, 0);
  if (on) {
    for (int e = rowptr[k] + sl; e < rowptr[k + 1]; e += 8) {
      const int j = col[e];
      for (int t = 0; t < nl.n; ++t) {
        const double2 z = nl.val[t][e];
        double2 xv = nl.x[t][xoff + (size_t)b * ns + j];
        if (nl.dinv) {
          const double2 d = nl.dinv[j];
          xv = make_double2(xv.x * d.x - xv.y * d.y, xv.x * d.y + xv.y * d.x);
        }
        nr.x += z.x * xv.x - z.y * xv.y;
        nr.y += z.x * xv.y + z.y * xv.x;
      }
    }
  }
  // sum over the 8 lanes of a group: the first exchange splits real (sl < 4) and
  // imaginary (sl >= 4) parts, so 3 FP64 additions cover both
  const bool hi = sl & 4;
  double keep = hi ? nr.y : nr.x;
  keep += __shfl_xor_sync(0xffffffffu, hi ? nr.x : nr.y, 4);
  keep += __shfl_xor_sync(0xffffffffu, keep, 2);
  keep += __shfl_xor_sync(0xffffffffu, keep, 1);
  const double nim = __shfl_down_sync(0xffffffffu, keep, 4);
  double2 out = make_double2(0, 0);
  if (on && sl == 0) {
    if (ys.sel) y += (*ys.sel + ys.off) * ys.stride;
    const double re = (double)mine.x + xscale * keep, im = (double)mine.y + xscale * nim;
    out = make_double2(sign * re, sign * im);
    if (base) {
      const double2 bb = base[(size_t)b * ns + k];
      out = make_double2(bb.x + out.x, bb.y + out.y);
    }
    y[(size_t)b * ns + k] = out;
  }
  if (df.V) {
    __shared__ double2 wsm[kInterpBlockRows];
    __shared__ int last;
    if (sl == 0) wsm[warp * kInterpRows + r] = out;  // zero for rows past ns
    __syncthreads();
    const int J = *df.jdev + 1;
    const int pb = rb * kInterpBlockRows + lane;
    const int kb = pb < ns ? order[pb] : 0;
    const double2* Vb = df.V + (size_t)b * ns;
    for (int i = warp; i < J; i += 8) {
      double2 t = make_double2(0, 0);
      if (pb < ns) {
        const double2 v = Vb[i * df.vstride + kb], w = wsm[lane];
        t = make_double2(v.x * w.x + v.y * w.y, v.x * w.y - v.y * w.x);  // conj(v) w
      }
      t = warp_sum_c(t);
      if (lane == 0) df.pd[((size_t)b * 64 + i) * df.P + rb] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      last = atomicAdd(df.ucnt + b, 1u) == (unsigned)df.P - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      if (threadIdx.x == 0) df.ucnt[b] = 0u;
      for (int i = warp; i < J; i += 8) {
        const double2* p = df.pd + ((size_t)b * 64 + i) * df.P;
        double2 t = make_double2(0, 0);
        for (int q = lane; q < df.P; q += 32) {
          const double2 v = __ldcg(p + q);
          t.x += v.x;
          t.y += v.y;
        }
        t = warp_sum_c(t);
        if (lane == 0) df.d[b * 64 + i] = t;
      }
    }
  }
  pdl_trigger();
}

// ---------------------------------------------------------------- launch helpers
template <class K>
static void smem_opt_in(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) AIM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

// precision selectors for the context tables
inline const float2* sel_tw(aim_ctx* c, float2*) { return c->d_twf; }
inline const double2* sel_tw(aim_ctx* c, double2*) { return c->d_tw; }
inline const float2* sel_twz(aim_ctx* c, float2*) { return c->d_twzf; }
inline const double2* sel_twz(aim_ctx* c, double2*) { return c->d_twz; }
inline const float2* sel_kspec(aim_ctx* c, float2*) { return c->d_kspecf; }
inline const double2* sel_kspec(aim_ctx* c, double2*) { return c->d_kspec; }
inline const float4* sel_ncoef(aim_ctx* c, float2*) { return c->d_ncoeff; }
inline const double4_32a* sel_ncoef(aim_ctx* c, double2*) { return c->d_ncoef; }
inline const float* sel_lam(aim_ctx* c, float2*) { return c->d_lamf; }
inline const float2* sel_sai(aim_ctx* c, float2*) { return c->d_saif; }
inline const double2* sel_sai(aim_ctx* c, double2*) { return c->d_sai; }
inline const double* sel_lam(aim_ctx* c, double2*) { return c->d_lam; }

// Tile widths the z and y passes are instantiated for (the autotuner picks among them).
template <class F>
inline void with_width(int w, F&& f) {
  switch (w) {
    case 8: f(std::integral_constant<int, 8>{}); break;
    case 16: f(std::integral_constant<int, 16>{}); break;
    case 32: f(std::integral_constant<int, 32>{}); break;
    case 64: f(std::integral_constant<int, 64>{}); break;
    default: throw AimError{AIM_ERR_ARG, "launch plan: unsupported tile width"};
  }
}
// z transform lengths the z pass is instantiated for (aim_ctx::LZ is one of them)
template <class F>
inline void with_zlen(int lz, F&& f) {
  switch (lz) {
    case 16: f(std::integral_constant<int, 16>{}); break;
    case 32: f(std::integral_constant<int, 32>{}); break;
    case 64: f(std::integral_constant<int, 64>{}); break;
    case 128: f(std::integral_constant<int, 128>{}); break;
    case 192: f(std::integral_constant<int, 192>{}); break;
    case 256: f(std::integral_constant<int, 256>{}); break;
    case 768: f(std::integral_constant<int, 768>{}); break;
    default: throw AimError{AIM_ERR_ARG, "unsupported z transform length"};
  }
}
constexpr size_t kPlanSmemMax = 220 * 1024;  // dynamic shared memory a plan may ask for

template <int L, class C>
struct GridOps {
  // ------------------------------------------------------------ launch shapes
  static int def_zw(const aim_ctx* c) {
    int w = 0;
    with_zlen(c->LZ, [&](auto lz) { w = zcol_width<decltype(lz)::value, C>(); });
    return w;
  }
  static int def_cw() { return col_width_p2<L, C>(); }
  static int def_rp() { return pow2_len(L) ? std::max(1, 4096 / L) : std::max(1, 256 / split_r1(L)); }
  static int def_ypb() { return std::max(1, 256 / (L / 2)); }
  static size_t smem_z(int lz, int w) { return (size_t)(lz + lz * w) * sizeof(C); }
  static size_t smem_y(int w) { return (size_t)(L + L * w) * sizeof(C); }
  static size_t smem_x(int rp) { return (size_t)(L + rp * row_tmp_pitch<L>()) * sizeof(C); }
  static size_t smem_anterp(int yp) { return (size_t)(L + 4 * yp * L + row_scratch<L>(4 * yp)) * sizeof(C); }
  // the plan holds the shapes of the context's own precision (the FP64 residual of the
  // refinement on the complex64 path runs with the defaults)
  static bool own(const aim_ctx* c) { return (c->precision == AIM_C64) == (sizeof(C) == sizeof(float2)); }
  static int zw(const aim_ctx* c) { return own(c) && c->plan.zw ? c->plan.zw : def_zw(c); }
  static int cw(const aim_ctx* c) { return own(c) && c->plan.cw ? c->plan.cw : def_cw(); }
  static int rp(const aim_ctx* c) { return own(c) && c->plan.rp ? c->plan.rp : def_rp(); }
  static int ypb(const aim_ctx* c) { return own(c) && c->plan.ypb ? c->plan.ypb : def_ypb(); }
  // candidates the autotuner times: z tiles of x-adjacent columns (w divides L), y tiles
  static std::vector<int> zwidths(const aim_ctx* c) {
    std::vector<int> v;
    for (int w : {8, 16, 32, 64})
      if (w <= L && L % w == 0 && smem_z(c->LZ, w) <= kPlanSmemMax) v.push_back(w);
    return v;
  }
  static std::vector<int> ywidths() {
    std::vector<int> v;
    for (int w : {8, 16, 32, 64})
      if (w <= L && L % w == 0 && smem_y(w) <= kPlanSmemMax) v.push_back(w);
    return v;
  }
  static std::vector<int> rps() {
    std::vector<int> v;
    for (int r : {2, 4, 8, 16, 32, 64})
      if (smem_x(r) <= 100 * 1024) v.push_back(r);
    return v;
  }
  static std::vector<int> ypbs(int N) {
    std::vector<int> v;
    for (int y : {1, 2, 4, 8})
      if (y <= N && smem_anterp(y) <= 100 * 1024) v.push_back(y);
    return v;
  }

  // stage i + forward x and y passes: v[nb][ns] (optionally times dinv) -> slab [nb][4][nz][L][L]
  // dinv non-null asks for the context's right preconditioner: the diagonal dinv, or the
  // near-zone SAI when the context built one
  static void prep(aim_ctx* c, int nb, const double2* v, const double2* dinv, VecSel vs, const int* active,
                   bool want_fp64) {
    const long long n = (long long)nb * c->ns;
    KScope ks(c, AIM_K_PREP);
    if (dinv && c->d_sai)
      launch_pdl(c->stream, dim3((unsigned)((n * 16 + 255) / 256)), dim3(256), 0, k_prep_sai<C>, v,
                 std::is_same<C, float2>::value ? (const float2*)c->d_vf : (const float2*)nullptr,
                 sel_sai(c, (C*)nullptr), (const int*)c->d_srowptr, (const int*)c->d_scol, vs, active, c->ns, nb,
                 reinterpret_cast<C*>(c->d_xs), want_fp64 ? c->d_xd : (double2*)nullptr);
    else
      launch_pdl(c->stream, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, k_prep<C>, v, dinv, vs, active, c->ns,
                 nb, reinterpret_cast<C*>(c->d_xs), want_fp64 ? c->d_xd : (double2*)nullptr);
  }

  // the active box (x, y, z node ranges): every pass touches only the grid lines that are
  // non-zero on input or needed on output; the buffers hold the box's nz z-planes only
  static int nbox(const aim_ctx* c, int d) { return c->box_hi[d] - c->box_lo[d] + 1; }
  static ZGeom zgeom(const aim_ctx* c) { return ZGeom{L, c->N, c->NZ}; }

  // anterpolation gather + forward x pass: d_xs -> A (rows of the active box)
  static void anterp_x(aim_ctx* c, int nb, const int* active) {
    const int N = c->N, yp = ypb(c);
    const size_t sm = smem_anterp(yp);
    smem_opt_in(k_anterp_rows<L, C>, sm);
    KScope ks(c, AIM_K_ANTERP_XFFT);
    launch_pdl(c->stream, dim3(nb, (nbox(c, 1) + yp - 1) / yp, c->NZ), dim3(256), sm, k_anterp_rows<L, C>,
               (const int*)c->d_nptr, (const int*)c->d_nidx, ncoef(c), reinterpret_cast<const C*>(c->d_xs), active,
               c->ns, N, yp, reinterpret_cast<C*>(c->d_A), twiddles(c), c->box_lo[1], c->box_hi[1], c->box_lo[2],
               c->NZ);
  }

  // forward y pass (pruned input): A -> slab
  static void y_fwd(aim_ctx* c, int nb, C* slab) {
    static_assert(two_step_len(L), "every supported padded length has a two-step plan");
    const int N = c->N, nz = c->NZ;
    const C* A = reinterpret_cast<const C*>(c->d_A);
    KScope ks(c, AIM_K_YFFT_FWD);
    with_width(cw(c), [&](auto wt) {
      constexpr int CW = decltype(wt)::value;
      if constexpr (CW <= L) {
        const size_t sm = smem_y(CW);
        smem_opt_in(k_cols_p2<L, CW, false, C, true>, sm);
        // lines (plane, x): inputs y in the box, all L outputs
        launch_pdl(c->stream, dim3(L / CW, nz, nb * 4), dim3(256), sm, k_cols_p2<L, CW, false, C, true>, A, slab,
                   c->box_hi[1] + 1, L, (long long)L, (long long)L, L, (long long)N * L, (long long)L * L,
                   (long long)nz * N * L, (long long)nz * L * L, twiddles(c), c->box_lo[1], 0, 0);
      } else {
        throw AimError{AIM_ERR_ARG, "launch plan: tile wider than the line"};
      }
    });
  }

  // inverse y pass (pruned output): Bf -> A
  static void y_inv(aim_ctx* c, int nb) {
    const int N = c->N, nz = c->NZ;
    KScope ks(c, AIM_K_YFFT_INV);
    with_width(cw(c), [&](auto wt) {
      constexpr int CW = decltype(wt)::value;
      if constexpr (CW <= L) {
        const size_t sm = smem_y(CW);
        smem_opt_in(k_cols_p2<L, CW, true, C>, sm);
        // lines (plane, x): all L inputs, outputs y in the box
        launch_pdl(c->stream, dim3(L / CW, nz, nb * 4), dim3(256), sm, k_cols_p2<L, CW, true, C>,
                   (const C*)c->d_Bf, reinterpret_cast<C*>(c->d_A), L, c->box_hi[1] + 1, (long long)L, (long long)L, L,
                   (long long)L * L, (long long)N * L, (long long)nz * L * L, (long long)nz * N * L, twiddles(c), 0,
                   c->box_lo[1], 0);
      } else {
        throw AimError{AIM_ERR_ARG, "launch plan: tile wider than the line"};
      }
    });
  }

  // inverse x pass (pruned output): A -> P, the rows of the active box, outputs x in the box
  static void x_inv(aim_ctx* c, int nb) {
    const int N = c->N, r = rp(c), nz = c->NZ, ny = nbox(c, 1), nrows = nb * 4 * nz * ny;
    const size_t sm = smem_x(r);
    smem_opt_in(k_rows_p2<L, true, C>, sm);
    KScope ks(c, AIM_K_XFFT_INV);
    launch_pdl(c->stream, dim3((nrows + r - 1) / r), dim3(256), sm, k_rows_p2<L, true, C>, (const C*)c->d_A,
               reinterpret_cast<C*>(c->d_P), nrows, L, c->box_hi[0] + 1, (long long)L, (long long)N, twiddles(c), r,
               RowBox{nz, ny, 0, c->box_lo[1], nz, N}, c->box_lo[0]);
  }

  static void forward_slab(aim_ctx* c, int nb, const double2* v, const double2* dinv, const int* active, C* slab,
                           VecSel vs = VecSel(), bool want_fp64 = false) {
    prep(c, nb, v, dinv, vs, active, want_fp64);
    anterp_x(c, nb, active);
    y_fwd(c, nb, slab);
  }

  // inverse y and x passes: Bf slab -> P, then interpolation + near terms
  static void backward(aim_ctx* c, int nb, const NearList& nl, const double2* base, double sign, const int* active,
                       double2* y, VecSel ys = VecSel()) {
    y_inv(c, nb);
    x_inv(c, nb);
    interp(c, nb, reinterpret_cast<const C*>(c->d_P), nl, base, sign, active, y, ys);
  }

  static void interp(aim_ctx* c, int nb, const C* P, const NearList& nl, const double2* base, double sign,
                     const int* active, double2* y, VecSel ys = VecSel()) {
    KScope ks(c, AIM_K_INTERP_NEAR);
    const unsigned nrb = (unsigned)((c->ns + kInterpBlockRows - 1) / kInterpBlockRows);
    if (nrb > 65535u) throw AimError{AIM_ERR_ARG, "interpolation: more than 2 097 120 RWGs"};
    launch_pdl(c->stream, dim3((unsigned)nb, nrb), dim3(256),
               0, k_interp_near<C>, P, (const int*)c->d_anchor, (const int*)c->d_order, lam(c), c->N, c->NZ,
               c->box_lo[2], c->ns, nb,
               (const int*)c->d_rowptr, (const int*)c->d_col, nl, base, sign, active, y, ys, c->dotfuse);
  }

  // size of one kernel-spectrum octant [LZ/2 + 1][N + 1][N + 1]
  static size_t octant(const aim_ctx* c) { return (size_t)(c->N + 1) * (c->N + 1) * (c->LZ / 2 + 1); }

  static void zconv(aim_ctx* c, int nb, int m, const int* active) {
    C* Bf = reinterpret_cast<C*>(c->d_Bf);
    const C* G = kspec(c) + (size_t)m * 2 * octant(c);
    KScope ks(c, AIM_K_ZCONV);
    with_zlen(c->LZ, [&](auto lz) {
      constexpr int LZ = decltype(lz)::value;
      if constexpr (LZ <= L) {
        with_width(zw(c), [&](auto wt) {
          constexpr int ZW = decltype(wt)::value;
          if constexpr (ZW <= L) {
            const size_t sm = smem_z(LZ, ZW);
            smem_opt_in(k_zconv_p2<LZ, ZW, C>, sm);
            launch_pdl(c->stream, dim3(nb * 4, L / ZW, L), dim3(kZThreads), sm, k_zconv_p2<LZ, ZW, C>, Bf, G,
                       zgeom(c), active, ztwiddles(c));
          } else {
            throw AimError{AIM_ERR_ARG, "launch plan: tile wider than the line"};
          }
        });
      } else {
        throw AimError{AIM_ERR_ARG, "z transform longer than the padded length"};
      }
    });
    AIM_CHECK_LAUNCH();
  }

  // Autotuner: time every candidate launch shape of each pass on this context's buffers
  // (nb = batch_max right-hand sides, the contents are irrelevant to the timing) and keep
  // the fastest.  Each pass's arithmetic per line is the same for every shape.
  static void tune(aim_ctx* c) {
    const int nb = c->batch_max;
    cudaEvent_t e0, e1;
    AIM_CUDA(cudaEventCreate(&e0));
    AIM_CUDA(cudaEventCreate(&e1));
    auto time_ms = [&](const std::function<void()>& launch) {
      launch();  // first launch: shared-memory attribute and warm-up
      float best = 1e30f;
      for (int r = 0; r < 3; ++r) {
        AIM_CUDA(cudaEventRecord(e0, c->stream));
        launch();
        AIM_CUDA(cudaEventRecord(e1, c->stream));
        AIM_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        AIM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
      }
      return best;
    };
    KPlan& p = c->plan;
    auto pick = [&](int& field, const std::vector<int>& cand, const std::function<void()>& launch) {
      float best = 1e30f;
      int arg = cand.empty() ? 0 : cand[0];
      for (int v : cand) {
        field = v;
        const float t = time_ms(launch);
        if (t < best) {
          best = t;
          arg = v;
        }
      }
      field = arg;
    };
    pick(p.zw, zwidths(c), [&] { zconv(c, nb, 0, nullptr); });
    pick(p.cw, ywidths(), [&] {
      y_fwd(c, nb, reinterpret_cast<C*>(c->d_Bf));
      y_inv(c, nb);
    });
    pick(p.rp, rps(), [&] { x_inv(c, nb); });
    pick(p.ypb, ypbs(c->N), [&] { anterp_x(c, nb, nullptr); });
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }

  // forward z-FFT of the slab in Bf into the z-spectral history layout at dst
  // (power-of-two z lengths only)
  static void zfwd(aim_ctx* c, int nb, C* dst) {
    with_zlen(c->LZ, [&](auto lz) {
      constexpr int LZ = decltype(lz)::value;
      if constexpr (pow2_len(LZ) && LZ <= L) {
        constexpr int ZW = zcol_width<LZ, C>();
        const size_t sm = smem_z(LZ, ZW);
        KScope ks(c, AIM_K_ZFWD);
        smem_opt_in(k_zfwd_spec<LZ, ZW, C>, sm);
        k_zfwd_spec<LZ, ZW, C><<<dim3(L / ZW, L, nb * 4), kZThreads, sm, c->stream>>>(
            reinterpret_cast<const C*>(c->d_Bf), dst, zgeom(c), ztwiddles(c));
        AIM_CHECK_LAUNCH();
      } else {
        throw AimError{AIM_ERR_ARG, "z-spectral history needs a power-of-two z length"};
      }
    });
  }

  static void zrhs(aim_ctx* c, int nb, const SlabList& sl) {
    C* Bf = reinterpret_cast<C*>(c->d_Bf);
    KScope ks(c, AIM_K_ZRHS);
    with_zlen(c->LZ, [&](auto lz) {
      constexpr int LZ = decltype(lz)::value;
      if constexpr (LZ <= L) {
        if constexpr (pow2_len(LZ) && LZ <= 256 && L <= 256 && std::is_same<C, float2>::value) {
          // the spectra's ring slots (the march and aim_rhs keep every history slab in the ring)
          const size_t slab = op_slab_bytes(c, c->batch_max);
          SlabRing sr{};
          sr.n = sl.n;
          bool in_ring = c->ring_tma && sl.n > 0;
          for (int i = 0; i < sl.n && in_ring; ++i) {
            const long long off = (const char*)sl.p[i] - (const char*)c->d_ring;
            in_ring = off >= 0 && off % (long long)slab == 0 && off / (long long)slab < c->n_delays;
            sr.slot[i] = in_ring ? (int)(off / (long long)slab) : 0;
            sr.m[i] = sl.m[i];
          }
          if (in_ring) {
            constexpr int ZW = L < 16 ? L : 16;
            const size_t sm = 128 + (2 * LZ * ZW + LZ + LZ * ZW) * sizeof(C);
            smem_opt_in(k_zrhs_spec_tma<LZ, ZW>, sm);
            k_zrhs_spec_tma<LZ, ZW><<<dim3(L / ZW, L, nb * 4), kZThreads, sm, c->stream>>>(
                c->ring_map, sr, kspec(c), zgeom(c), Bf, ztwiddles(c), c->d_err);
            AIM_CHECK_LAUNCH();
            return;
          }
        }
        if constexpr (pow2_len(LZ)) {
          // 16 columns per tile: one step-B item per thread, so the delay sum held in
          // registers stays at one radix-R2 slice
          constexpr int ZW = L < 16 ? L : 16;
          const size_t sm = smem_z(LZ, ZW);
          smem_opt_in(k_zrhs_spec<LZ, ZW, C>, sm);
          k_zrhs_spec<LZ, ZW, C><<<dim3(L / ZW, L, nb * 4), kZThreads, sm, c->stream>>>(sl, kspec(c), zgeom(c), Bf,
                                                                                      ztwiddles(c));
        } else {
          // 8 columns per tile: one step-B item per thread, the delay sum held in registers
          constexpr int ZW = L < 8 ? L : 8;
          const size_t sm = smem_z(LZ, ZW);
          smem_opt_in(k_zrhs_2s<LZ, ZW, C>, sm);
          k_zrhs_2s<LZ, ZW, C><<<dim3(nb * 4, L / ZW, L), kZThreads, sm, c->stream>>>(sl, kspec(c), zgeom(c), Bf,
                                                                                    ztwiddles(c));
        }
        AIM_CHECK_LAUNCH();
      } else {
        throw AimError{AIM_ERR_ARG, "z transform longer than the padded length"};
      }
    });
  }

  // blocked right-hand side: pending z-spectra -> slab of potentials in Bf (cleared)
  static void zinv_pending(aim_ctx* c, int nb, C* S) {
    with_zlen(c->LZ, [&](auto lz) {
      constexpr int LZ = decltype(lz)::value;
      if constexpr (pow2_len(LZ) && LZ <= L) {
        constexpr int ZW = L < 16 ? L : 16;
        const size_t sm = smem_z(LZ, ZW);
        KScope ks(c, AIM_K_ZINV_PENDING);
        smem_opt_in(k_zinv_pending<LZ, ZW, C>, sm);
        k_zinv_pending<LZ, ZW, C><<<dim3(L / ZW, L, nb * 4), kZThreads, sm, c->stream>>>(
            S, zgeom(c), reinterpret_cast<C*>(c->d_Bf), ztwiddles(c));
        AIM_CHECK_LAUNCH();
      } else {
        throw AimError{AIM_ERR_ARG, "the blocked right-hand side needs a power-of-two z length"};
      }
    });
  }

  static void block_square(aim_ctx* c, int nb, const BlockSquare& sq) {
    const long long n = (long long)nb * 4 * c->LZ * L * L;
    const int grid = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
    KScope ks(c, AIM_K_BLOCK_SQUARE);
    auto go = [&](auto bt) {
      constexpr int B = decltype(bt)::value;
      k_block_square<B, C><<<grid, 256, 0, c->stream>>>(sq, kspec(c), zgeom(c), c->LZ, c->n_delays, n);
    };
    switch (sq.b) {
      case 1: go(std::integral_constant<int, 1>{}); break;
      case 2: go(std::integral_constant<int, 2>{}); break;
      case 4: go(std::integral_constant<int, 4>{}); break;
      case 8: go(std::integral_constant<int, 8>{}); break;
      case 16: go(std::integral_constant<int, 16>{}); break;
      default: throw AimError{AIM_ERR_ARG, "blocked right-hand side: square size"};
    }
    AIM_CHECK_LAUNCH();
  }

  static const C* twiddles(aim_ctx* c) { return sel_tw(c, (C*)nullptr); }
  static const C* ztwiddles(aim_ctx* c) { return sel_twz(c, (C*)nullptr); }
  static const C* kspec(aim_ctx* c) { return sel_kspec(c, (C*)nullptr); }
  static const typename Real<C>::F4* ncoef(aim_ctx* c) { return sel_ncoef(c, (C*)nullptr); }
  static const typename Real<C>::T* lam(aim_ctx* c) { return sel_lam(c, (C*)nullptr); }
};
