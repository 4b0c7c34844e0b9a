// Batched line transforms over the padded grid, built on block_fft.
//
// k_rows:  contiguous lines (x direction).  Row r reads n_in elements at
//          in + r*rs_in (the rest of the length-L line is zero: pruned zero
//          padding) and writes the first n_out outputs at out + r*rs_out.
// k_cols:  strided lines (y or z direction) processed as tiles of W adjacent
//          x positions, so every global access is a contiguous run of W elements.
//          Line (p2, p1, x) element i lives at base + p2*ps2 + p1*ps1 + x + i*es.
#pragma once
#include "fft.cuh"

extern __shared__ __align__(16) unsigned char aim_smem[];

template <class C>
__device__ __forceinline__ void load_twiddles(C* tw, const C* __restrict__ twg, int L) {
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = twg[i];
}

// Transform the lines of a tile (after a __syncthreads that publishes a); returns
// the buffer holding the natural-order result.  Lengths with a two-step plan use the
// two-step transform, any other the Stockham passes.
template <int L, int W, bool INV, class C>
__device__ __forceinline__ C* line_fft_cols(C* a, C* b, const C* tw) {
  if constexpr (two_step_len(L)) {
    col_fft2<L, W, INV, C>(a, b, tw);
    return a;
  } else {
    return block_fft<L, INV, true, C>(a, b, W, W, 1, tw);
  }
}
template <int L, bool INV, class C>
__device__ __forceinline__ C* line_fft_rows(C* a, C* b, int nl, const C* tw) {
  if constexpr (two_step_len(L)) {
    row_fft2<L, INV, C>(a, b, nl, tw);
    return a;
  } else {
    return block_fft<L, INV, false, C>(a, b, nl, 1, L, tw);
  }
}
// scratch elements a row tile of nl lines needs beside the tile itself
template <int L>
__host__ __device__ constexpr int row_scratch(int nl) {
  return two_step_len(L) ? nl * row_tmp_pitch<L>() : nl * L;
}

template <int L, bool INV, class C>
__global__ void __launch_bounds__(256) k_rows(const C* __restrict__ in, C* __restrict__ out, int nrows,
                                              int n_in, int n_out, long long rs_in, long long rs_out,
                                              const C* __restrict__ twg, int rpb) {
  C* tw = reinterpret_cast<C*>(aim_smem);
  C* b0 = tw + L;
  C* b1 = b0 + rpb * L;
  load_twiddles(tw, twg, L);
  const int r0 = blockIdx.x * rpb;
  (void)b1;
  const int nr = min(rpb, nrows - r0);
  for (int t = threadIdx.x; t < rpb * L; t += blockDim.x) {
    int rr = t / L, i = t % L;
    C v = mkc((decltype(C().x))0, (decltype(C().x))0);
    if (rr < nr && i < n_in) v = in[(long long)(r0 + rr) * rs_in + i];
    b0[t] = v;
  }
  __syncthreads();
  C* res = line_fft_rows<L, INV, C>(b0, b1, rpb, tw);
  for (int t = threadIdx.x; t < rpb * L; t += blockDim.x) {
    int rr = t / L, i = t % L;
    if (rr < nr && i < n_out) out[(long long)(r0 + rr) * rs_out + i] = res[t];
  }
}

// Rows of a box of a buffer of np planes of N rows per (right-hand side, component):
// row r (0 <= r < nbc * nz * ny) is buffer row ((bc * np + z0 + zz) * N + y0 + yy) with
// (bc, zz, yy) its coordinates in the box.
struct RowBox {
  int nz, ny, z0, y0, np, N;
  __device__ __forceinline__ long long row(int r) const {
    const int yy = r % ny, q = r / ny, zz = q % nz, bc = q / nz;
    return ((long long)bc * np + z0 + zz) * N + y0 + yy;
  }
};

// Two-step L = R1 * R2 rows without staging copies: thread (r, n2) reads inputs
// R2 n1 + n2 < n_in of row r straight from memory, radix-R1 butterfly, twiddle, one
// exchange through the padded tile; thread (r, k1) runs the radix-R2 butterfly and
// stores outputs out_lo <= k1 + R1 k2 < n_out straight to memory.  256 threads, rpb
// rows of the box.
template <int L, bool INV, class C>
__global__ void __launch_bounds__(256) k_rows_p2(const C* __restrict__ in, C* __restrict__ out, int nrows,
                                                 int n_in, int n_out, long long rs_in, long long rs_out,
                                                 const C* __restrict__ twg, int rpb, RowBox box, int out_lo) {
  pdl_wait();
  constexpr int R1 = split_r1(L), R2 = L / R1, P = row_tmp_pitch<L>();
  C* tw = reinterpret_cast<C*>(aim_smem);
  C* t = tw + L;
  load_twiddles(tw, twg, L);
  __syncthreads();
  const int r0 = blockIdx.x * rpb;
  const int nr = min(rpb, nrows - r0);
  for (int u = threadIdx.x; u < nr * R2; u += 256) {
    const int n2 = u % R2, r = u / R2;
    const C* src = in + box.row(r0 + r) * rs_in;
    C v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const int i = R2 * n1 + n2;
      v[n1] = i < n_in ? src[i] : C{};
    }
    DFTL<R1, L, INV, C>::run(v, tw);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      C x = v[k1];
      if (k1 && n2) {
        const C w = tw[n2 * k1];
        x = x * (INV ? conjc(w) : w);
      }
      t[r * P + k1 * (R2 + 1) + n2] = x;
    }
  }
  __syncthreads();
  for (int u = threadIdx.x; u < nr * R1; u += 256) {
    const int k1 = u % R1, r = u / R1;
    C* dst = out + box.row(r0 + r) * rs_out;
    C v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) v[n2] = t[r * P + k1 * (R2 + 1) + n2];
    DFTL<R2, L, INV, C>::run(v, tw);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int k = k1 + R1 * k2;
      if (k >= out_lo && k < n_out) dst[k] = v[k2];
    }
  }
  pdl_trigger();
}

// HALF: the input is the first L/2 samples (pruned zero padding, n_in = L/2), read
// without the zero half.
template <int L, int W, bool INV, class C, bool HALF = false>
__global__ void __launch_bounds__(256) k_cols(const C* __restrict__ in, C* __restrict__ out, int n_in,
                                              int n_out, long long es_in, long long es_out, int nx,
                                              long long ps1_in, long long ps1_out, long long ps2_in,
                                              long long ps2_out, const C* __restrict__ twg) {
  C* tw = reinterpret_cast<C*>(aim_smem);
  C* b0 = tw + L;
  C* b1 = b0 + L * W;
  load_twiddles(tw, twg, L);
  const int x0 = blockIdx.x * W;
  const int nw = min(W, nx - x0);
  const C* src = in + blockIdx.z * ps2_in + blockIdx.y * ps1_in + x0;
  C* dst = out + blockIdx.z * ps2_out + blockIdx.y * ps1_out + x0;
  constexpr bool half = HALF && two_step_len(L);
  const int rows = half ? L / 2 : L;
  for (int t = threadIdx.x; t < rows * W; t += blockDim.x) {
    int i = t / W, l = t % W;
    C v = mkc((decltype(C().x))0, (decltype(C().x))0);
    if (i < n_in && l < nw) v = src[i * es_in + l];
    b0[t] = v;
  }
  __syncthreads();
  C* res;
  if constexpr (half) {
    col_fft2<L, W, INV, C, true>(b0, b1, tw);
    res = b0;
  } else {
    res = line_fft_cols<L, W, INV, C>(b0, b1, tw);
  }
  for (int t = threadIdx.x; t < n_out * W; t += blockDim.x) {
    int i = t / W, l = t % W;
    if (l < nw) dst[i * es_out + l] = res[t];
  }
}

// Two-step L = R1 * R2 without staging copies: thread (l, n2) reads its R1 inputs
// i = R2 n1 + n2, in_lo <= i < n_in, straight from memory (HALF: n1 < R1/2 only; the
// others are zero), radix-R1 butterfly, twiddle, one exchange through
// t[(k1 R2 + n2) W + l]; thread (l, k1) runs the radix-R2 butterfly and stores the
// outputs out_lo <= k1 + R1 k2 < n_out straight to memory.  Line p1 = blockIdx.y + p1_off.
// 256 threads; tile t of L x W elements after the L twiddles.
template <int L, int W, bool INV, class C, bool HALF = false>
__global__ void __launch_bounds__(256) k_cols_p2(const C* __restrict__ in, C* __restrict__ out, int n_in,
                                                 int n_out, long long es_in, long long es_out, int nx,
                                                 long long ps1_in, long long ps1_out, long long ps2_in,
                                                 long long ps2_out, const C* __restrict__ twg, int in_lo,
                                                 int out_lo, int p1_off) {
  pdl_wait();
  constexpr int R1 = split_r1(L), R2 = L / R1;
  C* tw = reinterpret_cast<C*>(aim_smem);
  C* t = tw + L;
  load_twiddles(tw, twg, L);
  __syncthreads();
  const int x0 = blockIdx.x * W;
  const int nw = min(W, nx - x0);
  const long long p1 = (long long)blockIdx.y + p1_off;
  const C* src = in + blockIdx.z * ps2_in + p1 * ps1_in + x0;
  C* dst = out + blockIdx.z * ps2_out + p1 * ps1_out + x0;
  for (int u = threadIdx.x; u < W * R2; u += 256) {
    const int l = u % W, n2 = u / W;
    C v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const int i = R2 * n1 + n2;
      v[n1] = ((!HALF || n1 < R1 / 2) && i >= in_lo && i < n_in && l < nw) ? src[(long long)i * es_in + l] : C{};
    }
    if constexpr (HALF && R1 % 2 == 0)
      dft_half_in<R1, L, INV, C>(v, tw);
    else
      DFTL<R1, L, INV, C>::run(v, tw);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      C x = v[k1];
      if (k1 && n2) {
        const C w = tw[n2 * k1];
        x = x * (INV ? conjc(w) : w);
      }
      t[(k1 * R2 + n2) * W + l] = x;
    }
  }
  __syncthreads();
  for (int u = threadIdx.x; u < W * R1; u += 256) {
    const int l = u % W, k1 = u / W;
    C v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) v[n2] = t[(k1 * R2 + n2) * W + l];
    DFTL<R2, L, INV, C>::run(v, tw);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int k = k1 + R1 * k2;
      if (k >= out_lo && k < n_out && l < nw) dst[(long long)k * es_out + l] = v[k2];
    }
  }
  pdl_trigger();
}

// tile width of the direct two-step column passes (one L x W tile, at most ~100 KB of
// shared memory so that two blocks share an SM)
template <int L, class C>
constexpr int col_width_p2() {
  return (int)sizeof(C) == 8 ? (L < 32 ? L : L >= 512 ? 16 : 32) : (L < 16 ? L : L >= 512 ? 8 : 16);
}

// tile width of a column pass: keep 2 (or 3) L x W buffers within ~160 KB
template <int L, class C>
constexpr int col_width() {
  return (2 * L * 16 * (int)sizeof(C) <= 160 * 1024) ? 16 : (2 * L * 8 * (int)sizeof(C) <= 160 * 1024) ? 8 : 4;
}
