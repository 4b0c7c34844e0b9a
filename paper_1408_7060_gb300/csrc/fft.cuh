// Shared-memory complex FFT of padded grid lines (length L = 2N), Stockham autosort.
//
// A line of length L = R_1 R_2 ... R_s is transformed in s radix-R passes.  Pass
// with radix R and accumulated sub-length Ns reads v[r] = in[j + r L/R] for
// j in [0, L/R), applies the twiddles W_{Ns R}^{r (j mod Ns)}, a length-R DFT, and
// writes out[(j/Ns) Ns R + (j mod Ns) + r Ns]; the output is in natural order
// after the last pass.  Twiddles come from a table W_L^t = exp(-2 pi i t / L)
// computed on the host in FP64.  Forward uses exp(-...), inverse exp(+...), and
// neither scales (the 1/L^3 of the inverse is folded into the kernel spectra).
#pragma once
#include "cplx.cuh"

// radix plans: every supported padded length
__host__ __device__ constexpr int plan_len(int L) {
  return L == 16 ? 2 : L == 32 ? 2 : L == 64 ? 2 : L == 96 ? 3 : L == 128 ? 3 : L == 192 ? 3
       : L == 256 ? 3 : L == 384 ? 4 : L == 512 ? 3 : L == 768 ? 4 : 0;
}
__host__ __device__ constexpr int plan_rad(int L, int s) {
  return L == 16 ? 4
       : L == 32 ? (s == 0 ? 8 : 4)
       : L == 64 ? 8
       : L == 96 ? (s == 0 ? 8 : s == 1 ? 4 : 3)
       : L == 128 ? (s == 0 ? 8 : 4)
       : L == 192 ? (s < 2 ? 8 : 3)
       : L == 256 ? (s < 2 ? 8 : 4)
       : L == 384 ? (s == 0 ? 8 : s < 3 ? 4 : 3)
       : L == 512 ? 8
       : L == 768 ? (s < 2 ? 8 : s == 2 ? 4 : 3)
       : 0;
}

// ---------------------------------------------------------------- small DFTs
template <bool INV, class C>
__device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a - b;
  a = a + b;
  b = t;
}

template <bool INV, class C>
__device__ __forceinline__ C rot_q(C a) {  // multiply by W_4 = -i (forward) / +i (inverse)
  return INV ? mul_pi(a) : mul_mi(a);
}

template <bool INV, class C>
__device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
  C t0 = v0 + v2, t1 = v0 - v2, t2 = v1 + v3, t3 = rot_q<INV>(v1 - v3);
  v0 = t0 + t2;
  v2 = t0 - t2;
  v1 = t1 + t3;
  v3 = t1 - t3;
}

template <int R, bool INV, class C> struct DFT;

template <bool INV, class C> struct DFT<2, INV, C> {
  __device__ __forceinline__ static void run(C* v) { dft2<INV>(v[0], v[1]); }
};
template <bool INV, class C> struct DFT<4, INV, C> {
  __device__ __forceinline__ static void run(C* v) { dft4<INV>(v[0], v[1], v[2], v[3]); }
};
template <bool INV, class C> struct DFT<8, INV, C> {
  __device__ __forceinline__ static void run(C* v) {
    using Rl = decltype(v[0].x);
    const Rl h = (Rl)0.70710678118654752440;  // 1/sqrt(2)
    dft4<INV>(v[0], v[2], v[4], v[6]);       // even samples -> E_q
    dft4<INV>(v[1], v[3], v[5], v[7]);       // odd samples  -> O_q
    // X_q = E_q + W_8^q O_q, X_{q+4} = E_q - W_8^q O_q
    C o1 = v[3], o2 = v[5], o3 = v[7];
    C w1 = INV ? mkc(h * (o1.x - o1.y), h * (o1.x + o1.y)) : mkc(h * (o1.x + o1.y), h * (o1.y - o1.x));
    C w2 = rot_q<INV>(o2);
    C w3 = INV ? mkc(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : mkc(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = e0 + o0; v[4] = e0 - o0;
    v[1] = e1 + w1; v[5] = e1 - w1;
    v[2] = e2 + w2; v[6] = e2 - w2;
    v[3] = e3 + w3; v[7] = e3 - w3;
  }
};
template <bool INV, class C> struct DFT<3, INV, C> {
  __device__ __forceinline__ static void run(C* v) {
    using Rl = decltype(v[0].x);
    const Rl s3 = (Rl)0.86602540378443864676;  // sqrt(3)/2
    C s = v[1] + v[2], d = v[1] - v[2];
    C t = mkc(v[0].x - (Rl)0.5 * s.x, v[0].y - (Rl)0.5 * s.y);
    C jd = mkc(-s3 * d.y, s3 * d.x);  // i sqrt(3)/2 d
    v[0] = v[0] + s;
    v[1] = INV ? t + jd : t - jd;
    v[2] = INV ? t - jd : t + jd;
  }
};

// ---------------------------------------------------------------- one pass
// nl lines; element i of line l sits at buf[l*ls + i*es].  LF: consecutive
// threads walk consecutive lines (column tiles); else consecutive butterflies.
template <int L, int R, int NS, bool INV, bool LF, class C>
__device__ __forceinline__ void fft_pass(const C* __restrict__ in, C* __restrict__ out, int nl, int es,
                                         int ls, const C* __restrict__ tw) {
  constexpr int NB = L / R;
  const int units = nl * NB;
  for (int t = threadIdx.x; t < units; t += blockDim.x) {
    int line, j;
    if (LF) { line = t % nl; j = t / nl; } else { j = t % NB; line = t / NB; }
    const C* src = in + line * ls;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(j + r * NB) * es];
    if (NS > 1) {
      const int k = j % NS;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = tw[r * k * (L / (NS * R))];
        v[r] = v[r] * (INV ? conjc(w) : w);
      }
    }
    DFT<R, INV, C>::run(v);
    const int base = (j / NS) * NS * R + (j % NS);
    C* dst = out + line * ls;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(base + r * NS) * es] = v[r];
  }
}

template <int L, int S, int NS, bool INV, bool LF, class C>
__device__ __forceinline__ C* fft_passes(C* a, C* b, int nl, int es, int ls, const C* tw) {
  if constexpr (S == plan_len(L)) {
    return a;
  } else {
    constexpr int R = plan_rad(L, S);
    fft_pass<L, R, NS, INV, LF, C>(a, b, nl, es, ls, tw);
    __syncthreads();
    return fft_passes<L, S + 1, NS * R, INV, LF, C>(b, a, nl, es, ls, tw);
  }
}

// Transform nl lines held in a; b is scratch of the same size.  Returns the
// buffer holding the result.  Must be called by every thread of the block, after
// a __syncthreads() that publishes a.
template <int L, bool INV, bool LF, class C>
__device__ __forceinline__ C* block_fft(C* a, C* b, int nl, int es, int ls, const C* tw) {
  static_assert(plan_len(L) > 0, "unsupported FFT length");
  return fft_passes<L, 0, 1, INV, LF, C>(a, b, nl, es, ls, tw);
}

// ---------------------------------------------------------------- radix-16 in registers
// 16 = 4 x 4: four DFT4 over stride-4 samples, twiddles W_16^{n2 k1}, four DFT4 across.
template <bool INV, class C> struct DFT<16, INV, C> {
  __device__ __forceinline__ static C w16(C a, int q) {  // a * W_16^q (forward) or conj
    using Rl = decltype(a.x);
    const Rl c1 = (Rl)0.92387953251128675613, s1 = (Rl)0.38268343236508977173, h = (Rl)0.70710678118654752440;
    Rl c, s;  // W_16^q = c - i s
    switch (q) {
      case 0: return a;
      case 1: c = c1; s = s1; break;
      case 2: c = h; s = h; break;
      case 3: c = s1; s = c1; break;
      case 4: c = 0; s = 1; break;
      case 6: c = -h; s = h; break;
      case 9: c = -c1; s = -s1; break;
      default: c = 0; s = 0; break;
    }
    if (INV) s = -s;
    return mkc(a.x * c + a.y * s, a.y * c - a.x * s);
  }
  __device__ __forceinline__ static void run(C* v) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
    // now v[4 k1 + n2] holds y[k1][n2]; twiddle then DFT4 over n2
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
      for (int n2 = 1; n2 < 4; ++n2) v[4 * k1 + n2] = w16(v[4 * k1 + n2], k1 * n2);
    C t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      C a0 = v[4 * k1], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
      dft4<INV>(a0, a1, a2, a3);
      t[k1] = a0;
      t[k1 + 4] = a1;
      t[k1 + 8] = a2;
      t[k1 + 12] = a3;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = t[q];
  }
};

// ---------------------------------------------------------------- composite radices in registers
// The two-step transforms of the lengths with a factor 3 (768 = 32 x 24, 192 = 16 x 12,
// 96 = 8 x 12) need radices 12, 24, 48 and 32.  A radix R = RA RB is split once more in
// registers, with n = RB na + nb and k = ka + RA kb:
//   X[ka + RA kb] = sum_nb W_RB^{nb kb} [W_R^{nb ka} sum_na x[RB na + nb] W_RA^{na ka}].
// Its twiddles W_R^q = cos(2 pi q/R) - i sin(2 pi q/R) are compile-time constants: the
// loops are unrolled, q is known, and qcos<R> holds cos(2 pi r/R) for r = 0..R/4 (the
// exact values to 21 digits, from a 30-digit evaluation); the other quadrants follow by
// symmetry.  (The table argument tw is unused by these radices.)
template <int R> __device__ __forceinline__ double qcos(int r);
template <> __device__ __forceinline__ double qcos<4>(int r) { return r == 0 ? 1.0 : 0.0; }
template <> __device__ __forceinline__ double qcos<8>(int r) {
  return r == 0 ? 1.0 : r == 1 ? 0.707106781186547524401 : 0.0;
}
template <> __device__ __forceinline__ double qcos<16>(int r) {
  switch (r) {
    case 0: return 1.0;
    case 1: return 0.923879532511286756128;
    case 2: return 0.707106781186547524401;
    case 3: return 0.382683432365089771728;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double qcos<12>(int r) {
  switch (r) {
    case 0: return 1.0;
    case 1: return 0.866025403784438646764;
    case 2: return 0.5;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double qcos<24>(int r) {
  switch (r) {
    case 0: return 1.0;
    case 1: return 0.96592582628906828675;
    case 2: return 0.866025403784438646764;
    case 3: return 0.707106781186547524401;
    case 4: return 0.5;
    case 5: return 0.258819045102520762349;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double qcos<32>(int r) {
  switch (r) {
    case 0: return 1.0;
    case 1: return 0.980785280403230449126;
    case 2: return 0.923879532511286756128;
    case 3: return 0.831469612302545237079;
    case 4: return 0.707106781186547524401;
    case 5: return 0.555570233019602224743;
    case 6: return 0.382683432365089771728;
    case 7: return 0.195090322016128267848;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double qcos<48>(int r) {
  switch (r) {
    case 0: return 1.0;
    case 1: return 0.991444861373810411145;
    case 2: return 0.96592582628906828675;
    case 3: return 0.923879532511286756128;
    case 4: return 0.866025403784438646764;
    case 5: return 0.79335334029123516458;
    case 6: return 0.707106781186547524401;
    case 7: return 0.608761429008720639416;
    case 8: return 0.5;
    case 9: return 0.382683432365089771728;
    case 10: return 0.258819045102520762349;
    case 11: return 0.130526192220051591548;
    default: return 0.0;
  }
}

// a * W_R^q (forward) or a * conj(W_R^q) (inverse), W_R^q = exp(-2 pi i q / R)
template <int R, bool INV, class C>
__device__ __forceinline__ C mul_root(C a, int q) {
  using Rl = decltype(a.x);
  double c, s;  // cos, sin of 2 pi q / R
  if constexpr (R == 6) {
    const double h = 0.866025403784438646764;
    const int m = q % 6;
    c = m == 0 ? 1.0 : m == 3 ? -1.0 : (m == 1 || m == 5) ? 0.5 : -0.5;
    s = (m == 1 || m == 2) ? h : (m == 4 || m == 5) ? -h : 0.0;
  } else {
    constexpr int Q = R / 4;
    const int m = q % R, j = m / Q, r = m % Q;
    const double c0 = qcos<R>(r), s0 = qcos<R>(Q - r);
    c = j == 0 ? c0 : j == 1 ? -s0 : j == 2 ? -c0 : s0;
    s = j == 0 ? s0 : j == 1 ? c0 : j == 2 ? -s0 : -c0;
  }
  if (INV) s = -s;
  const Rl cr = (Rl)c, sr = (Rl)s;  // a (c - i s)
  return mkc(a.x * cr + a.y * sr, a.y * cr - a.x * sr);
}
template <int R> struct RadixSplit { static constexpr int A = 0, B = 0; };
template <> struct RadixSplit<6> { static constexpr int A = 2, B = 3; };
template <> struct RadixSplit<12> { static constexpr int A = 4, B = 3; };
template <> struct RadixSplit<24> { static constexpr int A = 8, B = 3; };
template <> struct RadixSplit<48> { static constexpr int A = 16, B = 3; };
template <> struct RadixSplit<32> { static constexpr int A = 8, B = 4; };

template <int R> __host__ __device__ constexpr bool simple_radix() { return R == 2 || R == 3 || R == 4 || R == 8 || R == 16; }

template <int R, int L, bool INV, class C>
struct DFTL {
  __device__ __forceinline__ static void run(C* v, const C* tw) {
    if constexpr (simple_radix<R>()) {
      DFT<R, INV, C>::run(v);
    } else {
      constexpr int RA = RadixSplit<R>::A, RB = RadixSplit<R>::B;
      static_assert(RA * RB == R && L % R == 0, "unsupported composite radix");
      C t[R];
#pragma unroll
      for (int nb = 0; nb < RB; ++nb) {
        C a[RA];
#pragma unroll
        for (int na = 0; na < RA; ++na) a[na] = v[RB * na + nb];
        DFTL<RA, L, INV, C>::run(a, tw);
#pragma unroll
        for (int ka = 0; ka < RA; ++ka) {
          C x = a[ka];
          if (ka && nb) x = mul_root<R, INV, C>(x, nb * ka);
          t[ka * RB + nb] = x;
        }
      }
#pragma unroll
      for (int ka = 0; ka < RA; ++ka) {
        C b[RB];
#pragma unroll
        for (int nb = 0; nb < RB; ++nb) b[nb] = t[ka * RB + nb];
        DFTL<RB, L, INV, C>::run(b, tw);
#pragma unroll
        for (int kb = 0; kb < RB; ++kb) v[ka + RA * kb] = b[kb];
      }
    }
  }
};

// Even radix R with only the first R/2 inputs non-zero (the pruned zero padding):
//   X[2k] = DFT_{R/2}(x)[k],  X[2k+1] = DFT_{R/2}(x[n] W_R^n)[k],
// two half-length butterflies instead of a full one fed with zeros.  v[0..R/2) in,
// v[0..R) out in natural order.
template <int R, int L, bool INV, class C>
__device__ __forceinline__ void dft_half_in(C* v, const C* tw) {
  constexpr int H = R / 2;
  C e[H], o[H];
#pragma unroll
  for (int n = 0; n < H; ++n) {
    e[n] = v[n];
    o[n] = n ? mul_root<R, INV, C>(v[n], n) : v[n];
  }
  DFTL<H, L, INV, C>::run(e, tw);
  DFTL<H, L, INV, C>::run(o, tw);
#pragma unroll
  for (int k = 0; k < H; ++k) {
    v[2 * k] = e[k];
    v[2 * k + 1] = o[k];
  }
}

// Even radix R when only the first R/2 outputs are needed (the pruned inverse):
//   x[n] = A[n] + W_R^{+-n} B[n],  A, B the half-length transforms of the even and odd
// inputs.  v[0..R) in, v[0..R/2) out.
template <int R, int L, bool INV, class C>
__device__ __forceinline__ void dft_half_out(C* v, const C* tw) {
  constexpr int H = R / 2;
  C e[H], o[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = v[2 * j];
    o[j] = v[2 * j + 1];
  }
  DFTL<H, L, INV, C>::run(e, tw);
  DFTL<H, L, INV, C>::run(o, tw);
#pragma unroll
  for (int n = 0; n < H; ++n) v[n] = e[n] + (n ? mul_root<R, INV, C>(o[n], n) : o[n]);
}

// ---------------------------------------------------------------- two-step transform
// For L = R1 R2 (two_step_len): with n = R2 n1 + n2 and k = k1 + R1 k2,
//   X[k1 + R1 k2] = sum_{n2} W_{R2}^{n2 k2} W_L^{n2 k1} sum_{n1} x[R2 n1 + n2] W_{R1}^{n1 k1}.
// Step A: one radix-R1 DFT per (line, n2) and the twiddles W_L^{n2 k1};
// step B: one radix-R2 DFT per (line, k1).  Each step reads and writes shared memory once.
__host__ __device__ constexpr bool pow2_len(int L) { return L == 16 || L == 32 || L == 64 || L == 128 || L == 256 || L == 512; }
// lengths with a two-step plan: the powers of two and 96 = 8 x 12, 192 = 16 x 12, 768 = 32 x 24
__host__ __device__ constexpr bool two_step_len(int L) { return pow2_len(L) || L == 96 || L == 192 || L == 768; }
__host__ __device__ constexpr int split_r1(int L) {
  return L == 16 ? 4 : L == 32 ? 8 : L == 64 ? 8 : L == 128 ? 8 : L == 256 ? 16 : L == 512 ? 16
       : L == 96 ? 8 : L == 192 ? 16 : L == 768 ? 32 : 0;
}

// Column tile: W lines, element i of line l at a[i*W + l].  Result in natural order in a.
// HALF_IN: only the first L/2 samples are nonzero (zero padding), so step A reads
// n1 < R1/2 and the zero half is folded out of the radix-R1 butterfly.
template <int L, int W, bool INV, class C, bool HALF_IN = false>
__device__ __forceinline__ void col_fft2(C* a, C* tmp, const C* __restrict__ tw) {
  constexpr int R1 = split_r1(L), R2 = L / R1;
  for (int u = threadIdx.x; u < W * R2; u += blockDim.x) {
    const int l = u % W, n2 = u / W;
    C v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = (HALF_IN && n1 >= R1 / 2) ? C{} : a[(R2 * n1 + n2) * W + l];
    if constexpr (HALF_IN && R1 % 2 == 0)
      dft_half_in<R1, L, INV, C>(v, tw);
    else
      DFTL<R1, L, INV, C>::run(v, tw);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      C x = v[k1];
      if (k1 && n2) {
        C w = tw[n2 * k1];
        x = x * (INV ? conjc(w) : w);
      }
      tmp[(k1 * R2 + n2) * W + l] = x;
    }
  }
  __syncthreads();
  for (int u = threadIdx.x; u < W * R1; u += blockDim.x) {
    const int l = u % W, k1 = u / W;
    C v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) v[n2] = tmp[(k1 * R2 + n2) * W + l];
    DFTL<R2, L, INV, C>::run(v, tw);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) a[(k1 + R1 * k2) * W + l] = v[k2];
  }
  __syncthreads();
}

// Row tile: nl lines, element n of line r at a[r*L + n]; tmp holds nl * R1 * (R2 + 1)
// elements (one padding slot per k1 row against bank conflicts).  Result in a.
template <int L> __host__ __device__ constexpr int row_tmp_pitch() {
  return split_r1(L) * (L / split_r1(L) + 1);
}
template <int L, bool INV, class C, bool HALF_IN = false>
__device__ __forceinline__ void row_fft2(C* a, C* tmp, int nl, const C* __restrict__ tw) {
  constexpr int R1 = split_r1(L), R2 = L / R1, P = row_tmp_pitch<L>();
  for (int u = threadIdx.x; u < nl * R2; u += blockDim.x) {
    const int n2 = u % R2, r = u / R2;
    C v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = (HALF_IN && n1 >= R1 / 2) ? C{} : a[r * L + R2 * n1 + n2];
    if constexpr (HALF_IN && R1 % 2 == 0)
      dft_half_in<R1, L, INV, C>(v, tw);
    else
      DFTL<R1, L, INV, C>::run(v, tw);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      C x = v[k1];
      if (k1 && n2) {
        C w = tw[n2 * k1];
        x = x * (INV ? conjc(w) : w);
      }
      tmp[r * P + k1 * (R2 + 1) + n2] = x;
    }
  }
  __syncthreads();
  for (int u = threadIdx.x; u < nl * R1; u += blockDim.x) {
    const int k1 = u % R1, r = u / R1;
    C v[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) v[n2] = tmp[r * P + k1 * (R2 + 1) + n2];
    DFTL<R2, L, INV, C>::run(v, tw);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) a[r * L + k1 + R1 * k2] = v[k2];
  }
  __syncthreads();
}
