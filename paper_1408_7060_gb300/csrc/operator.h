// Operator entry points shared by the API, the solver and the march.
#pragma once
#include "aim_internal.h"

// Optional device-side selection of vector j of a Krylov-style array [j][B][ns]:
// address = base + (*sel + off) * stride; scale (if set) multiplies input b by
// scale[b * 64 + *sel + off].  A null sel means "base itself" (off, stride unused).
struct VecSel {
  const int* sel = nullptr;
  long long stride = 0;
  int off = 0;
  const double* scale = nullptr;
};

// near-zone terms summed by the interpolation kernel: sum_t Z~near_{m_t} x_t
struct NearList {
  const double2* val[aimc::kMaxDelays];  // [nnz] values of one delay
  const double2* x[aimc::kMaxDelays];    // [nb][ns] vector it multiplies
  const double2* dinv;                   // optional diagonal applied to every x (preconditioner)
  VecSel xsel;                           // selection applied to every x
  int n;
};

// ring slots (of the contiguous history ring) and delays of the slabs, for the TMA path
struct SlabRing {
  int slot[aimc::kMaxDelays];
  int m[aimc::kMaxDelays];
  int n;
};

// history slabs (z-spectra of the forward x/y-transformed grids for power-of-two lengths,
// the x/y-transformed grids otherwise) and the delay each one carries
struct SlabList {
  const void* p[aimc::kMaxDelays];
  int m[aimc::kMaxDelays];
  int n;
};

// One square of the multilevel blocked delay sums (Sec. 4 stage ii): the z-spectra of b
// consecutive steps (src[j], j = 0..b-1 oldest first) radiated to the pending
// accumulators of b consecutive steps (dst[i]): dst[i] += sum_j G^_{toff+i-j} . src[j],
// delays outside 1..N_g contributing nothing.  b a power of two <= 16 (a larger square
// is launched as sub-squares with their own toff).
struct BlockSquare {
  const void* src[16];
  void* dst[16];
  int b;
  int toff;
};

// y = base + sign * Z~AIM_m (dinv .* v)     (dinv, base optional; m = delay)
void op_apply(aim_ctx* c, int m, int nb, const double2* v, const double2* dinv, const double2* base, double sign,
              const int* active, double2* y, VecSel vin = VecSel(), VecSel yout = VecSel());
// y = base + sign * Z~AIM_m v with every grid stage in FP64, whatever the context's
// precision (the residual of the FP64 refinement on the complex64 path); needs the
// refinement buffers of a complex64 context
void op_apply_f64(aim_ctx* c, int m, int nb, const double2* v, const double2* base, double sign, double2* y);
// slab of one current vector (anterpolation + forward x and y passes) written to dst
void op_forward_slab(aim_ctx* c, int nb, const double2* v, void* dst);
// y = base + sign * [ sum_s Z~FFT_{m_s} (slab_s) + near terms ]
void op_apply_rhs(aim_ctx* c, int nb, const SlabList& sl, const NearList& nl, const double2* base, double sign,
                  double2* y);
// blocked right-hand side: y = base + sign * [ grid part from the pending z-spectra P
// (which are read and cleared) + near terms ]
void op_apply_rhs_pending(aim_ctx* c, int nb, void* P, const NearList& nl, const double2* base, double sign,
                          double2* y);
void op_block_square(aim_ctx* c, int nb, const BlockSquare& sq);
// V_l for the plane waves in exc (device parameter block [nb][6]: khat, phat)
void op_excitation(aim_ctx* c, int nb, const double* d_kp, double sigma, double t_d, int step_l, double2* out);
int op_kernel_count(const aim_ctx* c);
// choose the launch shapes of the grid passes (aim_opts.autotune: 1 tune or reuse the
// cached plan, 2 tune and refresh the cache); leaves the defaults on mode 0
void op_autotune(aim_ctx* c, int mode);
size_t op_slab_bytes(const aim_ctx* c, int nb);
