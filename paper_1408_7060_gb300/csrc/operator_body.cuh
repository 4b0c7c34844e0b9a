// Precision-generic operator sequences, dispatched over the supported padded lengths.
#pragma once
#include "operator_impl.cuh"

// supported padded lengths L = 2N (grid N in {8, 16, 32, 64, 96, 128, 384})
#define AIM_DISPATCH_L(Lrt, ...)                                      \
  switch (Lrt) {                                                       \
    case 16: { constexpr int LL = 16; __VA_ARGS__; } break;                   \
    case 32: { constexpr int LL = 32; __VA_ARGS__; } break;                   \
    case 64: { constexpr int LL = 64; __VA_ARGS__; } break;                   \
    case 128: { constexpr int LL = 128; __VA_ARGS__; } break;                 \
    case 192: { constexpr int LL = 192; __VA_ARGS__; } break;                 \
    case 256: { constexpr int LL = 256; __VA_ARGS__; } break;                 \
    case 768: { constexpr int LL = 768; __VA_ARGS__; } break;                 \
    default: throw AimError{AIM_ERR_ARG, "unsupported grid size"};     \
  }

template <class C>
void body_apply(aim_ctx* c, int m, int nb, const double2* v, const double2* dinv, const double2* base, double sign,
                const int* active, double2* y, VecSel vin, VecSel yout) {
  NearList nl{};
  nl.dinv = nullptr;
  nl.n = 0;
  if (c->nnz > 0) {  // the near term multiplies the prepared FP64 input
    nl.n = 1;
    nl.val[0] = c->d_near + (size_t)m * c->nnz;
    nl.x[0] = c->d_xd;
  }
  AIM_DISPATCH_L(c->L, {
    GridOps<LL, C>::forward_slab(c, nb, v, dinv, active, reinterpret_cast<C*>(c->d_Bf), vin, true);
    GridOps<LL, C>::zconv(c, nb, m, active);
    GridOps<LL, C>::backward(c, nb, nl, base, sign, active, y, yout);
  });
}

// a history slab: x/y-transformed (factor-3 z lengths) or, for power-of-two z lengths,
// also z-transformed (through Bf, which must not be dst)
template <class C>
void body_forward_slab(aim_ctx* c, int nb, const double2* v, void* dst) {
  AIM_DISPATCH_L(c->L, {
    if (pow2_len(c->LZ)) {
      GridOps<LL, C>::forward_slab(c, nb, v, nullptr, nullptr, reinterpret_cast<C*>(c->d_Bf));
      GridOps<LL, C>::zfwd(c, nb, reinterpret_cast<C*>(dst));
    } else {
      GridOps<LL, C>::forward_slab(c, nb, v, nullptr, nullptr, reinterpret_cast<C*>(dst));
    }
  });
}

template <class C>
void body_apply_rhs(aim_ctx* c, int nb, const SlabList& sl, const NearList& nl, const double2* base, double sign,
                    double2* y) {
  AIM_DISPATCH_L(c->L, {
    if (sl.n > 0) {
      GridOps<LL, C>::zrhs(c, nb, sl);
      GridOps<LL, C>::backward(c, nb, nl, base, sign, nullptr, y);
    } else {
      GridOps<LL, C>::interp(c, nb, nullptr, nl, base, sign, nullptr, y);
    }
  });
}

template <class C>
void body_apply_rhs_pending(aim_ctx* c, int nb, void* P, const NearList& nl, const double2* base, double sign,
                            double2* y) {
  AIM_DISPATCH_L(c->L, {
    GridOps<LL, C>::zinv_pending(c, nb, reinterpret_cast<C*>(P));
    GridOps<LL, C>::backward(c, nb, nl, base, sign, nullptr, y);
  });
}

template <class C>
void body_block_square(aim_ctx* c, int nb, const BlockSquare& sq) {
  AIM_DISPATCH_L(c->L, GridOps<LL, C>::block_square(c, nb, sq));
}

template <class C>
void body_tune(aim_ctx* c) {
  AIM_DISPATCH_L(c->L, GridOps<LL, C>::tune(c));
}

template <class C>
void body_plan_fill(aim_ctx* c) {
  AIM_DISPATCH_L(c->L, {
    KPlan& p = c->plan;
    p.zw = GridOps<LL, C>::zw(c);
    p.cw = GridOps<LL, C>::cw(c);
    p.rp = GridOps<LL, C>::rp(c);
    p.ypb = GridOps<LL, C>::ypb(c);
  });
}

#define AIM_INSTANTIATE_OPS(C)                                                                                   \
  template void body_tune<C>(aim_ctx*);                                                                         \
  template void body_plan_fill<C>(aim_ctx*);                                                                    \
  template void body_apply<C>(aim_ctx*, int, int, const double2*, const double2*, const double2*, double,       \
                              const int*, double2*, VecSel, VecSel);                                             \
  template void body_forward_slab<C>(aim_ctx*, int, const double2*, void*);                                     \
  template void body_apply_rhs<C>(aim_ctx*, int, const SlabList&, const NearList&, const double2*, double,      \
                                  double2*);                                                                   \
  template void body_apply_rhs_pending<C>(aim_ctx*, int, void*, const NearList&, const double2*, double,        \
                                          double2*);                                                           \
  template void body_block_square<C>(aim_ctx*, int, const BlockSquare&);
