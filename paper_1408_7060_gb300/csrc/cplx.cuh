// Complex arithmetic on float2 / double2 and the precision traits used by every kernel.
#pragma once
#include <cuda_runtime.h>

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

__host__ __device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

#define AIM_CPLX_OPS(C, R)                                                                         \
  __host__ __device__ __forceinline__ C operator+(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }   \
  __host__ __device__ __forceinline__ C operator-(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }   \
  __host__ __device__ __forceinline__ C operator*(C a, C b) {                                      \
    return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);                                       \
  }                                                                                                 \
  __host__ __device__ __forceinline__ C operator*(R s, C a) { return mkc(s * a.x, s * a.y); }       \
  __host__ __device__ __forceinline__ C conjc(C a) { return mkc(a.x, -a.y); }                      \
  /* multiply by -i (forward) or +i (inverse) */                                                    \
  __host__ __device__ __forceinline__ C mul_mi(C a) { return mkc(a.y, -a.x); }                     \
  __host__ __device__ __forceinline__ C mul_pi(C a) { return mkc(-a.y, a.x); }                     \
  __host__ __device__ __forceinline__ C& operator+=(C& a, C b) { a = a + b; return a; }

AIM_CPLX_OPS(float2, float)
AIM_CPLX_OPS(double2, double)
#undef AIM_CPLX_OPS

__host__ __device__ __forceinline__ float2 to_c(double2 a, float2) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ double2 to_c(double2 a, double2) { return a; }
__host__ __device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ double2 to_d(double2 a) { return a; }
