// complex64 instantiation of the grid stages (FP32 accumulation)
#include "operator_body.cuh"
AIM_INSTANTIATE_OPS(float2)
