// complex128 instantiation of the grid stages (the plain path)
#include "operator_body.cuh"
AIM_INSTANTIATE_OPS(double2)
