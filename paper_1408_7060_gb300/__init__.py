"""GB300-native ET-AIM: the per-time-step adaptive-integral operator and march of the
envelope-tracking EFIE (Kaur & Yilmaz, arXiv:1408.7060, Sec. 4, Eq. 5) as a CUDA
library for sm_103a behind a C ABI (``include/aim.h``), with a ctypes binding."""
from .abi import (AimContext, AimError, aim_destroy, aim_excitation_vector, aim_get_anterp, aim_get_info,
                  aim_get_kernel_spectrum, aim_get_near, aim_get_profile, aim_march, aim_march_continue,
                  aim_matvec, aim_profile, aim_num_unknowns, aim_rhs,
                  aim_rwg_table, aim_setup)

__all__ = ["AimContext", "AimError", "aim_setup", "aim_destroy", "aim_get_info", "aim_num_unknowns",
           "aim_rwg_table", "aim_matvec", "aim_rhs", "aim_excitation_vector", "aim_march", "aim_get_anterp",
           "aim_get_near", "aim_get_kernel_spectrum", "aim_march_continue", "aim_profile",
           "aim_get_profile"]
