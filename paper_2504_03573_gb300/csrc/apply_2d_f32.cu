// Apply kernels, 2D, float.
#include "apply_launch.cuh"
SIP_DEFINE_APPLY_TU(2d_f32, float, 2)
