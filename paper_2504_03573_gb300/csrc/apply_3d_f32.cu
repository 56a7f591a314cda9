// Apply kernels, 3D, float.
#include "apply_launch.cuh"
SIP_DEFINE_APPLY_TU(3d_f32, float, 3)
