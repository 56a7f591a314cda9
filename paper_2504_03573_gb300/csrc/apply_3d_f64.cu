// Apply kernels, 3D, double.
#define SIP_MAIN_LAUNCH_BOUNDS 256, 4
#include "apply_launch.cuh"
SIP_DEFINE_APPLY_TU(3d_f64, double, 3)
SIP_DEFINE_AUX_TU(3d, 3)
