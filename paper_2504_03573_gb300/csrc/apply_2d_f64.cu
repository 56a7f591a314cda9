// Apply kernels, 2D, double.
#define SIP_MAIN_LAUNCH_BOUNDS 256, 4
#include "apply_launch.cuh"
SIP_DEFINE_APPLY_TU(2d_f64, double, 2)
SIP_DEFINE_AUX_TU(2d, 2)
