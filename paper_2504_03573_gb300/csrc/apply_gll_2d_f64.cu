// Apply kernels, 2D, double, Gauss-Lobatto-Legendre points (traces gathered,
// fluxes scattered: GathrInterp / ScatrInterp).
#define SIP_TU_RULE SIP_RULE_GLL
#define SIP_MAIN_LAUNCH_BOUNDS 256, 4
#include "apply_launch.cuh"
SIP_DEFINE_APPLY_TU(gll_2d_f64, double, 2)
SIP_DEFINE_AUX_TU(gll_2d, 2)
