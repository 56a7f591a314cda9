// Apply kernels, 2D, float, Gauss-Lobatto-Legendre points (traces gathered,
// fluxes scattered: GathrInterp / ScatrInterp).
#define SIP_TU_RULE SIP_RULE_GLL
#include "apply_launch.cuh"
SIP_DEFINE_APPLY_TU(gll_2d_f32, float, 2)
