// Apply kernels, 3D, float, Gauss-Lobatto-Legendre points (traces gathered,
// fluxes scattered: GathrInterp / ScatrInterp).
#define SIP_TU_RULE SIP_RULE_GLL
#include "apply_launch.cuh"
SIP_DEFINE_APPLY_TU(gll_3d_f32, float, 3)
