"""Independent FP64 CPU oracle for the SIP Helmholtz operator.

TEST INFRASTRUCTURE ONLY.  Nothing in the library path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It assembles the symmetric-interior-penalty matrix element by element and face
by face, straight from the primal bilinear form (Sec. 2.2, Eq. primal, with the
element view of Eq. IP and the block structure of Appendix A), with dense basis
matrices at the quadrature points and no sum factorisation, blocking or fusion.
It shares no code with the CUDA path; the only common module is ``sip_inputs``
(seeded meshes, orders and random vectors, which hold none of the method's
arithmetic).

Parity status of each part (what pins it is in ``tests/test_oracle_*.py``):

* quadrature / Lagrange tables: pinned (library Gauss rule, closed forms,
  polynomial exactness);
* volume + interior-face + boundary-face blocks: pinned (symmetry, the
  penalty closed form for an element indicator, Galerkin consistency for
  polynomials vanishing on the boundary, constant null space of the
  pure-Neumann stiffness, manufactured-solution convergence order P+1);
* face geometry of non-affine (bilinear / trilinear) elements: pinned by
  Galerkin consistency on jittered meshes, which is exact there (the
  integrands are polynomials once the Jacobian's adjugate is factored out),
  and by the penalty closed form on jittered quads and hexahedra with
  independently computed areas and volumes; this also pins the penalty
  length h_F = min(|K-|, |K+|) / |F| (the paper leaves tau and h_F undefined;
  that definition is the reading, |F| by the face's shared Gauss rule);
* diffusivity kappa: pinned in the volume term by exact consistency with
  -div(kappa grad u) for a kappa equal to 1 on every face; that face terms
  keep kappa = 1 is a reading (the paper has no kappa), invisible to any pin
  built on such a kappa;
* point-to-point interpolation variant (Sec. 3.3, Table 2): pinned (equals
  the shared-rule operator on conforming meshes and wherever the low-order
  side's rule is exact; symmetric exactly under the paper's exactness
  condition; the paper's three Table 2 cases classified as the paper does).
"""
from .quadrature import gauss_legendre, gauss_lobatto, lagrange_matrix, lagrange_deriv_matrix
from .assembly import SipOracle

__all__ = ["gauss_legendre", "gauss_lobatto", "lagrange_matrix", "lagrange_deriv_matrix", "SipOracle"]
