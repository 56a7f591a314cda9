/*
 * sip.h — C ABI of the GB300 library for the matrix-free symmetric interior
 * penalty (SIP) Helmholtz operator on quad/hex meshes with per-element order.
 *
 * Operator (Sec. 2.2, Eq. IP and Eq. primal; shared trace space of Sec. 3.3):
 *
 *   a(v,u) = sum_K (kappa grad v, grad u)_K + lambda (v,u)_K
 *          - ({grad v},[[u]])_Gamma - ([[v]],{grad u})_Gamma + tau_F ([[u]],[[v]])_Gamma
 *
 * discretised with tensor Lagrange polynomials on P+1 Gauss-Lobatto-Legendre
 * nodes per direction (Table 1, Lagrange-GLL; Eq. expansion), a (P+2)-point
 * rule per direction in the volume (Eq. iproduct) and ONE rule with
 * max(P-,P+)+2 points per direction on each face, shared by both sides
 * (Sec. 3.3, "shared trace space"; the mortar-equivalent point evaluation of
 * Sec. 3.3).  The rules are Gauss-Legendre (default: traces evaluated from the
 * element, TracePhysEval / TraceIProduct of Sec. 3.2) or Gauss-Lobatto-Legendre
 * (sip_options.quad_rule = SIP_RULE_GLL: the volume points include the
 * endpoints, so a conforming trace is a gather of the boundary points and the
 * flux goes back by a scatter, GathrInterp / ScatrInterp of Sec. 3.2 and
 * Sec. 5.1).  Boundary faces use Nitsche's weak Dirichlet condition with g = 0
 * ([[u]] = u n, {grad u} = grad u).  Penalty:
 *   tau_F = tau_scale (max(P-,P+)+1)^2 / h_F,  h_F = min(|K-|,|K+|) / |F|.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - DOF vectors are element major: element e owns entries
 *   [dof_off[e], dof_off[e+1]) with (P_e+1)^dim values, node index
 *   i0 + N i1 (+ N^2 i2), N = P_e+1, i0 along the element's first reference
 *   axis (local vertex bit 0).  Multi-RHS arrays are [nrhs][ndof], contiguous.
 * - Quadrature-point arrays (kappa, its gradient, iproduct input) are element
 *   major with Q_e^dim volume points per element (Q_e = P_e + 2 unless
 *   sip_options.qorders says otherwise; points of the handle's rule),
 *   lexicographic, first reference axis fastest; offsets from sip_quad_offsets.
 * - Pointers named *_dev are CUDA device pointers owned by the caller; *_host
 *   are host pointers.  `stream` is a cudaStream_t passed as void* (NULL =
 *   legacy default stream).  Work is enqueued on that stream; the library does
 *   not synchronise the device except where a function says so.
 * - Every function returns SIP_OK (0) or a SIP_ERR_* code; nothing aborts and
 *   no device trap is used.  sip_last_error() returns a thread-local message
 *   describing the most recent failure on the calling thread.
 * - A handle is not thread safe: calls on one handle must be serialised by the
 *   caller (they share internal scratch buffers).
 */
#ifndef SIP_H
#define SIP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SIP_OK                0
#define SIP_ERR_ARG           1  /* invalid argument (null pointer, bad size, order outside 1..SIP_MAX_ORDER) */
#define SIP_ERR_MESH          2  /* non-manifold face, element glued to itself, non-positive Jacobian */
#define SIP_ERR_CUDA          3  /* a CUDA runtime call failed (message has the CUDA error string) */
#define SIP_ERR_OOM           4  /* device allocation failed */
#define SIP_ERR_NONFINITE     5  /* NaN/Inf in an input or in a CG scalar */
#define SIP_ERR_NOT_CONVERGED 6  /* CG reached max_iter; stats hold the last residual */
#define SIP_ERR_BREAKDOWN     7  /* p^T A p <= 0 in CG (operator not positive definite) */
#define SIP_ERR_NO_DEVICE     8  /* no CUDA device, or the library was built without it */

#define SIP_FP64 0              /* apply in double precision */
#define SIP_FP32 1              /* apply in single precision with single accumulation */

/* Interior-face flux evaluation (sip_options.face_scheme) */
#define SIP_FACES_SHARED    0   /* one rule per face shared by both sides (Sec. 3.3) */
#define SIP_FACES_P2P       1   /* point-to-point interpolation between the sides' own rules
                                   (Sec. 3.3 "Point-to-point interpolation", Table 2) */

/* Volume and face point sets (sip_options.quad_rule); P+2 points per direction either way */
#define SIP_RULE_GAUSS      0   /* Gauss-Legendre: traces evaluated from the element (TracePhysEval,
                                   Sec. 3.2), lifted by TraceIProduct */
#define SIP_RULE_GLL        1   /* Gauss-Lobatto-Legendre: the boundary points of the volume rule are the
                                   face points, so traces are gathered and fluxes scattered back before
                                   one IProduct (GathrInterp / ScatrInterp, Sec. 3.2, Sec. 5.1) */

#define SIP_CG_FP64         0   /* plain CG, FP64 apply */
#define SIP_CG_FP32_REFINED 1   /* FP64 iterative refinement around an FP32-apply CG */

#define SIP_MAX_ORDER 10

/* Mesh: vertex coordinates and element connectivity (read only, copied). */
typedef struct sip_mesh {
    int32_t dim;              /* 2 (quadrilaterals) or 3 (hexahedra) */
    int64_t n_vert;
    const double* vert;       /* host [n_vert][dim] */
    int64_t n_elem;
    const int64_t* elem_vert; /* host [n_elem][2^dim]; local vertex c sits at reference
                                 corner xi_k = (bit k of c) ? +1 : -1 (multilinear map) */
} sip_mesh;

typedef struct sip_options {
    double  tau_scale;        /* penalty factor in tau_F, default 2 */
    int32_t qvol_extra;       /* Q = P + qvol_extra volume points; only 2 is supported */
    int32_t boundary;         /* 1: Nitsche faces on the boundary (default); 0: drop them
                                 (pure Neumann operator) */
    double  inner_rtol;       /* FP32 inner CG tolerance in SIP_CG_FP32_REFINED, default 1e-5 */
    int32_t max_iter;         /* CG iteration cap (total inner iterations), default 20000 */
    int32_t check_every;      /* CG iterations per captured graph launch, default 16 */
    int32_t max_refine;       /* outer refinement steps cap, default 30 */
    int32_t checkpoint_every; /* save the CG state every k iterations (sip_cg_checkpoint_*); 0 = off */
    int32_t checkpoint_slots; /* ring size for checkpoints, default 8 */
    int32_t face_scheme;      /* SIP_FACES_SHARED (default) or SIP_FACES_P2P.  P2P: each side of
                                 an interior face evaluates the flux on its OWN (P+2)-point
                                 face rule, with the other side's two trace scalars (u and
                                 grad u . n) Lagrange-interpolated from that side's own points,
                                 and lifts it on its own rule.  The operator is then symmetric
                                 only where the lower-order side's rule integrates the face
                                 integrand exactly (Sec. 3.3), so P2P handles support sip_apply
                                 (and sip_apply_static_scratch) only: transpose applies, CG
                                 solves and gradients return SIP_ERR_ARG. */
    int32_t quad_rule;        /* SIP_RULE_GAUSS (default) or SIP_RULE_GLL: the point set of every
                                 volume and face rule (P+2 points per direction) */
    int32_t force_interp;     /* 1: every face goes through the interpolation to its shared rule and
                                 the projection back, also where both sides' rules coincide (the
                                 paper's measurement of the cost of non-conforming faces, Sec. 5.2);
                                 same operator, more work.  Default 0 */
    const int32_t* qorders;   /* NULL (default): P + 2 volume points per direction in every element.
                                 Else host [n_elem]: the points per direction of each element (read
                                 by sip_plan_create / sip_create, not kept).  P + 2 always; with
                                 SIP_RULE_GLL also (P, Q) = (1, 4), (1, 5), (2, 5): elements with the
                                 coefficients of one order and the points of a higher one, such as
                                 the transition layer of Sec. 3.3 (P2Q5 in the paper's counts,
                                 between P4Q5 and P2Q3) and Table 2's P3Q5.  Faces integrate on
                                 max(Q-, Q+) points (shared rule) or each side's own Q (P2P).
                                 Other values: SIP_ERR_ARG */
} sip_options;

typedef struct sip_stats {
    int32_t iterations;       /* CG iterations (all inner iterations for refined mode) */
    int32_t refinements;      /* outer refinement steps (0 for SIP_CG_FP64) */
    int32_t applies_fp64;
    int32_t applies_fp32;
    double  rel_residual;     /* max over RHS of ||b - A_fp64 x|| / ||b|| at exit */
    double  seconds;          /* host wall time of the call */
    int32_t converged;        /* 1 if every RHS met rtol */
    int32_t checkpoints;      /* checkpoints written during the call */
} sip_stats;

/* Counts of the host-side plan (mesh analysis); no GPU needed. */
typedef struct sip_plan_info {
    int32_t dim;
    int64_t n_elem, ndof, nquad;
    int64_t n_faces_interior, n_faces_boundary, n_faces_nonconforming;
    int64_t n_elem_affine;            /* elements whose map is affine (constant Jacobian) */
    int64_t orient_hist[8];           /* interior faces per orientation code of the plus side */
    int64_t order_hist[SIP_MAX_ORDER + 1];
    int64_t trace_points;             /* trace buffer size per right-hand side / 4 values:
                                         sum over faces of the shared face points (P2P: of
                                         the two sides' own points) */
    double  min_h_face, max_tau;
} sip_plan_info;

typedef struct sip_plan sip_plan;     /* host-side mesh analysis */
typedef struct sip_handle sip_handle; /* plan + device tables */

/* Fills *opt with the defaults listed above. */
void sip_options_default(sip_options* opt);

/* Host-only mesh analysis: face pairing by shared vertex sets, orientation of
 * each plus side relative to the minus side (the lower element id), geometric
 * factors at volume and face points, penalties, order buckets.  Copies the
 * mesh; the caller may free it afterwards.  opt may be NULL (defaults).
 * Errors: SIP_ERR_ARG (null pointer, dim, order outside 1..SIP_MAX_ORDER),
 * SIP_ERR_MESH (face shared by more than two elements, non-positive Jacobian
 * at a volume point). */
int  sip_plan_create(const sip_mesh* mesh, const int32_t* orders_host, const sip_options* opt,
                     sip_plan** out);
int  sip_plan_info_get(const sip_plan* plan, sip_plan_info* out);
void sip_plan_destroy(sip_plan* plan);

/* Plan + upload to the current CUDA device.  lambda >= 0 is the Helmholtz
 * coefficient (Sec. 2.2).  kappa defaults to 1.  Synchronises the device once.
 * Errors: as sip_plan_create, plus SIP_ERR_NO_DEVICE, SIP_ERR_CUDA, SIP_ERR_OOM. */
int  sip_create(const sip_mesh* mesh, const int32_t* orders_host, double lambda,
                const sip_options* opt, sip_handle** out);
void sip_destroy(sip_handle* h);

int64_t sip_num_dofs(const sip_handle* h);
int64_t sip_num_quad(const sip_handle* h);
int  sip_dof_offsets(const sip_handle* h, int64_t* out_host /* [n_elem+1] */);
int  sip_quad_offsets(const sip_handle* h, int64_t* out_host /* [n_elem+1] */);
int  sip_get_plan_info(const sip_handle* h, sip_plan_info* out);

/* Coefficients of the operator. lambda >= 0 (SIP_ERR_ARG otherwise).
 * kappa_dev: [nquad] FP64 diffusivity per volume point, copied (also to
 * an FP32 copy for SIP_FP32 applies); NULL resets kappa to 1. */
int  sip_set_lambda(sip_handle* h, double lambda);
int  sip_set_kappa(sip_handle* h, const double* kappa_dev, void* stream);

/* y = A x (a1-a7: volume term by sum factorisation, trace evaluation at the
 * shared face points, SIP flux, lift to both sides without atomics; with
 * face_scheme SIP_FACES_P2P, the point-to-point variant of Sec. 3.3).
 * precision SIP_FP64: x_dev, y_dev are double [nrhs][ndof];
 * SIP_FP32: float [nrhs][ndof] (FP32 arithmetic and accumulation).
 * x and y must not overlap.  nrhs >= 1. */
int  sip_apply(sip_handle* h, int precision, const void* x_dev, void* y_dev, int nrhs, void* stream);

/* y = A x with x and y in HOST memory [nrhs][ndof]: applies as sip_apply on
 * `stream` and returns once y is complete (synchronises the stream).  The
 * end-to-end form of the apply for callers that hold their vectors on the
 * host.  A vector in page-locked memory mapped into the device's address
 * space (cudaHostAlloc, cudaHostRegister; the whole vector in one allocation)
 * is read or written in place by the kernels over the host link; a pageable one
 * is copied through a device buffer owned by the handle (grown to the largest
 * nrhs used, freed with the handle).  Errors as sip_apply, plus SIP_ERR_OOM for
 * the buffers. */
int  sip_apply_host(sip_handle* h, int precision, const void* x_host, void* y_host, int nrhs, void* stream);

/* y = A^T x with the roles of trial side (trace evaluation) and test side
 * (lift) exchanged in the face terms (Appendix A: A^T has blocks M'_C <-> M_C^T).
 * For this operator A^T = A, so the result equals sip_apply up to rounding.
 * SIP_FACES_P2P handles: SIP_ERR_ARG. */
int  sip_apply_transpose(sip_handle* h, int precision, const void* x_dev, void* y_dev, int nrhs,
                         void* stream);

/* Solves A x = b by conjugate gradients (Sec. 2.2: the symmetric system is
 * solved by CG), x0 = 0, to ||b - A x|| <= rtol ||b|| in the FP64 operator for
 * every RHS.  mode SIP_CG_FP64: FP64 CG.  mode SIP_CG_FP32_REFINED: outer FP64
 * residual r = b - A x and update x += d, inner CG on A d = r with FP32
 * applies and FP32 vectors, FP64 dot products, to inner_rtol.
 * b_dev, x_dev: double [nrhs][ndof].  Dots are deterministic (fixed-order
 * reductions), so repeated calls give bit-identical x.  stats may be NULL.
 * Synchronises the stream every check_every iterations (convergence test).
 * Errors: SIP_ERR_NOT_CONVERGED, SIP_ERR_BREAKDOWN, SIP_ERR_NONFINITE. */
int  sip_cg_solve(sip_handle* h, int mode, const double* b_dev, double* x_dev, int nrhs,
                  double rtol, sip_stats* stats, void* stream);

/* Solves A^T x = b with the transpose apply (adjoint solve); same contract.
 * Both solves, and sip_cg_replay, need the symmetric operator: SIP_FACES_P2P
 * handles return SIP_ERR_ARG. */
int  sip_cg_solve_transpose(sip_handle* h, int mode, const double* b_dev, double* x_dev, int nrhs,
                            double rtol, sip_stats* stats, void* stream);

/* Checkpoints of the most recent solve (options.checkpoint_every > 0): every
 * checkpoint_every iterations of the running CG recurrence, for any nrhs, the
 * solver copies its state into a ring of checkpoint_slots entries (device
 * memory owned by the handle, grown to nrhs * ndof * 3 doubles per entry):
 * FP64 CG: x, r, p (FP64) and the per-RHS scalars; SIP_CG_FP32_REFINED: the FP64
 * iterate and the FP32 recurrence's r, p and scalars (taken at the graph-chunk
 * boundaries, checkpoint_every rounded up to whole check_every chunks; the FP64
 * CG that may finish such a solve checkpoints as FP64 CG).  The adjoint solve
 * of the backward pass needs none of them (it uses the converged u); they let a
 * caller resume or audit a solve.
 * sip_cg_checkpoint_count: entries kept (the oldest is slot 0). */
int  sip_cg_checkpoint_count(const sip_handle* h);

typedef struct sip_checkpoint_info {
    int32_t iteration;    /* iterations of the recurrence done when it was taken */
    int32_t refinements;  /* outer refinements done (FP32-refined recurrence) */
    int32_t restarts;     /* residual replacements done (FP64 recurrence) */
    int32_t mode;         /* SIP_CG_FP64 or SIP_CG_FP32_REFINED: which recurrence */
    int32_t nrhs;
    int32_t transpose;    /* 1: taken in sip_cg_solve_transpose */
} sip_checkpoint_info;
int  sip_cg_checkpoint_info(const sip_handle* h, int slot, sip_checkpoint_info* out);

/* The checkpoint's FP64 iterate into x_dev (double [nrhs][ndof]), on stream. */
int  sip_cg_checkpoint_iterate(sip_handle* h, int slot, double* x_dev, void* stream);

/* Continues the recurrence of checkpoint `slot` for `iters` iterations exactly
 * as the solve ran it (same kernels, graph chunks and, for FP64 CG, the same
 * per-RHS convergence masking between chunks; no residual replacement or
 * refinement) and writes the resulting FP64 iterate into x_dev [nrhs][ndof].
 * Where the solve did no replacement or refinement in those iterations, the
 * result equals the later checkpoint's iterate bit for bit.  Uses the handle's
 * solver workspace (not the ring) and synchronises the stream.
 * Errors: SIP_ERR_ARG (slot out of range, iters < 0, SIP_FACES_P2P handle). */
int  sip_cg_checkpoint_replay(sip_handle* h, int slot, int iters, double* x_dev, void* stream);

/* FP64 single-RHS checkpoints only: copy-out of slot i into caller device
 * buffers x, r, p [ndof] plus host scalars rr and k (SIP_ERR_ARG for others). */
int  sip_cg_checkpoint_get(sip_handle* h, int slot, double* x_dev, double* r_dev, double* p_dev,
                           double* rr_host, int* iter_host, void* stream);
/* Runs `iters` FP64 CG iterations starting from a state (x, r, p, rr) and
 * writes the resulting state back in place (replay from a checkpoint). */
int  sip_cg_replay(sip_handle* h, double* x_dev, double* r_dev, double* p_dev, double* rr_host,
                   int iters, void* stream);

/* kbar[q] (+)= w_q |J_q| grad ybar_h(x_q) . grad x_h(x_q) per volume Gauss
 * point: d(ybar^T A(kappa) x)/d kappa_q.  ybar, x: double [ndof];
 * kbar: double [nquad]; accumulate != 0 adds to kbar. */
int  sip_grad_kappa(sip_handle* h, const double* ybar_dev, const double* x_dev, double* kbar_dev,
                    int accumulate, void* stream);

/* *out_dev = a^T M b with the (P+2)-point volume rule: d(a^T A(lambda) b)/d lambda. */
int  sip_mass_dot(sip_handle* h, const double* a_dev, const double* b_dev, double* out_dev,
                  void* stream);

/* b_i = sum_q w_q |J_q| phi_i(x_q) f_q (IProduct, Eq. iproduct). f: double [nquad]. */
int  sip_iproduct(sip_handle* h, const double* f_dev, double* b_dev, void* stream);

/* Physical coordinates of the volume points: double [nquad][dim]. */
int  sip_quad_points(sip_handle* h, double* xq_dev, void* stream);

/* Algorithmic work of one apply (per RHS) under the library's work model:
 * flops of the trace kernel and of the main kernel, and the minimum DRAM bytes
 * (x read, y written, geometry and face data read, traces written and read). */
typedef struct sip_work {
    double flops_trace, flops_main;
    double bytes_x, bytes_y, bytes_geometry, bytes_trace;
} sip_work;
int  sip_work_model(const sip_handle* h, int precision, sip_work* out);

/* Launch schedule.  Elements are grouped in tiles of one order (at most a set
 * number of elements per tile for each order) and each CTA runs a list of tiles
 * of one order.  The schedule is balanced for (CTAs per SM) x SMs CTAs resident
 * at once, using per-element flop counts (sip_work_model's):
 *  - one tile per CTA: where the tile sizes give fewer tiles than that, tiles are
 *    split further so that there are about that many, each with the same share
 *    of the apply's flops: one wave of equal CTAs keeps every SM busy to the end
 *    of the launch whichever SM each CTA lands on; more tiles run in waves that
 *    the hardware balances;
 *  - persistent: exactly that many CTAs (about), each with an equal share of the
 *    flops cut into tiles that it runs one after the other, the order's tables
 *    loaded once.
 *
 * Autotuner: coordinate descent over the orders present, timing the whole
 * apply (best of three batches of reps launches) for a few candidate tile sizes
 * of one order at a time, then over the threads per CTA and the CTAs per SM in
 * the three modes (one tile per CTA, persistent, single launch); installs the
 * fastest for this precision.  Set-up call: allocates temporaries and
 * synchronises the stream.  The paper picks a kernel configuration per order
 * (Sec. 5.1); this chooses it by measurement on the current GPU. */
int  sip_autotune(sip_handle* h, int precision, int reps, void* stream);

/* A launch schedule of the apply kernels. */
typedef struct sip_tiling {
    int32_t epb[SIP_MAX_ORDER + 1]; /* elements per tile, at most, for order P, P = 0..SIP_MAX_ORDER
                                       (set: 0 = the default for the order, at most 32;
                                       get: the value in use, 0 where the order is absent) */
    int32_t ctas_per_sm;            /* resident CTAs per SM balanced for (set: 0 = as many as
                                       fit, at most the tiles per SM that epb gives; larger
                                       values are capped at the occupancy) */
    int32_t persistent;             /* 1: each CTA runs several tiles; 2: also the whole apply in ONE
                                       cooperative launch (all CTAs resident: trace phase, grid-wide
                                       barrier, main phase; the barrier's waits are bounded and a wait
                                       that gives up is reported by the solver as SIP_ERR_CUDA), used
                                       while CTAs x nrhs fit on the device (and the device accepts the
                                       cooperative launch), else the two kernels */
    int32_t threads;                /* threads per CTA: 32, 64, 128 or 256 (set: 0 = 256) */
    int32_t cta_layout;             /* block order of the CTAs (set: 0 = SIP_CTAS_SEQUENTIAL):
                                       SIP_CTAS_SEQUENTIAL: block b runs the b-th CTA of the
                                       order-sorted list; SIP_CTAS_SM_MAJOR: blocks b, b + S,
                                       b + 2S, ... (S = the SM count), which the hardware places
                                       on one SM in its first wave, run consecutive CTAs of that
                                       list, so that an SM runs mostly one (N, Q) specialisation.
                                       Either way the results are bit-identical. */
    int64_t ntiles, nctas;          /* get only: tiles and CTAs per right-hand side */
} sip_tiling;

#define SIP_CTAS_SM_MAJOR   1
#define SIP_CTAS_SEQUENTIAL 2

/* Current schedule of one precision. */
int  sip_get_tiling(const sip_handle* h, int precision, sip_tiling* out);

/* Install a schedule by hand (t = NULL: all defaults); ntiles and nctas are
 * ignored.  Set-up call: synchronises the device.  Errors: SIP_ERR_ARG for an
 * out-of-range value or a tile too large for shared memory (the previous
 * schedule stays). */
int  sip_set_tiling(sip_handle* h, int precision, const sip_tiling* t);

/* Device time of the last apply's kernels, per phase, measured with CUDA events
 * on the apply's stream when timing is enabled (sip_set_timing(h, 1)); ms. */
int  sip_set_timing(sip_handle* h, int enable);
int  sip_last_kernel_ms(sip_handle* h, float* trace_ms, float* main_ms);

/* y = A x like sip_apply, but allocating nothing: the trace scratch is a
 * file-scope device array of 16 MiB (SIP_STATIC_TRACE_BYTES) that every GPU
 * loading the library holds until the process exits.  For callers that must
 * not allocate device memory once running (e.g. a process whose device memory
 * is fully reserved by its own caching allocator, or a latency-critical loop
 * where cudaMalloc and its implicit synchronisation are not allowed); the
 * handle itself is still created (and allocated) by sip_create beforehand.
 * The paper has no counterpart; this is an interface variant, not part of the
 * method.
 * - Needs the apply's scratch to fit: nrhs * (4 * trace_points + nquad)
 *   doubles in SIP_FP64; in SIP_FP32 nrhs * (4 * trace_points + nquad) floats
 *   on quads and nrhs * 4 * trace_points floats on hexes (plus 256-byte
 *   alignment), at most SIP_STATIC_TRACE_BYTES (trace_points and nquad from
 *   sip_get_plan_info); larger requests return SIP_ERR_ARG without launching
 *   anything.
 * - The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 * - All calls on all handles of a device share the one array and it keeps the
 *   last call's contents (nothing in it needs clearing: every entry read is
 *   written earlier in the same call).  Calls whose kernels overlap on the GPU
 *   (different streams, or different host threads) race on it: serialise them.
 * Arguments, layout and other errors as sip_apply; the handle must belong to the
 * current device. */
#define SIP_STATIC_TRACE_BYTES (16u << 20)
int  sip_apply_static_scratch(sip_handle* h, int precision, const void* x_dev, void* y_dev, int nrhs,
                              void* stream);

/* Measured arithmetic peak of the current device's FP64 (precision SIP_FP64) or
 * FP32 (SIP_FP32) units in TFLOP/s: 8 independent FMA chains of `iters` steps in
 * every thread of as many 256-thread CTAs as fit on the device at once, timed
 * with CUDA events on `stream` (best of three launches after one warm-up; an
 * FMA counts 2 flops).  The denominator of the apply's roofline: the paper
 * states its CPU efficiency against the machine's peak (Sec. 5.2), this measures
 * the GPU's.  Allocates a small device buffer and synchronises the stream.
 * Errors: SIP_ERR_ARG (null output, iters < 1, precision), SIP_ERR_CUDA. */
int  sip_fp_peak(int precision, int iters, void* stream, double* tflops_out);

const char* sip_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SIP_H */
