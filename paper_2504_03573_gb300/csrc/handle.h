// sip_handle internals (host side).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "sip_internal.h"

namespace sip {

template <typename T>
struct DevGeom {
  T* vgeo = nullptr;
  T* fgeo = nullptr;
  T* tau = nullptr;
  T* kappa = nullptr;
};

// One checkpoint of a CG recurrence: everything needed to continue it bit for
// bit.  FP64 CG: x, r, p in FP64.  FP32-apply CG in FP64 refinement: the FP64
// iterate x and the FP32 recurrence vectors r, p.  Vectors [nrhs][ndof].
struct Checkpoint {
  void* x = nullptr;
  void* r = nullptr;
  void* p = nullptr;
  size_t cap = 0;              // bytes allocated for each of x, r, p
  std::vector<double> scal;    // the recurrence's per-RHS scalars
  std::vector<double> tol;     // per-RHS stopping tolerance of the recurrence
  int iter = 0;                // CG iterations done when it was taken
  int refinements = 0;         // outer refinements done (FP32-refined mode)
  int restarts = 0;            // residual replacements done (FP64 mode)
  int mode = 0;                // SIP_CG_FP64 or SIP_CG_FP32_REFINED (the recurrence's kind)
  int nrhs = 0;
  int transpose = 0;
};

// CG workspace for one (vector type, nrhs) configuration
struct CgWork {
  int nrhs = 0;
  size_t elem = 0;          // bytes per vector element (8 or 4)
  void* x = nullptr;        // iterate (internal, so captured graphs stay valid)
  void* r = nullptr;
  void* p = nullptr;
  void* ap = nullptr;
  double* scal = nullptr;   // per RHS: rr, pap, alpha, beta, rr_new, active, scratch...
  double* partial = nullptr;
  int* status = nullptr;    // device status word (breakdown / non-finite)
  void* xext = nullptr;     // FP64 iterate updated instead of x (mixed-precision CG)
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0;
  int graph_transpose = -1;
  void* graph_xext = nullptr;
  void release();
};

}  // namespace sip

struct sip_handle {
  sip::Plan plan;
  int device = 0;
  double lambda = 1.0;
  bool kappa_set = false;
  // device tables
  int64_t* dof_off = nullptr;
  int64_t* quad_off = nullptr;
  int64_t* vgoff = nullptr;
  int64_t* f_troff = nullptr;
  int64_t* f_goff = nullptr;
  sip::FaceSlot* slots = nullptr;
  int32_t* elist = nullptr;
  int8_t* eaff = nullptr;
  sip::ElemDesc* desc_e = nullptr;   // element / slot descriptors in elist order
  sip::SlotDesc* desc_s = nullptr;
  sip::Tile* tiles_d[2] = {nullptr, nullptr};   // per precision (FP64, FP32)
  std::vector<sip::Tile> tiles_h[2];
  int32_t* cta_d[2] = {nullptr, nullptr};       // CTA b runs tiles cta_off[b] .. cta_off[b+1]-1
  uint16_t* flist_d[2] = {nullptr, nullptr};    // face lists of the tiles
  std::vector<int32_t> cta_h[2];
  int epb[2][sip::kNMax + 2] = {};                // elements per tile per order in use (0: default)
  int ctas_per_sm[2] = {0, 0};                    // resident CTAs per SM the schedule is balanced for
  int persistent[2] = {0, 0};                     // CTAs run several tiles each
  int fused_cap[2] = {0, 0};                      // > 0: single cooperative launch per apply while
                                                  // CTAs x nrhs <= fused_cap (resident at once)
  unsigned int* gbar = nullptr;                   // grid barrier words of the single-launch apply
  // the rule's tables and weights in global memory (per device, kept for the process)
  const double* gtab_d = nullptr;
  const float* gtab_f = nullptr;
  const double* ggw_d = nullptr;
  const float* ggw_f = nullptr;
  int threads[2] = {256, 256};                    // threads per CTA
  int cta_layout[2] = {SIP_CTAS_SEQUENTIAL, SIP_CTAS_SEQUENTIAL};  // block order of the CTAs
  double* xq = nullptr;
  // point-to-point interpolation matrices between Gauss rules (SIP_FACES_P2P only)
  double* p2p_I_d = nullptr;
  float* p2p_I_f = nullptr;
  sip::DevGeom<double> gd;
  sip::DevGeom<float> gf;
  template <typename T>
  const sip::DevGeom<T>& geom() const;
  template <typename T>
  const T* p2p_interp() const;
  bool p2p() const { return plan.opt.face_scheme == SIP_FACES_P2P; }
  // scratch (sized for the largest nrhs seen, in doubles): trace buffer and, for
  // FP64 applies, the Gauss-point values handed from the trace to the main kernel
  double* trace_d = nullptr;
  size_t trace_cap = 0;
  double* ug_d = nullptr;
  size_t ug_cap = 0;
  // device copies of host vectors for sip_apply_host (x, y; bytes each)
  void* io_x = nullptr;
  void* io_y = nullptr;
  size_t io_cap = 0;
  size_t smem_trace[2] = {0, 0};
  size_t smem_main[2] = {0, 0};
  // timing
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool timing = false;
  bool timed_pending = false;
  // solver state
  cudaStream_t solve_stream = nullptr;
  sip::CgWork cg64, cg32;
  double* r64 = nullptr;     // outer residual / true residual workspace [nrhs][ndof]
  double* x64 = nullptr;     // outer iterate
  double* xbak = nullptr;    // outer iterate at the last refinement (mixed-precision CG)
  double* red = nullptr;     // reduction partials for aux kernels
  double* scal_host = nullptr;
  int work_nrhs = 0;
  // checkpoints of the last solve (a ring of checkpoint_slots entries)
  std::vector<sip::Checkpoint> ck;
  int ck_count = 0, ck_next = 0;
  void release();
};

template <>
inline const sip::DevGeom<double>& sip_handle::geom<double>() const { return gd; }
template <>
inline const sip::DevGeom<float>& sip_handle::geom<float>() const { return gf; }
template <>
inline const double* sip_handle::p2p_interp<double>() const { return p2p_I_d; }
template <>
inline const float* sip_handle::p2p_interp<float>() const { return p2p_I_f; }

namespace sip {
// NVTX range for the lifetime of the object: the library's entry points mark
// themselves (sip_apply, sip_cg_solve, refinement steps, sip_autotune) so that
// profilers can select them; without an attached tool this costs a branch.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
// Tiles of one precision and the CTA that runs each, with the shared memory of
// the two kernels.  per_sm: resident CTAs per SM the CTAs were balanced for.
struct Schedule {
  std::vector<Tile> tiles;
  std::vector<int32_t> cta_off;
  std::vector<uint16_t> flists;
  size_t smem_t = 0, smem_m = 0;
  int per_sm = 0;
  bool persistent = false;
  int fused_cap = 0;  // > 0: one cooperative launch per apply (persistent CTAs), up to this many CTAs
  int threads = 256;
  int layout = SIP_CTAS_SEQUENTIAL;
  int nctas() const { return (int)cta_off.size() - 1; }
};
// epb: elements per tile by order (nullptr or 0 entries: default); ctas_per_sm <= 0:
// as many as fit, capped at the number of default-sized tiles per SM; mode 1
// (persistent): per_sm x SMs CTAs with several tiles each (build_tiles); mode 2:
// persistent CTAs all resident at once, the apply one cooperative launch;
// layout: SIP_CTAS_SM_MAJOR or SIP_CTAS_SEQUENTIAL (the block order of the CTAs)
int make_schedule(const sip_handle* h, int precision, const int* epb, int ctas_per_sm, int mode, int threads,
                  int layout, Schedule& s);
// device copy of a schedule
struct DevSchedule {
  Tile* tiles = nullptr;
  int32_t* cta = nullptr;
  uint16_t* flist = nullptr;
};
cudaError_t upload_schedule(const Schedule& sc, DevSchedule& d);
void free_schedule(DevSchedule& d);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);
// scratch_override: caller-provided scratch holding the trace buffer followed by
// (FP64) the Gauss-point buffer, laid out as apply_scratch_bytes() describes.
int apply_any(sip_handle* h, int precision, const void* x, void* y, int nrhs, cudaStream_t s,
              int transpose, void* scratch_override);
size_t apply_scratch_bytes(const sip_handle* h, int precision, int nrhs, size_t* ug_offset);
int apply_tiles(sip_handle* h, int precision, const Tile* tiles_d, const int32_t* cta_d, const uint16_t* flist_d,
                int nctas, int threads, size_t smem_t, size_t smem_m, int fused_cap, const void* x, void* y, int nrhs,
                cudaStream_t s, int transpose, void* scratch_override);
int set_tiles(sip_handle* h, int precision, const int* epb_by_n, int ctas_per_sm, int mode, int threads,
              int layout);
int handle_grow_trace(sip_handle* h, int nrhs);
}  // namespace sip
