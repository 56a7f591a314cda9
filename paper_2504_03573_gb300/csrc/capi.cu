// C ABI: plan, handle life cycle, apply, queries.  Solver and gradient entry
// points live in solver.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "handle.h"

namespace sip {

thread_local std::string g_err;
thread_local int g_fused_fallbacks = 0;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SIP_ERR_OOM : SIP_ERR_CUDA;
}

// Elements per tile: enough work items per CTA to keep its threads busy in every
// stage (Gauss points in 2D, lines of Gauss points in 3D), within 64 KB of
// shared memory.
int apply_epb(int dim, int n, int q, int precision, int threads) {
  // one Gauss point per work item (2D; FP64 in 3D) or one line of Q points (FP32 in 3D)
  const bool lines = dim == 3 && precision == SIP_FP32;
  const int items = lines ? q * q : (dim == 2 ? q * q : q * q * q);
  int epb = std::max(1, (dim == 3 && !lines ? 3 * threads / 2 : threads) / items);
  const int es = precision == SIP_FP32 ? 4 : 8;
  const int per = std::max(per_elem_trace(dim, n, q), per_elem_main(dim, n, q)) * es;
  const int room = (64 * 1024 - table_block_bytes(es, n, q) - kMetaBytes) / per;
  return std::max(1, std::min(std::min(epb, room), kMaxEpb));
}

// Per (point rule, dimension, precision) translation unit: table upload, kernel
// attributes, occupancy and the apply launch (apply_[gll_]{2d,3d}_{f64,f32}.cu).
#define SIP_DECLARE_APPLY_TU(SUFFIX, TYPE)                                                            \
  cudaError_t upload_tables_##SUFFIX(const double*, const float*, const int*, const double*, const float*); \
  cudaError_t prepare_##SUFFIX();                                                                      \
  cudaError_t occupancy_##SUFFIX(int, size_t, size_t, int*);                                           \
  cudaError_t occupancy_fused_##SUFFIX(int, size_t, int*);                                             \
  cudaError_t launch_apply_##SUFFIX(const ApplyArgs<TYPE>&, int, int, int, size_t, size_t, cudaStream_t, \
                                    cudaEvent_t, cudaEvent_t, cudaEvent_t, bool);
SIP_DECLARE_APPLY_TU(2d_f64, double)
SIP_DECLARE_APPLY_TU(2d_f32, float)
SIP_DECLARE_APPLY_TU(3d_f64, double)
SIP_DECLARE_APPLY_TU(3d_f32, float)
SIP_DECLARE_APPLY_TU(gll_2d_f64, double)
SIP_DECLARE_APPLY_TU(gll_2d_f32, float)
SIP_DECLARE_APPLY_TU(gll_3d_f64, double)
SIP_DECLARE_APPLY_TU(gll_3d_f32, float)
#undef SIP_DECLARE_APPLY_TU
cudaError_t prepare_aux_2d();
cudaError_t prepare_aux_3d();
cudaError_t prepare_aux_gll_2d();
cudaError_t prepare_aux_gll_3d();

// the unit of (rule, dim, precision): index [rule][dim - 2][precision]
using UploadFn = cudaError_t (*)(const double*, const float*, const int*, const double*, const float*);
using PrepareFn = cudaError_t (*)();
using OccupancyFn = cudaError_t (*)(int, size_t, size_t, int*);
static const UploadFn kUpload[2][2][2] = {{{upload_tables_2d_f64, upload_tables_2d_f32}, {upload_tables_3d_f64, upload_tables_3d_f32}},
                                          {{upload_tables_gll_2d_f64, upload_tables_gll_2d_f32},
                                           {upload_tables_gll_3d_f64, upload_tables_gll_3d_f32}}};
static const PrepareFn kPrepare[2][2][2] = {{{prepare_2d_f64, prepare_2d_f32}, {prepare_3d_f64, prepare_3d_f32}},
                                            {{prepare_gll_2d_f64, prepare_gll_2d_f32}, {prepare_gll_3d_f64, prepare_gll_3d_f32}}};
using OccupancyFusedFn = cudaError_t (*)(int, size_t, int*);
static const OccupancyFusedFn kOccupancyFused[2][2][2] = {
    {{occupancy_fused_2d_f64, occupancy_fused_2d_f32}, {occupancy_fused_3d_f64, occupancy_fused_3d_f32}},
    {{occupancy_fused_gll_2d_f64, occupancy_fused_gll_2d_f32}, {occupancy_fused_gll_3d_f64, occupancy_fused_gll_3d_f32}}};
static const OccupancyFn kOccupancy[2][2][2] = {
    {{occupancy_2d_f64, occupancy_2d_f32}, {occupancy_3d_f64, occupancy_3d_f32}},
    {{occupancy_gll_2d_f64, occupancy_gll_2d_f32}, {occupancy_gll_3d_f64, occupancy_gll_3d_f32}}};

static cudaError_t launch_apply(int rule, int dim, const ApplyArgs<double>& a, int nctas, int nrhs, int threads,
                                size_t st, size_t sm, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, cudaEvent_t e2,
                                bool fused) {
  if (rule == SIP_RULE_GLL)
    return dim == 2 ? launch_apply_gll_2d_f64(a, nctas, nrhs, threads, st, sm, s, e0, e1, e2, fused)
                    : launch_apply_gll_3d_f64(a, nctas, nrhs, threads, st, sm, s, e0, e1, e2, fused);
  return dim == 2 ? launch_apply_2d_f64(a, nctas, nrhs, threads, st, sm, s, e0, e1, e2, fused)
                  : launch_apply_3d_f64(a, nctas, nrhs, threads, st, sm, s, e0, e1, e2, fused);
}
static cudaError_t launch_apply(int rule, int dim, const ApplyArgs<float>& a, int nctas, int nrhs, int threads,
                                size_t st, size_t sm, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, cudaEvent_t e2,
                                bool fused) {
  if (rule == SIP_RULE_GLL)
    return dim == 2 ? launch_apply_gll_2d_f32(a, nctas, nrhs, threads, st, sm, s, e0, e1, e2, fused)
                    : launch_apply_gll_3d_f32(a, nctas, nrhs, threads, st, sm, s, e0, e1, e2, fused);
  return dim == 2 ? launch_apply_2d_f32(a, nctas, nrhs, threads, st, sm, s, e0, e1, e2, fused)
                  : launch_apply_3d_f32(a, nctas, nrhs, threads, st, sm, s, e0, e1, e2, fused);
}

namespace {

constexpr int kMaxDevices = 64;
bool g_tables_uploaded[kMaxDevices] = {false};
// per device and rule: the tables and weights in global memory, the source of
// the kernels' per-CTA table copies (coalesced reads); allocated once, kept for
// the process
struct GlobalTables {
  double* tab_d = nullptr;
  float* tab_f = nullptr;
  double* gw_d = nullptr;
  float* gw_f = nullptr;
};
GlobalTables g_tables[kMaxDevices][2];

template <typename T>
cudaError_t upload(T** dst, const void* src, size_t bytes) {
  cudaError_t e = cudaMalloc((void**)dst, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) return e;
  if (bytes) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  return e;
}

template <typename T>
std::vector<float> to_float(const std::vector<T>& v) {
  std::vector<float> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (float)v[i];
  return o;
}

int ensure_tables(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return fail(SIP_ERR_CUDA, "device index out of range");
  if (g_tables_uploaded[dev]) return SIP_OK;
  cudaError_t e;
  for (int rule : {SIP_RULE_GAUSS, SIP_RULE_GLL}) {
    std::vector<double> tab;
    fill_tables(rule, tab);
    std::vector<float> tabf = to_float(tab);
    int ioff[kQMax + 1][kQMax + 1];
    for (int q = 0; q <= kQMax; ++q)
      for (int f = 0; f <= kQMax; ++f) ioff[q][f] = (q >= kQMin && f >= q) ? tab_I(q, f) : 0;
    double gwd[kQMax + 1][kQMax] = {};
    float gwf[kQMax + 1][kQMax] = {};
    for (int q = 2; q <= kQMax; ++q) {
      std::vector<double> gx, gw;
      point_rule(rule, q, gx, gw);
      for (int z = 0; z < q; ++z) { gwd[q][z] = gw[z]; gwf[q][z] = (float)gw[z]; }
    }
    for (int d = 0; d < 2; ++d)
      for (int pr = 0; pr < 2; ++pr)
        if ((e = kUpload[rule][d][pr](tab.data(), tabf.data(), &ioff[0][0], &gwd[0][0], &gwf[0][0])) != cudaSuccess)
          return cuda_fail(e, "tables");
    GlobalTables& gt = g_tables[dev][rule];
    const size_t ngw = (size_t)(kQMax + 1) * kQMax;
    if ((e = upload(&gt.tab_d, tab.data(), tab.size() * sizeof(double))) != cudaSuccess ||
        (e = upload(&gt.tab_f, tabf.data(), tabf.size() * sizeof(float))) != cudaSuccess ||
        (e = upload(&gt.gw_d, &gwd[0][0], ngw * sizeof(double))) != cudaSuccess ||
        (e = upload(&gt.gw_f, &gwf[0][0], ngw * sizeof(float))) != cudaSuccess)
      return cuda_fail(e, "tables");
  }
  // dynamic shared-memory limits, set once per device (never during a stream capture)
  for (int rule = 0; rule < 2; ++rule)
    for (int d = 0; d < 2; ++d)
      for (int pr = 0; pr < 2; ++pr)
        if ((e = kPrepare[rule][d][pr]()) != cudaSuccess) return cuda_fail(e, "kernel attributes");
  for (auto fn : {prepare_aux_2d, prepare_aux_3d, prepare_aux_gll_2d, prepare_aux_gll_3d})
    if ((e = fn()) != cudaSuccess) return cuda_fail(e, "kernel attributes");
  g_tables_uploaded[dev] = true;
  return SIP_OK;
}

}  // namespace

int handle_grow_trace(sip_handle* h, int nrhs) {
  const size_t need = (size_t)nrhs * 4 * (size_t)h->plan.trace_points;
  if (need > h->trace_cap) {
    if (h->trace_d) cudaFree(h->trace_d);
    h->trace_d = nullptr;
    h->trace_cap = 0;
    cudaError_t e = cudaMalloc((void**)&h->trace_d, need * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "trace buffer");
    h->trace_cap = need;
  }
  const size_t needu = (size_t)nrhs * (size_t)h->plan.nquad;
  if (needu > h->ug_cap) {
    if (h->ug_d) cudaFree(h->ug_d);
    h->ug_d = nullptr;
    h->ug_cap = 0;
    cudaError_t e = cudaMalloc((void**)&h->ug_d, needu * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "Gauss-point buffer");
    h->ug_cap = needu;
  }
  return SIP_OK;
}

// Whether the main phase takes the volume-point values from the trace phase
// (the hand-off buffer) instead of recomputing them: always in FP64, where the
// recomputation costs FP64 flops, and in FP32 on quads, where it costs two
// barrier-separated stages of kernels that wait on latency; FP32 hexes
// recompute (more values per element, and throughput-bound stages).
bool uses_handoff(const sip_handle* h, int precision) { return precision == SIP_FP64 || h->plan.dim == 2; }

// Scratch of one apply: trace buffer [nrhs][4 trace_points], then (where the
// main phase takes them over) the volume-point values [nrhs][nquad], 256-byte
// aligned.
size_t apply_scratch_bytes(const sip_handle* h, int precision, int nrhs, size_t* ug_offset) {
  const size_t es = precision == SIP_FP64 ? sizeof(double) : sizeof(float);
  const size_t tr = ((size_t)nrhs * 4 * (size_t)h->plan.trace_points * es + 255) / 256 * 256;
  if (ug_offset) *ug_offset = tr;
  return uses_handoff(h, precision) ? tr + (size_t)nrhs * (size_t)h->plan.nquad * es : tr;
}

namespace {

// Block b of the launch runs the CTA that is k-th in the order of the blocks by
// (b mod nsm, b / nsm): the blocks the hardware places on one SM in its first
// wave (b, b + nsm, ...) take consecutive CTAs of the order-sorted list, i.e.
// mostly tiles of one (N, Q), so that an SM's instruction cache holds the code
// of one specialisation rather than of every order at once.  Which block runs a
// tile changes no arithmetic.  (On the 64^2 quads with orders 2..6 this order is
// 10-12 % slower than the sequential one, which stays the default.)
void sm_major_ctas(Schedule& s, int nsm) {
  const int C = s.nctas();
  if (C <= nsm || nsm <= 1) return;
  std::vector<int> blocks(C);
  for (int b = 0; b < C; ++b) blocks[b] = b;
  std::stable_sort(blocks.begin(), blocks.end(), [nsm](int a, int b) {
    return a % nsm != b % nsm ? a % nsm < b % nsm : a / nsm < b / nsm;
  });
  std::vector<int> cta_of(C);
  for (int k = 0; k < C; ++k) cta_of[blocks[k]] = k;
  std::vector<Tile> tiles;
  tiles.reserve(s.tiles.size());
  std::vector<int32_t> off(1, 0);
  for (int b = 0; b < C; ++b) {
    const int k = cta_of[b];
    tiles.insert(tiles.end(), s.tiles.begin() + s.cta_off[k], s.tiles.begin() + s.cta_off[k + 1]);
    off.push_back((int32_t)tiles.size());
  }
  s.tiles = std::move(tiles);
  s.cta_off = std::move(off);
}

}  // namespace

int make_schedule(const sip_handle* h, int precision, const int* epb, int ctas_per_sm, int mode, int threads,
                  int layout, Schedule& s) {
  if (mode < 0 || mode > 2) return fail(SIP_ERR_ARG, "schedule mode must be 0, 1 or 2");
  if (layout != SIP_CTAS_SM_MAJOR && layout != SIP_CTAS_SEQUENTIAL) return fail(SIP_ERR_ARG, "cta_layout");
  s.layout = layout;
  const bool persistent = mode >= 1, fused = mode == 2;
  const Plan& p = h->plan;
  const int es = precision == SIP_FP32 ? 4 : 8;
  // per CTA: its table block (up to the finest face rule of its tiles, as the
  // kernels compute it), the tile meta and its largest tile
  auto size_smem = [&]() {
    s.smem_t = s.smem_m = 0;
    for (size_t c = 0; c + 1 < s.cta_off.size(); ++c) {
      if (s.cta_off[c] == s.cta_off[c + 1]) continue;
      const int n = s.tiles[s.cta_off[c]].n, q = s.tiles[s.cta_off[c]].q;
      int fmax = q, cmax = 1;
      for (int32_t ti = s.cta_off[c]; ti < s.cta_off[c + 1]; ++ti) {
        fmax = std::max(fmax, s.tiles[ti].flags & kTileQfMask);
        cmax = std::max(cmax, (int)s.tiles[ti].count);
      }
      const size_t fixed = (size_t)table_block_bytes(es, n, q, fmax) + meta_bytes(p.dim, cmax);
      for (int32_t ti = s.cta_off[c]; ti < s.cta_off[c + 1]; ++ti) {
        const Tile& t = s.tiles[ti];
        s.smem_t = std::max(s.smem_t, fixed + (size_t)t.count * per_elem_trace(p.dim, t.n, t.q) * es);
        s.smem_m = std::max(s.smem_m, fixed + (size_t)t.count * per_elem_main(p.dim, t.n, t.q) * es +
                                          (precision == SIP_FP64 ? kFaceListBytes : 0));
      }
    }
  };
  // one CTA per tile of the largest size epb allows: the tile count and shared
  // memory bound the rest (a CTA's tiles are never larger)
  if (threads != 32 && threads != 64 && threads != 128 && threads != 256)
    return fail(SIP_ERR_ARG, "threads per CTA must be 32, 64, 128 or 256");
  build_tiles(p, precision, epb, threads, 0, false, s.tiles, s.cta_off, s.flists);
  size_smem();
  s.per_sm = 1;
  s.persistent = persistent;
  s.threads = threads;
  if (s.smem_t > 200 * 1024 || s.smem_m > 200 * 1024) return fail(SIP_ERR_ARG, "tile too large for shared memory");
  const int64_t ntile = (int64_t)s.tiles.size();
  if (ntile == 0) return SIP_OK;
  int occ = 0, nsm = 0;
  cudaError_t e;
  const int pr = precision == SIP_FP64 ? 0 : 1;
  if (fused)  // the single launch holds both phases' shared memory
    e = kOccupancyFused[p.opt.quad_rule][p.dim - 2][pr](threads, std::max(s.smem_t, s.smem_m), &occ);
  else
    e = kOccupancy[p.opt.quad_rule][p.dim - 2][pr](threads, s.smem_t, s.smem_m, &occ);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy");
  occ = std::max(1, occ);
  nsm = std::max(1, nsm);
  // per_sm x SMs CTAs of equal flops, all resident at once
  const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ)
                                     : (int)std::min<int64_t>(occ, std::max<int64_t>(1, ntile / nsm));
  build_tiles(p, precision, epb, threads, nsm * per_sm, persistent, s.tiles, s.cta_off, s.flists);
  size_smem();
  s.per_sm = per_sm;
  s.fused_cap = 0;
  if (fused) {
    int of = 0;
    e = kOccupancyFused[p.opt.quad_rule][p.dim - 2][pr](threads, std::max(s.smem_t, s.smem_m), &of);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    s.fused_cap = std::max(1, of) * nsm;
    // the per-order shares are rounded, so the CTA count can exceed the target
    // by a few: aim lower until every CTA fits at once
    for (int target = nsm * per_sm; s.nctas() > s.fused_cap && target > 1;) {
      target = std::max(1, target - (s.nctas() - s.fused_cap));
      build_tiles(p, precision, epb, threads, target, true, s.tiles, s.cta_off, s.flists);
      size_smem();
    }
    if (s.nctas() > s.fused_cap) return fail(SIP_ERR_ARG, "single-launch schedule larger than the resident CTAs");
  }
  if (layout == SIP_CTAS_SM_MAJOR) sm_major_ctas(s, nsm);
  return SIP_OK;
}

cudaError_t upload_schedule(const Schedule& sc, DevSchedule& d) {
  d = DevSchedule{};
  cudaError_t e = cudaMalloc((void**)&d.tiles, std::max<size_t>(16, sc.tiles.size() * sizeof(Tile)));
  if (e == cudaSuccess) e = cudaMalloc((void**)&d.cta, sc.cta_off.size() * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&d.flist, std::max<size_t>(16, sc.flists.size() * sizeof(uint16_t)));
  if (e == cudaSuccess && !sc.tiles.empty())
    e = cudaMemcpy(d.tiles, sc.tiles.data(), sc.tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d.cta, sc.cta_off.data(), sc.cta_off.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !sc.flists.empty())
    e = cudaMemcpy(d.flist, sc.flists.data(), sc.flists.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_schedule(d);
    cudaGetLastError();
  }
  return e;
}

void free_schedule(DevSchedule& d) {
  cudaFree(d.tiles);
  cudaFree(d.cta);
  cudaFree(d.flist);
  d = DevSchedule{};
}

// (Re)build the schedule of one precision (epb_by_n[n] > 0 overrides the default
// elements per tile for order n - 1; ctas_per_sm > 0 fixes the resident CTAs per
// SM it is balanced for), upload it and size the shared memory.
int set_tiles(sip_handle* h, int precision, const int* epb_by_n, int ctas_per_sm, int mode, int threads,
              int layout) {
  const int pi = precision == SIP_FP32 ? 1 : 0;
  Schedule sc;
  int rc = make_schedule(h, precision, epb_by_n, ctas_per_sm, mode, threads, layout, sc);
  if (rc) return rc;
  DevSchedule d;
  cudaError_t e = upload_schedule(sc, d);
  if (e != cudaSuccess) return cuda_fail(e, "tiles");
  if (h->tiles_d[pi] || h->cta_d[pi] || h->flist_d[pi]) {
    cudaDeviceSynchronize();  // earlier launches may still read the old schedule
    cudaFree(h->tiles_d[pi]);
    cudaFree(h->cta_d[pi]);
    cudaFree(h->flist_d[pi]);
  }
  h->tiles_d[pi] = d.tiles;
  h->cta_d[pi] = d.cta;
  h->flist_d[pi] = d.flist;
  h->tiles_h[pi] = std::move(sc.tiles);
  h->cta_h[pi] = std::move(sc.cta_off);
  h->ctas_per_sm[pi] = sc.per_sm;
  h->persistent[pi] = sc.persistent ? 1 : 0;
  h->fused_cap[pi] = sc.fused_cap;
  h->threads[pi] = sc.threads;
  h->cta_layout[pi] = sc.layout;
  h->smem_trace[pi] = sc.smem_t;
  h->smem_main[pi] = sc.smem_m;
  for (auto* W : {&h->cg64, &h->cg32})
    if (W->graph) { cudaGraphExecDestroy(W->graph); W->graph = nullptr; }
  return SIP_OK;
}

template <typename T>
ApplyArgs<T> make_args(sip_handle* h, const T* x, T* y, T* trace, T* ug, int transpose) {
  ApplyArgs<T> a;
  const DevGeom<T>& g = h->geom<T>();
  a.dof_off = h->dof_off;
  a.vgoff = h->vgoff;
  a.vgeo = g.vgeo;
  a.quad_off = h->quad_off;
  a.kappa = h->kappa_set ? g.kappa : nullptr;
  a.slots = h->slots;
  a.f_troff = h->f_troff;
  a.f_goff = h->f_goff;
  a.f_tau = g.tau;
  a.fgeo = g.fgeo;
  a.elist = h->elist;
  a.eaff = h->eaff;
  a.desc_e = h->desc_e;
  a.desc_s = h->desc_s;
  a.tiles = h->tiles_d[std::is_same<T, float>::value ? 1 : 0];
  a.cta_off = h->cta_d[std::is_same<T, float>::value ? 1 : 0];
  a.flists = h->flist_d[std::is_same<T, float>::value ? 1 : 0];
  a.x = x;
  a.y = y;
  a.trace = trace;
  a.ug = ug;
  a.ndof = h->plan.ndof;
  a.nquad = h->plan.nquad;
  a.trace_stride = 4 * h->plan.trace_points;
  a.lambda = (T)h->lambda;
  a.transpose = transpose;
  a.p2p_I = h->p2p_interp<T>();
  a.gbar = h->gbar;
  if constexpr (std::is_same<T, double>::value) {
    a.gtab = h->gtab_d;
    a.ggw = h->ggw_d;
  } else {
    a.gtab = h->gtab_f;
    a.ggw = h->ggw_f;
  }
  return a;
}

int apply_tiles(sip_handle* h, int precision, const Tile* tiles_d, const int32_t* cta_d, const uint16_t* flist_d,
                int nctas, int threads, size_t smem_t, size_t smem_m, int fused_cap, const void* x, void* y, int nrhs,
                cudaStream_t s, int transpose, void* scratch_override) {
  // one cooperative launch where the schedule allows it and every CTA of all
  // right-hand sides fits on the device at once; otherwise the two kernels
  const bool fused = fused_cap > 0 && (int64_t)nctas * nrhs <= fused_cap;
  size_t ug_off = 0;
  apply_scratch_bytes(h, precision, nrhs, &ug_off);
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  if (h->timing) { e0 = h->ev[0]; e1 = h->ev[1]; e2 = h->ev[2]; }
  cudaError_t e;
  if (precision == SIP_FP64) {
    double* tr = scratch_override ? (double*)scratch_override : h->trace_d;
    double* ug = scratch_override ? (double*)((char*)scratch_override + ug_off) : h->ug_d;
    auto a = make_args<double>(h, (const double*)x, (double*)y, tr, ug, transpose);
    a.tiles = tiles_d;
    a.cta_off = cta_d;
    a.flists = flist_d;
    e = launch_apply(h->plan.opt.quad_rule, h->plan.dim, a, nctas, nrhs, threads, smem_t, smem_m, s, e0, e1, e2, fused);
  } else {
    float* tr = scratch_override ? (float*)scratch_override : (float*)h->trace_d;
    float* ug = !uses_handoff(h, precision) ? nullptr
                : scratch_override ? (float*)((char*)scratch_override + ug_off) : (float*)h->ug_d;
    auto a = make_args<float>(h, (const float*)x, (float*)y, tr, ug, transpose);
    a.tiles = tiles_d;
    a.cta_off = cta_d;
    a.flists = flist_d;
    e = launch_apply(h->plan.opt.quad_rule, h->plan.dim, a, nctas, nrhs, threads, smem_t, smem_m, s, e0, e1, e2, fused);
  }
  if (e != cudaSuccess) return cuda_fail(e, "apply launch");
  h->timed_pending = h->timing;
  return SIP_OK;
}

int apply_any(sip_handle* h, int precision, const void* x, void* y, int nrhs, cudaStream_t s,
              int transpose, void* scratch_override) {
  if (!h || !x || !y) return fail(SIP_ERR_ARG, "null handle or vector");
  if (nrhs < 1) return fail(SIP_ERR_ARG, "nrhs must be >= 1");
  if (precision != SIP_FP64 && precision != SIP_FP32) return fail(SIP_ERR_ARG, "precision");
  if (transpose && h->p2p())
    return fail(SIP_ERR_ARG, "the transpose apply needs the shared-rule operator (face_scheme SIP_FACES_SHARED)");
  if (!scratch_override) {
    int rc = handle_grow_trace(h, nrhs);
    if (rc) return rc;
  }
  const int pi = precision == SIP_FP32 ? 1 : 0;
  return apply_tiles(h, precision, h->tiles_d[pi], h->cta_d[pi], h->flist_d[pi], (int)h->cta_h[pi].size() - 1,
                     h->threads[pi], h->smem_trace[pi], h->smem_main[pi], h->fused_cap[pi], x, y, nrhs, s, transpose,
                     scratch_override);
}

}  // namespace sip

using namespace sip;

namespace {

// The address under which the current device reaches the host range [p, p +
// bytes) directly, or nullptr: page-locked memory mapped into the device's
// address space (cudaHostAlloc, cudaHostRegister), the whole range inside one
// such allocation.  Pageable memory gives nullptr.
void* mapped_host_range(const void* p, size_t bytes) {
  cudaPointerAttributes a0{}, a1{};
  if (cudaPointerGetAttributes(&a0, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a0.type != cudaMemoryTypeHost || a0.devicePointer == nullptr) return nullptr;
  const void* last = static_cast<const char*>(p) + (bytes - 1);
  if (cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a1.type != cudaMemoryTypeHost || a1.devicePointer != static_cast<char*>(a0.devicePointer) + (bytes - 1))
    return nullptr;
  return a0.devicePointer;
}

}  // namespace

extern "C" {

const char* sip_last_error(void) { return g_err.c_str(); }

void sip_options_default(sip_options* o) {
  if (!o) return;
  o->tau_scale = 2.0;
  o->qvol_extra = 2;
  o->boundary = 1;
  o->inner_rtol = 1e-5;
  o->max_iter = 20000;
  o->check_every = 16;
  o->max_refine = 30;
  o->checkpoint_every = 0;
  o->checkpoint_slots = 8;
  o->face_scheme = SIP_FACES_SHARED;
  o->quad_rule = SIP_RULE_GAUSS;
  o->force_interp = 0;
  o->qorders = nullptr;
}

struct sip_plan {
  Plan p;
};

static void fill_info(const Plan& p, sip_plan_info* out) {
  std::memset(out, 0, sizeof(*out));
  out->dim = p.dim;
  out->n_elem = p.E;
  out->ndof = p.ndof;
  out->nquad = p.nquad;
  out->n_faces_interior = p.n_int;
  out->n_faces_boundary = p.n_bnd;
  out->n_faces_nonconforming = p.n_nonconf;
  for (int8_t a : p.affine) out->n_elem_affine += a;
  for (int i = 0; i < 8; ++i) out->orient_hist[i] = p.orient_hist[i];
  for (int32_t o : p.P) out->order_hist[o] += 1;
  out->trace_points = p.trace_points;
  double hmin = 1e300, tmax = 0.0;
  for (size_t f = 0; f < p.f_tau.size(); ++f) {
    const int pm = p.f_ep[f] >= 0 ? std::max(p.P[p.f_em[f]], p.P[p.f_ep[f]]) : p.P[p.f_em[f]];
    const double h = p.opt.tau_scale * (pm + 1.0) * (pm + 1.0) / p.f_tau[f];
    hmin = std::min(hmin, h);
    tmax = std::max(tmax, p.f_tau[f]);
  }
  out->min_h_face = hmin;
  out->max_tau = tmax;
}

int sip_plan_create(const sip_mesh* mesh, const int32_t* orders, const sip_options* opt, sip_plan** out) {
  if (!out) return fail(SIP_ERR_ARG, "null out");
  *out = nullptr;
  sip_plan* p = new sip_plan();
  std::string err;
  int rc = build_plan(mesh, orders, opt, p->p, err);
  if (rc != SIP_OK) {
    delete p;
    return fail(rc, err);
  }
  *out = p;
  return SIP_OK;
}

int sip_plan_info_get(const sip_plan* plan, sip_plan_info* out) {
  if (!plan || !out) return fail(SIP_ERR_ARG, "null plan or out");
  fill_info(plan->p, out);
  return SIP_OK;
}

void sip_plan_destroy(sip_plan* plan) { delete plan; }

void sip_destroy(sip_handle* h) {
  if (!h) return;
  h->release();
  delete h;
}

int sip_create(const sip_mesh* mesh, const int32_t* orders, double lambda, const sip_options* opt,
               sip_handle** out) {
  if (!out) return fail(SIP_ERR_ARG, "null out");
  *out = nullptr;
  if (!(lambda >= 0.0)) return fail(SIP_ERR_ARG, "lambda must be >= 0");
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(SIP_ERR_NO_DEVICE, std::string("no CUDA device: ") + cudaGetErrorString(ce));
  }
  sip_handle* h = new sip_handle();
  std::string err;
  int rc = build_plan(mesh, orders, opt, h->plan, err);
  if (rc != SIP_OK) {
    delete h;
    return fail(rc, err);
  }
  h->lambda = lambda;
  cudaGetDevice(&h->device);
  rc = ensure_tables(h->device);
  if (rc) { delete h; return rc; }
  {
    const GlobalTables& gt = g_tables[h->device][h->plan.opt.quad_rule];
    h->gtab_d = gt.tab_d;
    h->gtab_f = gt.tab_f;
    h->ggw_d = gt.gw_d;
    h->ggw_f = gt.gw_f;
  }
  const Plan& p = h->plan;
  cudaError_t e = cudaSuccess;
#define UP(dst, vec) \
  if (e == cudaSuccess) e = upload(&(dst), (vec).data(), (vec).size() * sizeof((vec)[0]))
  UP(h->dof_off, p.dof_off);
  UP(h->quad_off, p.quad_off);
  UP(h->vgoff, p.vgoff);
  UP(h->f_troff, p.f_troff);
  UP(h->f_goff, p.f_goff);
  UP(h->slots, p.slots);
  UP(h->elist, p.elist);
  UP(h->eaff, p.affine);
  UP(h->desc_e, p.desc_e);
  UP(h->desc_s, p.desc_s);
  UP(h->gd.vgeo, p.vgeo);
  UP(h->gd.fgeo, p.fgeo);
  UP(h->gd.tau, p.f_tau);
  std::vector<float> vf = to_float(p.vgeo), ff = to_float(p.fgeo), tf = to_float(p.f_tau);
  UP(h->gf.vgeo, vf);
  UP(h->gf.fgeo, ff);
  UP(h->gf.tau, tf);
  UP(h->xq, p.xq);
  if (h->p2p()) {
    // Lagrange interpolation from every f-point rule to every t-point one (the
    // handle's point rule): block (f, t) at (f (kQMax+1) + t) kQMax^2, entry
    // [z][r] = l_{f,r}(xi_{t,z})
    const size_t blk = (size_t)kQMax * kQMax;
    std::vector<double> I((size_t)(kQMax + 1) * (kQMax + 1) * blk, 0.0);
    std::vector<double> xf, wf, xt, wt;
    for (int f = kQMin; f <= kQMax; ++f) {
      point_rule(p.opt.quad_rule, f, xf, wf);
      for (int t = kQMin; t <= kQMax; ++t) {
        point_rule(p.opt.quad_rule, t, xt, wt);
        double* B = &I[((size_t)f * (kQMax + 1) + t) * blk];
        for (int z = 0; z < t; ++z)
          for (int r = 0; r < f; ++r) B[z * kQMax + r] = lagrange(xf, r, xt[z]);
      }
    }
    std::vector<float> If = to_float(I);
    UP(h->p2p_I_d, I);
    UP(h->p2p_I_f, If);
  }
#undef UP
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->gbar, 4 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(h->gbar, 0, 4 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->gd.kappa, std::max<size_t>(16, p.nquad * sizeof(double)));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->gf.kappa, std::max<size_t>(16, p.nquad * sizeof(float)));
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreate(&h->ev[i]);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "sip_create upload");
    sip_destroy(h);
    return rc;
  }
  for (int prec : {SIP_FP64, SIP_FP32}) {
    rc = set_tiles(h, prec, nullptr, 0, 0, 256, SIP_CTAS_SEQUENTIAL);
    if (rc) { sip_destroy(h); return rc; }
  }
  rc = handle_grow_trace(h, 1);
  if (rc) { sip_destroy(h); return rc; }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "sip_create sync");
    sip_destroy(h);
    return rc;
  }
  *out = h;
  return SIP_OK;
}

int64_t sip_num_dofs(const sip_handle* h) { return h ? h->plan.ndof : -1; }
int64_t sip_num_quad(const sip_handle* h) { return h ? h->plan.nquad : -1; }

int sip_dof_offsets(const sip_handle* h, int64_t* out) {
  if (!h || !out) return fail(SIP_ERR_ARG, "null handle or out");
  std::memcpy(out, h->plan.dof_off.data(), h->plan.dof_off.size() * sizeof(int64_t));
  return SIP_OK;
}

int sip_quad_offsets(const sip_handle* h, int64_t* out) {
  if (!h || !out) return fail(SIP_ERR_ARG, "null handle or out");
  std::memcpy(out, h->plan.quad_off.data(), h->plan.quad_off.size() * sizeof(int64_t));
  return SIP_OK;
}

int sip_get_plan_info(const sip_handle* h, sip_plan_info* out) {
  if (!h || !out) return fail(SIP_ERR_ARG, "null handle or out");
  fill_info(h->plan, out);
  return SIP_OK;
}

int sip_set_lambda(sip_handle* h, double lambda) {
  if (!h) return fail(SIP_ERR_ARG, "null handle");
  if (!(lambda >= 0.0)) return fail(SIP_ERR_ARG, "lambda must be >= 0");
  h->lambda = lambda;
  // lambda is a kernel argument captured in the CG graphs: drop them
  for (auto* W : {&h->cg64, &h->cg32})
    if (W->graph) { cudaGraphExecDestroy(W->graph); W->graph = nullptr; }
  return SIP_OK;
}

int sip_apply(sip_handle* h, int precision, const void* x, void* y, int nrhs, void* stream) {
  NvtxRange r("sip_apply");
  return apply_any(h, precision, x, y, nrhs, (cudaStream_t)stream, 0, nullptr);
}

int sip_apply_host(sip_handle* h, int precision, const void* x, void* y, int nrhs, void* stream) {
  NvtxRange r("sip_apply_host");
  if (!h || !x || !y) return fail(SIP_ERR_ARG, "null handle or vector");
  if (nrhs < 1) return fail(SIP_ERR_ARG, "nrhs must be >= 1");
  if (precision != SIP_FP64 && precision != SIP_FP32) return fail(SIP_ERR_ARG, "precision");
  const size_t bytes = (size_t)nrhs * (size_t)h->plan.ndof * (precision == SIP_FP64 ? sizeof(double) : sizeof(float));
  cudaStream_t s = (cudaStream_t)stream;
  // page-locked, mapped vectors are read and written in place by the kernels
  // (over the host link, no staging copy); others go through the handle's
  // device buffers
  const void* x_map = mapped_host_range(x, bytes);
  void* y_map = mapped_host_range(y, bytes);
  if ((!x_map || !y_map) && bytes > h->io_cap) {
    cudaStreamSynchronize(s);  // earlier calls may still use the old buffers
    cudaFree(h->io_x);
    cudaFree(h->io_y);
    h->io_x = h->io_y = nullptr;
    h->io_cap = 0;
    cudaError_t e = cudaMalloc(&h->io_x, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->io_y, bytes);
    if (e != cudaSuccess) {
      cudaFree(h->io_x);
      h->io_x = nullptr;
      return cuda_fail(e, "sip_apply_host buffers");
    }
    h->io_cap = bytes;
  }
  cudaError_t e = cudaSuccess;
  if (!x_map) {
    e = cudaMemcpyAsync(h->io_x, x, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "sip_apply_host copy in");
  }
  int rc = apply_any(h, precision, x_map ? x_map : h->io_x, y_map ? y_map : h->io_y, nrhs, s, 0, nullptr);
  if (rc) return rc;
  if (!y_map) e = cudaMemcpyAsync(y, h->io_y, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? SIP_OK : cuda_fail(e, "sip_apply_host copy out");
}

int sip_apply_transpose(sip_handle* h, int precision, const void* x, void* y, int nrhs, void* stream) {
  NvtxRange r("sip_apply_transpose");
  return apply_any(h, precision, x, y, nrhs, (cudaStream_t)stream, 1, nullptr);
}

int sip_set_timing(sip_handle* h, int enable) {
  if (!h) return fail(SIP_ERR_ARG, "null handle");
  h->timing = enable != 0;
  return SIP_OK;
}

int sip_last_kernel_ms(sip_handle* h, float* trace_ms, float* main_ms) {
  if (!h || !trace_ms || !main_ms) return fail(SIP_ERR_ARG, "null argument");
  if (!h->timed_pending) return fail(SIP_ERR_ARG, "no timed apply since timing was enabled");
  cudaError_t e = cudaEventSynchronize(h->ev[2]);
  if (e != cudaSuccess) return cuda_fail(e, "event sync");
  cudaEventElapsedTime(trace_ms, h->ev[0], h->ev[1]);
  cudaEventElapsedTime(main_ms, h->ev[1], h->ev[2]);
  return SIP_OK;
}

}  // extern "C"
