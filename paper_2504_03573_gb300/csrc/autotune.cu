// Autotuner of the tile shape: coordinate descent over the orders present,
// trying a few elements-per-tile choices for one order at a time and timing the
// whole apply (all order buckets in one launch), keeping a change only for a
// clear gain.  The GPU counterpart of choosing a per-order kernel configuration
// (Sec. 5.1).  Runs at set-up time; it allocates and synchronises.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>
#include <vector>

#include "common.cuh"
#include "handle.h"

namespace sip {
namespace {

}  // namespace
}  // namespace sip

using namespace sip;

extern "C" int sip_autotune(sip_handle* h, int precision, int reps, void* stream) {
  if (!h) return fail(SIP_ERR_ARG, "null handle");
  if (precision != SIP_FP64 && precision != SIP_FP32) return fail(SIP_ERR_ARG, "precision");
  NvtxRange range("sip_autotune");
  if (reps < 1) reps = 10;
  cudaStream_t s = (cudaStream_t)stream;
  const Plan& p = h->plan;
  const int pi = precision == SIP_FP32 ? 1 : 0;
  const int es = precision == SIP_FP32 ? 4 : 8;
  int rc = handle_grow_trace(h, 1);
  if (rc) return rc;
  const size_t vb = (size_t)p.ndof * es;
  void* x = nullptr;
  void* y = nullptr;
  cudaError_t e = cudaMalloc(&x, vb);
  if (e == cudaSuccess) e = cudaMalloc(&y, vb);
  if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, vb, s);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    cudaFree(x); cudaFree(y);
    return cuda_fail(e, "autotune set-up");
  }
  std::set<int> orders;
  for (int32_t o : p.P) orders.insert(o + 1);
  // coordinate descent over the orders, each candidate timed on the full apply
  // (all buckets in one launch, as the solver runs it)
  int cur[kNMax + 2] = {};
  for (int n : orders) cur[n] = apply_epb(p.dim, n, n + 1, precision, 256);
  const bool timing = h->timing;
  h->timing = false;
  auto time_full = [&](const int* epb, int per_sm, int mode, int threads, int layout, float* ms_out,
                       int* per_sm_out) -> int {
    Schedule sc;
    int r2 = make_schedule(h, precision, epb, per_sm, mode, threads, layout, sc);
    if (r2 == SIP_ERR_ARG) { *ms_out = 1e30f; return SIP_OK; }  // tile too large for shared memory
    if (r2) return r2;
    if (per_sm_out) *per_sm_out = sc.per_sm;
    DevSchedule d;
    cudaError_t ee = upload_schedule(sc, d);
    if (ee != cudaSuccess) return cuda_fail(ee, "autotune tiles");
    auto run = [&]() {
      return apply_tiles(h, precision, d.tiles, d.cta, d.flist, sc.nctas(), sc.threads, sc.smem_t, sc.smem_m,
                         sc.fused_cap, x, y, 1, s, 0, nullptr);
    };
    const int fb0 = g_fused_fallbacks;
    for (int w = 0; w < 2 && r2 == SIP_OK; ++w) r2 = run();
    if (r2 == SIP_OK && g_fused_fallbacks != fb0) {  // not the schedule it claims to be
      free_schedule(d);
      *ms_out = 1e30f;
      return SIP_OK;
    }
    // best of three batches of reps launches
    float best = 1e30f;
    for (int batch = 0; batch < 3 && r2 == SIP_OK; ++batch) {
      cudaEventRecord(a, s);
      for (int r = 0; r < reps && r2 == SIP_OK; ++r) r2 = run();
      cudaEventRecord(b, s);
      ee = cudaEventSynchronize(b);
      if (ee != cudaSuccess) { r2 = cuda_fail(ee, "autotune timing"); break; }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, a, b);
      best = std::min(best, ms);
    }
    free_schedule(d);
    *ms_out = best;
    return r2;
  };
  float cur_ms = 1e30f;
  int cur_per_sm = 0, auto_per_sm = 0, cur_threads = 256;
  int cur_mode = 0, cur_layout = SIP_CTAS_SEQUENTIAL;
  rc = time_full(cur, 0, 0, 256, cur_layout, &cur_ms, &auto_per_sm);
  // short applies: enough launches per timed batch (>= 2 ms) that the batch
  // times decide between candidates rather than the timer's noise
  if (rc == SIP_OK && cur_ms < 2.0f && cur_ms > 0.0f) {
    reps = std::min(400, (int)std::ceil(reps * 2.0f / cur_ms));
    rc = time_full(cur, 0, 0, 256, cur_layout, &cur_ms, &auto_per_sm);
  }
  // 1. elements per tile, one order at a time (256 threads, default grid)
  for (int n : orders) {
    if (rc) break;
    const int base = cur[n];
    int qmax = n + 1;  // the largest point count among the elements of this order
    for (size_t e = 0; e < p.P.size(); ++e)
      if (p.P[e] + 1 == n) qmax = std::max(qmax, (int)p.Q[e]);
    const int per = std::max(per_elem_trace(p.dim, n, qmax), per_elem_main(p.dim, n, qmax)) * es;
    const int room = (160 * 1024 - table_block_bytes(es, n, qmax) - kMetaBytes) / per;
    std::set<int> cand;
    for (int c : {base / 4, base / 2, 2 * base, 4 * base}) cand.insert(std::max(1, std::min({c, room, kMaxEpb})));
    cand.erase(base);
    for (int c : cand) {
      int trial[kNMax + 2];
      std::memcpy(trial, cur, sizeof(trial));
      trial[n] = c;
      float ms = 0.0f;
      rc = time_full(trial, 0, 0, 256, cur_layout, &ms, nullptr);
      if (rc) break;
      if (ms < 0.97f * cur_ms) {  // keep a change only for a clear gain
        cur_ms = ms;
        cur[n] = c;
      }
    }
  }
  // 2. threads per CTA (tiles scaled with them), then the resident CTAs per SM
  //    the schedule is balanced for, with one tile per CTA, persistent CTAs, or
  //    persistent CTAs running the whole apply in one cooperative launch
  int best_epb[kNMax + 2];
  std::memcpy(best_epb, cur, sizeof(cur));
  for (int threads : {256, 128, 64, 32}) {
    int scaled[kNMax + 2] = {};
    for (int n : orders) scaled[n] = std::max(1, cur[n] * threads / 256);
    for (int pers = 0; pers < 3 && rc == SIP_OK; ++pers)
      for (int ps = 0; ps <= 32 && rc == SIP_OK; ++ps) {
        if (ps == 0 && (pers || threads == 256)) continue;  // the default grid was timed above
        if (ps > 0 && threads == 256 && !pers && ps == auto_per_sm) continue;
        float ms = 0.0f;
        int got = 0;
        rc = time_full(scaled, ps, pers, threads, cur_layout, &ms, &got);
        if (rc || (ps > 0 && got != ps)) break;  // beyond the occupancy
        if (ms < 0.97f * cur_ms) {
          cur_ms = ms;
          cur_per_sm = ps;
          cur_mode = pers;
          cur_threads = threads;
          std::memcpy(best_epb, scaled, sizeof(scaled));
        }
      }
    if (rc) break;
  }
  // 3. the other block order of the CTAs, with the best of the above
  if (rc == SIP_OK) {
    float ms = 0.0f;
    int got = 0;
    rc = time_full(best_epb, cur_per_sm, cur_mode, cur_threads, SIP_CTAS_SM_MAJOR, &ms, &got);
    if (rc == SIP_OK && ms < 0.97f * cur_ms) {
      cur_ms = ms;
      cur_layout = SIP_CTAS_SM_MAJOR;
    }
  }
  h->timing = timing;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(x);
  cudaFree(y);
  if (rc) return rc;
  rc = set_tiles(h, precision, best_epb, cur_per_sm, cur_mode, cur_threads, cur_layout);
  if (rc) return rc;
  std::memcpy(h->epb[pi], best_epb, sizeof(best_epb));
  return SIP_OK;
}

extern "C" int sip_get_tiling(const sip_handle* h, int precision, sip_tiling* out) {
  if (!h || !out) return fail(SIP_ERR_ARG, "null argument");
  if (precision != SIP_FP64 && precision != SIP_FP32) return fail(SIP_ERR_ARG, "precision");
  const int pi = precision == SIP_FP32 ? 1 : 0;
  std::memset(out, 0, sizeof(*out));
  for (const Tile& t : h->tiles_h[pi]) {
    const int set = h->epb[pi][t.n];
    out->epb[t.n - 1] = std::min(kMaxEpb, set > 0 ? set : apply_epb(h->plan.dim, t.n, t.q, precision, h->threads[pi]));
  }
  out->ctas_per_sm = h->ctas_per_sm[pi];
  out->persistent = h->fused_cap[pi] > 0 ? 2 : h->persistent[pi];
  out->threads = h->threads[pi];
  out->cta_layout = h->cta_layout[pi];
  out->ntiles = (int64_t)h->tiles_h[pi].size();
  out->nctas = (int64_t)h->cta_h[pi].size() - 1;
  return SIP_OK;
}

extern "C" int sip_set_tiling(sip_handle* h, int precision, const sip_tiling* t) {
  if (!h) return fail(SIP_ERR_ARG, "null handle");
  if (precision != SIP_FP64 && precision != SIP_FP32) return fail(SIP_ERR_ARG, "precision");
  int e[kNMax + 2] = {};
  int per_sm = 0, threads = 256, pers = 0, layout = SIP_CTAS_SEQUENTIAL;
  if (t) {
    for (int P = 0; P <= kMaxOrder; ++P) {
      if (t->epb[P] < 0 || t->epb[P] > kMaxEpb) return fail(SIP_ERR_ARG, "elements per tile must be in 0.." + std::to_string(kMaxEpb));
      e[P + 1] = t->epb[P];
    }
    if (t->ctas_per_sm < 0) return fail(SIP_ERR_ARG, "ctas_per_sm must be >= 0");
    if (t->persistent < 0 || t->persistent > 2) return fail(SIP_ERR_ARG, "persistent must be 0, 1 or 2");
    per_sm = t->ctas_per_sm;
    pers = t->persistent;
    threads = t->threads == 0 ? 256 : t->threads;
    layout = t->cta_layout == 0 ? SIP_CTAS_SEQUENTIAL : t->cta_layout;
  }
  const int pi = precision == SIP_FP32 ? 1 : 0;
  int rc = set_tiles(h, precision, e, per_sm, pers, threads, layout);
  if (rc) return rc;
  std::memcpy(h->epb[pi], e, sizeof(e));
  return SIP_OK;
}
