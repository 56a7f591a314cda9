// Conjugate gradients on the SIP operator (Sec. 2.2: the symmetric SIP system
// is solved by CG), FP64 and FP32-apply inside FP64 iterative refinement; and
// the auxiliary entry points (kappa, gradients, IProduct, quadrature points,
// work model).
//
// Every reduction is deterministic: fixed grid, fixed per-thread strides,
// fixed-order shared-memory trees, then one fixed-order final pass.  So a
// solve, and a replay from a checkpoint, reproduce their iterates bit for bit.
// The CG iteration (apply + 2 dots + 3 vector updates = 7 launches) is
// captured in a CUDA graph of `check_every` iterations; the host reads the
// residual norms only between graph launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "aux_kernels.cuh"
#include "handle.h"

namespace sip {

cudaError_t launch_aux_2d(const AuxArgs&, int, size_t, cudaStream_t);
cudaError_t launch_aux_3d(const AuxArgs&, int, size_t, cudaStream_t);
cudaError_t launch_aux_gll_2d(const AuxArgs&, int, size_t, cudaStream_t);
cudaError_t launch_aux_gll_3d(const AuxArgs&, int, size_t, cudaStream_t);

namespace {

constexpr int kRedThreads = 256;
constexpr int kScal = 8;  // per-RHS scalars
enum { S_RR = 0, S_PAP = 1, S_ALPHA = 2, S_BETA = 3, S_ACTIVE = 4, S_RR0 = 5, S_AUX = 6 };
enum { ST_BREAKDOWN = 1, ST_NONFINITE = 2 };

int red_blocks(int64_t n) {
  int64_t b = (n + kRedThreads * 4 - 1) / (kRedThreads * 4);
  return (int)std::max<int64_t>(1, std::min<int64_t>(1024, b));
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int h = kRedThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  return red[0];
}

// partial[rhs][block] = sum over this block's fixed strided subset of a*b
template <typename TA, typename TB>
__global__ void __launch_bounds__(kRedThreads) k_dot_partial(const TA* a, const TB* b, int64_t n, double* partial) {
  __shared__ double red[kRedThreads];
  const int rhs = blockIdx.y;
  a += rhs * n;
  b += rhs * n;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads)
    s += (double)a[i] * (double)b[i];
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) partial[rhs * gridDim.x + blockIdx.x] = t;
}

// out = sum of nblk partials (fixed order), stored into scal[rhs*kScal + slot],
// then the CG scalar step selected by `what`:
//   0: plain store; 1: alpha = rr / pAp (breakdown check); 2: beta = rr_new / rr, rr = rr_new
__global__ void __launch_bounds__(kRedThreads) k_final(const double* partial, int nblk, double* scal, int slot,
                                                       int what, int* status) {
  __shared__ double red[kRedThreads];
  const int rhs = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += kRedThreads) s += partial[rhs * nblk + i];
  const double t = block_sum(s, red);
  if (threadIdx.x != 0) return;
  double* sc = scal + rhs * kScal;
  const bool active = sc[S_ACTIVE] != 0.0;
  if (what == 0) {
    sc[slot] = t;
  } else if (what == 1) {
    sc[S_PAP] = t;
    double alpha = 0.0;
    if (active) {
      if (!(t > 0.0)) {
        if (!isfinite(t)) atomicOr(status, ST_NONFINITE);
        else atomicOr(status, ST_BREAKDOWN);
        sc[S_ACTIVE] = 0.0;
      } else {
        alpha = sc[S_RR] / t;
      }
    }
    sc[S_ALPHA] = alpha;
  } else {
    double beta = 0.0;
    if (active) {
      if (!isfinite(t)) atomicOr(status, ST_NONFINITE);
      beta = sc[S_RR] > 0.0 ? t / sc[S_RR] : 0.0;
      sc[S_RR] = t;
    }
    sc[S_BETA] = beta;
  }
}

// x += alpha p (in the precision of x), r -= alpha Ap, partial sums of r.r
template <typename TX, typename T>
__global__ void __launch_bounds__(kRedThreads) k_update_xr(TX* x, T* r, const T* p, const T* ap, int64_t n,
                                                           const double* scal, double* partial) {
  __shared__ double red[kRedThreads];
  const int rhs = blockIdx.y;
  const TX alpha_x = (TX)scal[rhs * kScal + S_ALPHA];
  const T alpha = (T)scal[rhs * kScal + S_ALPHA];
  x += rhs * n; r += rhs * n; p += rhs * n; ap += rhs * n;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kRedThreads) {
    x[i] = fma(alpha_x, (TX)p[i], x[i]);
    const T ri = fma(-alpha, ap[i], r[i]);
    r[i] = ri;
    s += (double)ri * (double)ri;
  }
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) partial[rhs * gridDim.x + blockIdx.x] = t;
}

// p = r + beta p
template <typename T>
__global__ void k_update_p(const T* r, T* p, int64_t n, const double* scal) {
  const int rhs = blockIdx.y;
  const T beta = (T)scal[rhs * kScal + S_BETA];
  r += rhs * n; p += rhs * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], r[i]);
}

// r = b - r (in place, r holds A x); FP64
__global__ void k_residual(const double* b, double* r, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - r[i];
}

// r32 = float(r64) (and p32 = r32 when p32 is given)
__global__ void k_r64_to_r32(const double* r64, float* r32, float* p32, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = (float)r64[i];
    r32[i] = v;
    if (p32) p32[i] = v;
  }
}

// r32 = float(s[rhs] * r64), x32 = 0, p32 = r32
__global__ void k_to_f32(const double* r64, float* r32, float* x32, float* p32, int64_t n, const double* s) {
  const int rhs = blockIdx.y;
  const double sc = s[rhs];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = (float)(sc * r64[rhs * n + i]);
    r32[rhs * n + i] = v;
    p32[rhs * n + i] = v;
    x32[rhs * n + i] = 0.0f;
  }
}

// x64 += s[rhs] * d32
__global__ void k_add_f32(double* x64, const float* d32, int64_t n, const double* s) {
  const int rhs = blockIdx.y;
  const double sc = s[rhs];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x64[rhs * n + i] += sc * (double)d32[rhs * n + i];
}

// kappa double -> float copy
__global__ void k_d2f(const double* a, float* b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

__global__ void k_nonfinite(const double* a, int64_t n, int* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(a[i])) *flag = 1;
}

dim3 vgrid(int64_t n, int nrhs) {
  int64_t b = (n + 255) / 256;
  return dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(2048, b)), (unsigned)nrhs);
}

}  // namespace

void CgWork::release() {
  if (graph) cudaGraphExecDestroy(graph);
  graph = nullptr;
  cudaFree(x); cudaFree(r); cudaFree(p); cudaFree(ap);
  cudaFree(scal); cudaFree(partial); cudaFree(status);
  x = r = p = ap = nullptr;
  scal = partial = nullptr;
  status = nullptr;
  nrhs = 0;
}

}  // namespace sip

void sip_handle::release() {
  cg64.release();
  cg32.release();
  cudaFree(r64); cudaFree(x64); cudaFree(xbak); cudaFree(red);
  if (scal_host) cudaFreeHost(scal_host);
  for (auto& c : ck) { cudaFree(c.x); cudaFree(c.r); cudaFree(c.p); }
  ck.clear();
  if (solve_stream) cudaStreamDestroy(solve_stream);
  cudaFree(dof_off); cudaFree(quad_off); cudaFree(vgoff); cudaFree(f_troff); cudaFree(f_goff);
  cudaFree(desc_e); cudaFree(desc_s); cudaFree(gbar);
  cudaFree(slots); cudaFree(elist); cudaFree(eaff); cudaFree(tiles_d[0]); cudaFree(tiles_d[1]); cudaFree(cta_d[0]); cudaFree(cta_d[1]); cudaFree(flist_d[0]); cudaFree(flist_d[1]); cudaFree(xq);
  cudaFree(gd.vgeo); cudaFree(gd.fgeo); cudaFree(gd.tau); cudaFree(gd.kappa);
  cudaFree(gf.vgeo); cudaFree(gf.fgeo); cudaFree(gf.tau); cudaFree(gf.kappa);
  cudaFree(trace_d);
  cudaFree(io_x);
  cudaFree(io_y);
  cudaFree(p2p_I_d);
  cudaFree(p2p_I_f);
  cudaFree(ug_d);
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
}

namespace sip {
namespace {

int ensure_cg(sip_handle* h, CgWork& W, size_t es, int nrhs) {
  if (W.nrhs == nrhs && W.elem == es) return SIP_OK;
  W.release();
  const size_t n = (size_t)h->plan.ndof * nrhs;
  const int nblk = red_blocks(h->plan.ndof);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&W.x, n * es);
  if (e == cudaSuccess) e = cudaMalloc(&W.r, n * es);
  if (e == cudaSuccess) e = cudaMalloc(&W.p, n * es);
  if (e == cudaSuccess) e = cudaMalloc(&W.ap, n * es);
  if (e == cudaSuccess) e = cudaMalloc((void**)&W.scal, sizeof(double) * kScal * nrhs);
  if (e == cudaSuccess) e = cudaMalloc((void**)&W.partial, sizeof(double) * nblk * nrhs);
  if (e == cudaSuccess) e = cudaMalloc((void**)&W.status, sizeof(int));
  if (e != cudaSuccess) { W.release(); return cuda_fail(e, "CG workspace"); }
  W.nrhs = nrhs;
  W.elem = es;
  return SIP_OK;
}

int ensure_solver(sip_handle* h, int nrhs) {
  if (!h->solve_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&h->solve_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "solver stream");
  }
  if (!h->scal_host) {
    cudaError_t e = cudaMallocHost((void**)&h->scal_host, sizeof(double) * kScal * 1024);
    if (e != cudaSuccess) return cuda_fail(e, "pinned scalars");
  }
  if (nrhs > 1000) return fail(SIP_ERR_ARG, "nrhs > 1000");
  if (h->work_nrhs < nrhs) {
    cudaFree(h->r64); cudaFree(h->x64); cudaFree(h->xbak);
    h->r64 = h->x64 = h->xbak = nullptr;
    const size_t n = (size_t)h->plan.ndof * nrhs;
    cudaError_t e = cudaMalloc((void**)&h->r64, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->x64, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->xbak, n * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "solver vectors");
    h->work_nrhs = nrhs;
  }
  if (!h->red) {
    const size_t nb = std::max<size_t>(h->tiles_h[0].size(), 1024) + 2048;
    cudaError_t e = cudaMalloc((void**)&h->red, nb * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "reduction buffer");
  }
  return handle_grow_trace(h, nrhs);
}

// dot products a_r . b_r for every RHS into scal[rhs*kScal + slot]
template <typename TA, typename TB>
void enqueue_dot(sip_handle* h, CgWork& W, const TA* a, const TB* b, int nrhs, int slot, int what, cudaStream_t s) {
  const int nblk = red_blocks(h->plan.ndof);
  k_dot_partial<TA, TB><<<dim3(nblk, nrhs), kRedThreads, 0, s>>>(a, b, h->plan.ndof, W.partial);
  k_final<<<nrhs, kRedThreads, 0, s>>>(W.partial, nblk, W.scal, slot, what, W.status);
}

// one CG iteration on workspace W (vector type T, apply precision prec)
template <typename T>
int enqueue_iter(sip_handle* h, CgWork& W, int nrhs, int prec, int transpose, cudaStream_t s) {
  const int64_t n = h->plan.ndof;
  int rc = apply_any(h, prec, W.p, W.ap, nrhs, s, transpose, nullptr);
  if (rc) return rc;
  enqueue_dot<T, T>(h, W, (const T*)W.p, (const T*)W.ap, nrhs, S_PAP, 1, s);
  const int nblk = red_blocks(n);
  if (W.xext)
    k_update_xr<double, T><<<dim3(nblk, nrhs), kRedThreads, 0, s>>>((double*)W.xext, (T*)W.r, (const T*)W.p,
                                                                   (const T*)W.ap, n, W.scal, W.partial);
  else
    k_update_xr<T, T><<<dim3(nblk, nrhs), kRedThreads, 0, s>>>((T*)W.x, (T*)W.r, (const T*)W.p, (const T*)W.ap, n,
                                                              W.scal, W.partial);
  k_final<<<nrhs, kRedThreads, 0, s>>>(W.partial, nblk, W.scal, S_RR, 2, W.status);
  k_update_p<T><<<vgrid(n, nrhs), 256, 0, s>>>((const T*)W.r, (T*)W.p, n, W.scal);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIP_OK : cuda_fail(e, "CG iteration");
}

// run `iters` iterations: as a captured graph (cached per workspace) or directly
template <typename T>
int run_iters(sip_handle* h, CgWork& W, int nrhs, int prec, int transpose, int iters, cudaStream_t s, bool use_graph) {
  if (!use_graph) {
    for (int i = 0; i < iters; ++i) {
      int rc = enqueue_iter<T>(h, W, nrhs, prec, transpose, s);
      if (rc) return rc;
    }
    return SIP_OK;
  }
  if (!W.graph || W.graph_iters != iters || W.graph_transpose != transpose || W.graph_xext != W.xext) {
    if (W.graph) cudaGraphExecDestroy(W.graph);
    W.graph = nullptr;
    const bool timing = h->timing;
    h->timing = false;
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { h->timing = timing; return cuda_fail(e, "begin capture"); }
    int rc = SIP_OK;
    for (int i = 0; i < iters && rc == SIP_OK; ++i) rc = enqueue_iter<T>(h, W, nrhs, prec, transpose, s);
    e = cudaStreamEndCapture(s, &g);
    h->timing = timing;
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&W.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    W.graph_iters = iters;
    W.graph_transpose = transpose;
    W.graph_xext = W.xext;
  }
  cudaError_t e = cudaGraphLaunch(W.graph, s);
  return e == cudaSuccess ? SIP_OK : cuda_fail(e, "graph launch");
}

int read_scal(sip_handle* h, CgWork& W, int nrhs, cudaStream_t s, int* status) {
  cudaMemcpyAsync(h->scal_host, W.scal, sizeof(double) * kScal * nrhs, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(h->scal_host + kScal * 1023, W.status, sizeof(int), cudaMemcpyDeviceToHost, s);
  // status word of the single-launch apply's grid barrier
  cudaMemcpyAsync(h->scal_host + kScal * 1023 + 1, h->gbar + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "CG scalars");
  std::memcpy(status, h->scal_host + kScal * 1023, sizeof(int));
  unsigned int gb = 0;
  std::memcpy(&gb, h->scal_host + kScal * 1023 + 1, sizeof(unsigned int));
  if (gb) return fail(SIP_ERR_CUDA, "a grid-barrier wait of the single-launch apply gave up");
  return SIP_OK;
}

int write_scal(sip_handle* h, CgWork& W, int nrhs, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(W.scal, h->scal_host, sizeof(double) * kScal * nrhs, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? SIP_OK : cuda_fail(e, "CG scalars upload");
}

// Save the recurrence state (x FP64; r, p of element size es; the per-RHS scalars,
// already on the host in scal_host) into the next slot of the checkpoint ring.
int save_checkpoint(sip_handle* h, const void* x, const void* r, const void* p, size_t es, int nrhs, int mode,
                    int transpose, int iter, int refinements, int restarts, const std::vector<double>& tol,
                    cudaStream_t s) {
  const int ns = std::max(1, h->plan.opt.checkpoint_slots);
  if ((int)h->ck.size() != ns) {
    for (auto& c : h->ck) { cudaFree(c.x); cudaFree(c.r); cudaFree(c.p); }
    h->ck.assign(ns, Checkpoint{});
    h->ck_count = h->ck_next = 0;
  }
  Checkpoint& c = h->ck[h->ck_next];
  const size_t n = (size_t)h->plan.ndof * nrhs;
  const size_t need = n * sizeof(double);
  if (c.cap < need) {
    cudaFree(c.x); cudaFree(c.r); cudaFree(c.p);
    c.x = c.r = c.p = nullptr;
    c.cap = 0;
    cudaError_t e = cudaMalloc(&c.x, need);
    if (e == cudaSuccess) e = cudaMalloc(&c.r, need);
    if (e == cudaSuccess) e = cudaMalloc(&c.p, need);
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint ring");
    c.cap = need;
  }
  cudaMemcpyAsync(c.x, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(c.r, r, n * es, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(c.p, p, n * es, cudaMemcpyDeviceToDevice, s);
  c.scal.assign(h->scal_host, h->scal_host + kScal * nrhs);
  c.tol = tol;
  c.iter = iter;
  c.refinements = refinements;
  c.restarts = restarts;
  c.mode = mode;
  c.nrhs = nrhs;
  c.transpose = transpose;
  h->ck_next = (h->ck_next + 1) % ns;
  h->ck_count = std::min(h->ck_count + 1, ns);
  return SIP_OK;
}

// Checkpointing of the FP64 recurrence inside cg_loop: iteration and restart
// counts of the solve at the loop's start.
struct CkCtx {
  bool on = false;
  int iter0 = 0;
  int restarts = 0;
};

// Inner CG loop from the state already in W (r, p, x, scal with RR and ACTIVE set).
// Runs until every active RHS has sqrt(rr) <= tol[rhs], or `budget` iterations,
// in chunks of `chunk` iterations (a captured graph each) with the convergence
// test between chunks; ck.on saves a checkpoint after every full chunk.
template <typename T>
int cg_loop(sip_handle* h, CgWork& W, int nrhs, int prec, int transpose, const std::vector<double>& tol,
            int budget, int* iters_done, cudaStream_t s, int chunk, const CkCtx& ck) {
  chunk = std::max(1, chunk);
  int done = 0;
  while (true) {
    int status = 0;
    int rc = read_scal(h, W, nrhs, s, &status);
    if (rc) return rc;
    if (status & ST_NONFINITE) return fail(SIP_ERR_NONFINITE, "non-finite CG scalar");
    if (status & ST_BREAKDOWN) return fail(SIP_ERR_BREAKDOWN, "CG breakdown: p^T A p <= 0");
    bool any = false, changed = false;
    for (int r = 0; r < nrhs; ++r) {
      double* sc = h->scal_host + r * kScal;
      if (sc[S_ACTIVE] == 0.0) continue;
      if (!std::isfinite(sc[S_RR])) return fail(SIP_ERR_NONFINITE, "non-finite residual");
      if (std::sqrt(sc[S_RR]) <= tol[r]) { sc[S_ACTIVE] = 0.0; changed = true; }
      else any = true;
    }
    if (changed) { rc = write_scal(h, W, nrhs, s); if (rc) return rc; }
    if (!any || done >= budget) break;
    const int it = std::min(chunk, budget - done);
    rc = run_iters<T>(h, W, nrhs, prec, transpose, it, s, it == chunk);
    if (rc) return rc;
    done += it;
    if (ck.on && it == chunk) {
      int status = 0;
      rc = read_scal(h, W, nrhs, s, &status);
      if (rc == SIP_OK)
        rc = save_checkpoint(h, W.x, W.r, W.p, sizeof(T), nrhs, SIP_CG_FP64, transpose, *iters_done + done, 0,
                             ck.restarts, tol, s);
      if (rc) return rc;
    }
  }
  *iters_done += done;
  return SIP_OK;
}

// ||v_r||^2 for every RHS (FP64), to host
int norms2(sip_handle* h, CgWork& W, const double* v, int nrhs, cudaStream_t s, std::vector<double>& out) {
  enqueue_dot<double, double>(h, W, v, v, nrhs, S_AUX, 0, s);
  int st = 0;
  int rc = read_scal(h, W, nrhs, s, &st);
  if (rc) return rc;
  out.resize(nrhs);
  for (int r = 0; r < nrhs; ++r) out[r] = h->scal_host[r * kScal + S_AUX];
  return SIP_OK;
}

int solve_impl(sip_handle* h, int mode, const double* b, double* x_out, int nrhs, double rtol,
               sip_stats* stats, cudaStream_t user, int transpose) {
  NvtxRange range(mode == SIP_CG_FP32_REFINED ? "sip_cg_solve fp32-refined" : "sip_cg_solve fp64");
  auto t0 = std::chrono::steady_clock::now();
  if (!h || !b || !x_out) return fail(SIP_ERR_ARG, "null argument");
  if (nrhs < 1) return fail(SIP_ERR_ARG, "nrhs must be >= 1");
  if (!(rtol > 0.0)) return fail(SIP_ERR_ARG, "rtol must be > 0");
  if (mode != SIP_CG_FP64 && mode != SIP_CG_FP32_REFINED) return fail(SIP_ERR_ARG, "mode");
  int rc = ensure_solver(h, nrhs);
  if (rc) return rc;
  const int64_t n = h->plan.ndof;
  const size_t bytes = sizeof(double) * n * nrhs;
  cudaStream_t s = h->solve_stream;
  // order after the caller's pending work
  cudaEvent_t evu;
  cudaEventCreateWithFlags(&evu, cudaEventDisableTiming);
  cudaEventRecord(evu, user);
  cudaStreamWaitEvent(s, evu, 0);
  sip_stats st;
  std::memset(&st, 0, sizeof(st));
  rc = ensure_cg(h, h->cg64, sizeof(double), nrhs);
  if (rc) { cudaEventDestroy(evu); return rc; }
  CgWork& W = h->cg64;
  // input check and ||b||
  {
    int zero = 0;
    cudaMemcpyAsync(W.status, &zero, sizeof(int), cudaMemcpyHostToDevice, s);
    k_nonfinite<<<vgrid(n * nrhs, 1), 256, 0, s>>>(b, n * nrhs, W.status);
    int flag = 0;
    cudaMemcpyAsync(&flag, W.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (flag) { cudaEventDestroy(evu); return fail(SIP_ERR_NONFINITE, "non-finite right-hand side"); }
  }
  std::vector<double> bn2;
  rc = norms2(h, W, b, nrhs, s, bn2);
  if (rc) { cudaEventDestroy(evu); return rc; }
  std::vector<double> tol(nrhs);
  for (int r = 0; r < nrhs; ++r) tol[r] = rtol * std::sqrt(bn2[r]);
  const int max_iter = h->plan.opt.max_iter;
  bool converged = false;
  double worst = 0.0;
  h->ck_count = 0;
  h->ck_next = 0;
  // checkpoints every checkpoint_every iterations of whichever recurrence runs
  // (FP64 CG, or the FP32 recurrence of the refined mode), any number of RHS
  const bool ckpt = h->plan.opt.checkpoint_every > 0;
  // FP64 CG from the state (W.x, W.r = b - A W.x, rr) until the true residual meets tol
  auto fp64_cg = [&](const std::vector<double>& r0n2) -> int {
    cudaMemcpyAsync(W.p, W.r, bytes, cudaMemcpyDeviceToDevice, s);
    for (int r = 0; r < nrhs; ++r) {
      double* sc = h->scal_host + r * kScal;
      std::fill(sc, sc + kScal, 0.0);
      sc[S_RR] = r0n2[r];
      sc[S_RR0] = r0n2[r];
      sc[S_ACTIVE] = std::sqrt(r0n2[r]) > tol[r] ? 1.0 : 0.0;
    }
    int zero = 0;
    cudaMemcpyAsync(W.status, &zero, sizeof(int), cudaMemcpyHostToDevice, s);
    int rc2 = write_scal(h, W, nrhs, s);
    int restarts = 0;
    while (rc2 == SIP_OK) {
      const CkCtx ck{ckpt, st.iterations, restarts};
      const int chunk = ckpt ? h->plan.opt.checkpoint_every : h->plan.opt.check_every;
      rc2 = cg_loop<double>(h, W, nrhs, SIP_FP64, transpose, tol, max_iter - st.iterations, &st.iterations, s, chunk, ck);
      if (rc2) break;
      // true residual r64 = b - A x
      rc2 = apply_any(h, SIP_FP64, W.x, h->r64, nrhs, s, transpose, nullptr);
      if (rc2) break;
      st.applies_fp64 += 1;
      k_residual<<<vgrid(n * nrhs, 1), 256, 0, s>>>(b, h->r64, n * nrhs);
      std::vector<double> rn2;
      rc2 = norms2(h, W, h->r64, nrhs, s, rn2);
      if (rc2) break;
      bool all = true;
      worst = 0.0;
      for (int r = 0; r < nrhs; ++r) {
        const double rel = bn2[r] > 0 ? std::sqrt(rn2[r] / bn2[r]) : 0.0;
        worst = std::max(worst, rel);
        double* sc = h->scal_host + r * kScal;
        if (std::sqrt(rn2[r]) > tol[r]) {
          all = false;
          sc[S_RR] = rn2[r];
          sc[S_ACTIVE] = 1.0;
        } else {
          sc[S_ACTIVE] = 0.0;
        }
      }
      if (all) { converged = true; break; }
      if (st.iterations >= max_iter || restarts > 50) break;
      // residual replacement for the columns that have not converged: r = r_true, p = r
      ++restarts;
      cudaMemcpyAsync(W.r, h->r64, bytes, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(W.p, h->r64, bytes, cudaMemcpyDeviceToDevice, s);
      rc2 = write_scal(h, W, nrhs, s);
    }
    return rc2;
  };
  if (mode == SIP_CG_FP64) {
    // x = 0, r = b, rr = ||b||^2
    cudaMemsetAsync(W.x, 0, bytes, s);
    cudaMemcpyAsync(W.r, b, bytes, cudaMemcpyDeviceToDevice, s);
    rc = fp64_cg(bn2);
    st.applies_fp64 += st.iterations;
    if (rc == SIP_OK) cudaMemcpyAsync(x_out, W.x, bytes, cudaMemcpyDeviceToDevice, s);
  } else {
    // FP32 apply inside FP64 iterative refinement, in reliable-update form: one
    // CG recurrence runs with FP32 vectors and the FP32 operator (FP64 dot
    // products, FP64 iterate x); whenever the FP32 residual has fallen by
    // kDelta since the last refinement, the FP64 residual r = b - A_64 x is
    // recomputed and replaces it, keeping the search direction.
    const double kDelta = 0.1;
    rc = ensure_cg(h, h->cg32, sizeof(float), nrhs);
    CgWork& V = h->cg32;
    V.xext = h->x64;
    if (rc == SIP_OK) {
      cudaMemsetAsync(h->x64, 0, bytes, s);
      cudaMemcpyAsync(h->r64, b, bytes, cudaMemcpyDeviceToDevice, s);
      k_r64_to_r32<<<vgrid(n * nrhs, 1), 256, 0, s>>>(h->r64, (float*)V.r, (float*)V.p, n * nrhs);
      for (int r = 0; r < nrhs; ++r) {
        double* sc = h->scal_host + r * kScal;
        std::fill(sc, sc + kScal, 0.0);
        sc[S_RR] = bn2[r];
        sc[S_RR0] = bn2[r];
        sc[S_ACTIVE] = bn2[r] > 0.0 ? 1.0 : 0.0;
      }
      int zero = 0;
      cudaMemcpyAsync(V.status, &zero, sizeof(int), cudaMemcpyHostToDevice, s);
      rc = write_scal(h, V, nrhs, s);
    }
    std::vector<double> rmax(nrhs);
    for (int r = 0; r < nrhs; ++r) rmax[r] = std::sqrt(bn2[r]);
    const int chunk = std::max(1, h->plan.opt.check_every);
    // the FP32 recurrence is checkpointed at chunk boundaries, every
    // checkpoint_every iterations rounded up to whole chunks
    const int ck_every_chunks = std::max(1, (h->plan.opt.checkpoint_every + chunk - 1) / chunk);
    int total = 0;
    bool all_conv = false;
    double best = 1e300;   // best worst-case true residual so far
    int stalled = 0;       // refinements without a 2x improvement of it
    bool polish = false;   // fall back to FP64 CG from the last refined iterate
    int since = 0;         // FP32 iterations since the last refinement
    cudaMemsetAsync(h->xbak, 0, bytes, s);
    while (rc == SIP_OK) {
      // iterate until some RHS's FP32 residual has dropped by kDelta (or is below
      // tol), or for a bounded number of iterations
      bool trigger = false, broke = false;
      const int cap = std::max(512, 4 * (st.refinements > 0 ? total / st.refinements : 0));
      while (rc == SIP_OK && !trigger && total < max_iter) {
        rc = run_iters<float>(h, V, nrhs, SIP_FP32, transpose, chunk, s, true);
        if (rc) break;
        total += chunk;
        since += chunk;
        int status = 0;
        rc = read_scal(h, V, nrhs, s, &status);
        if (rc) break;
        if (status & (ST_NONFINITE | ST_BREAKDOWN)) { broke = true; break; }
        if (ckpt && (total / chunk) % ck_every_chunks == 0) {
          rc = save_checkpoint(h, h->x64, V.r, V.p, sizeof(float), nrhs, SIP_CG_FP32_REFINED, transpose, total,
                               st.refinements, 0, tol, s);
          if (rc) break;
        }
        for (int r = 0; r < nrhs; ++r) {
          const double* sc = h->scal_host + r * kScal;
          if (sc[S_ACTIVE] == 0.0) continue;
          const double rn = std::sqrt(sc[S_RR]);
          if (!std::isfinite(rn)) broke = true;
          else if (rn <= kDelta * rmax[r] || rn <= tol[r]) trigger = true;
        }
        if (broke) break;
        if (since >= cap) trigger = true;
      }
      if (rc) break;
      if (broke) {
        // the FP32 recurrence broke down (typically below the FP64 residual
        // floor): return to the last refined iterate and finish in FP64
        cudaMemcpyAsync(h->x64, h->xbak, bytes, cudaMemcpyDeviceToDevice, s);
        if (st.refinements == 0) cudaMemcpyAsync(h->r64, b, bytes, cudaMemcpyDeviceToDevice, s);
        polish = true;
        break;
      }
      since = 0;
      // refinement: FP64 residual of the FP64 iterate
      NvtxRange refine("sip_cg refinement");
      rc = apply_any(h, SIP_FP64, h->x64, h->r64, nrhs, s, transpose, nullptr);
      if (rc) break;
      st.applies_fp64 += 1;
      st.refinements += 1;
      k_residual<<<vgrid(n * nrhs, 1), 256, 0, s>>>(b, h->r64, n * nrhs);
      cudaMemcpyAsync(h->xbak, h->x64, bytes, cudaMemcpyDeviceToDevice, s);  // r64 is its residual
      std::vector<double> rn2;
      rc = norms2(h, W, h->r64, nrhs, s, rn2);
      if (rc) break;
      // norms2 overwrote nothing in V; reload V's scalars to edit them
      int status = 0;
      rc = read_scal(h, V, nrhs, s, &status);
      if (rc) break;
      all_conv = true;
      worst = 0.0;
      for (int r = 0; r < nrhs; ++r) {
        double* sc = h->scal_host + r * kScal;
        worst = std::max(worst, bn2[r] > 0 ? std::sqrt(rn2[r] / bn2[r]) : 0.0);
        if (std::sqrt(rn2[r]) <= tol[r]) {
          sc[S_ACTIVE] = 0.0;
        } else {
          all_conv = false;
          sc[S_RR] = rn2[r];
          sc[S_ACTIVE] = 1.0;
          rmax[r] = std::sqrt(rn2[r]);
        }
      }
      if (all_conv || total >= max_iter) break;
      if (worst < 0.5 * best) { best = worst; stalled = 0; }
      else if (++stalled >= 4) { polish = true; break; }  // FP32 recurrence no longer gains: finish in FP64
      // replace the FP32 residual by the FP64 one, keep the search direction
      k_r64_to_r32<<<vgrid(n * nrhs, 1), 256, 0, s>>>(h->r64, (float*)V.r, nullptr, n * nrhs);
      rc = write_scal(h, V, nrhs, s);
    }
    converged = rc == SIP_OK && all_conv;
    st.iterations = total;
    st.applies_fp32 = total;
    V.xext = nullptr;
    if (rc == SIP_OK && polish) {
      // FP64 CG from x64 with r = b - A_64 x64 (already in r64)
      std::vector<double> rn2;
      rc = norms2(h, W, h->r64, nrhs, s, rn2);
      if (rc == SIP_OK) {
        cudaMemcpyAsync(W.x, h->x64, bytes, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(W.r, h->r64, bytes, cudaMemcpyDeviceToDevice, s);
        const int before = st.iterations;
        rc = fp64_cg(rn2);
        st.applies_fp64 += st.iterations - before;
        if (rc == SIP_OK) cudaMemcpyAsync(h->x64, W.x, bytes, cudaMemcpyDeviceToDevice, s);
      }
    }
    if (rc == SIP_OK) cudaMemcpyAsync(x_out, h->x64, bytes, cudaMemcpyDeviceToDevice, s);
  }
  cudaEventRecord(evu, s);
  cudaStreamWaitEvent(user, evu, 0);
  cudaStreamSynchronize(s);
  cudaEventDestroy(evu);
  st.rel_residual = worst;
  st.converged = converged ? 1 : 0;
  st.checkpoints = ckpt ? h->ck_count : 0;
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  if (rc) return rc;
  if (!converged) return fail(SIP_ERR_NOT_CONVERGED, "CG did not reach the tolerance within max_iter");
  return SIP_OK;
}

size_t aux_smem(sip_handle* h) {
  size_t m = 0;
  for (const Tile& t : h->tiles_h[0]) {
    m = std::max(m, (size_t)t.count * aux_smem_per_element(h->plan.dim, t.n, t.q) * sizeof(double));
  }
  return m + kRedThreads * sizeof(double);
}

int launch_aux(sip_handle* h, AuxArgs& a, cudaStream_t s) {
  a.dof_off = h->dof_off;
  a.quad_off = h->quad_off;
  a.vgoff = h->vgoff;
  a.vgeo = h->gd.vgeo;
  a.elist = h->elist;
  a.eaff = h->eaff;
  a.tiles = h->tiles_d[0];
  const int nt = (int)h->tiles_h[0].size();
  const bool gll = h->plan.opt.quad_rule == SIP_RULE_GLL;
  cudaError_t e = h->plan.dim == 2 ? (gll ? launch_aux_gll_2d : launch_aux_2d)(a, nt, aux_smem(h), s)
                                   : (gll ? launch_aux_gll_3d : launch_aux_3d)(a, nt, aux_smem(h), s);
  return e == cudaSuccess ? SIP_OK : cuda_fail(e, "aux kernel");
}

}  // namespace
}  // namespace sip

using namespace sip;

extern "C" {

int sip_cg_solve(sip_handle* h, int mode, const double* b, double* x, int nrhs, double rtol, sip_stats* stats,
                 void* stream) {
  if (h && h->p2p()) return fail(SIP_ERR_ARG, "CG needs the symmetric shared-rule operator (face_scheme SIP_FACES_SHARED)");
  return solve_impl(h, mode, b, x, nrhs, rtol, stats, (cudaStream_t)stream, 0);
}

int sip_cg_solve_transpose(sip_handle* h, int mode, const double* b, double* x, int nrhs, double rtol,
                           sip_stats* stats, void* stream) {
  if (h && h->p2p()) return fail(SIP_ERR_ARG, "CG needs the symmetric shared-rule operator (face_scheme SIP_FACES_SHARED)");
  return solve_impl(h, mode, b, x, nrhs, rtol, stats, (cudaStream_t)stream, 1);
}

int sip_cg_checkpoint_count(const sip_handle* h) { return h ? h->ck_count : -1; }

static const Checkpoint* checkpoint_at(const sip_handle* h, int slot) {
  if (slot < 0 || slot >= h->ck_count) return nullptr;
  const int ns = (int)h->ck.size();
  return &h->ck[(h->ck_next - h->ck_count + slot + 2 * ns) % ns];
}

int sip_cg_checkpoint_get(sip_handle* h, int slot, double* x, double* r, double* p, double* rr_host, int* iter_host,
                          void* stream) {
  if (!h || !x || !r || !p || !rr_host || !iter_host) return fail(SIP_ERR_ARG, "null argument");
  const Checkpoint* c = checkpoint_at(h, slot);
  if (!c) return fail(SIP_ERR_ARG, "checkpoint slot out of range");
  if (c->mode != SIP_CG_FP64 || c->nrhs != 1)
    return fail(SIP_ERR_ARG, "sip_cg_checkpoint_get copies FP64 single-RHS states; use sip_cg_checkpoint_replay");
  const size_t bytes = sizeof(double) * h->plan.ndof;
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemcpyAsync(x, c->x, bytes, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(r, c->r, bytes, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(p, c->p, bytes, cudaMemcpyDeviceToDevice, s);
  *rr_host = c->scal[S_RR];
  *iter_host = c->iter;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIP_OK : cuda_fail(e, "checkpoint copy");
}

int sip_cg_checkpoint_info(const sip_handle* h, int slot, sip_checkpoint_info* out) {
  if (!h || !out) return fail(SIP_ERR_ARG, "null argument");
  const Checkpoint* c = checkpoint_at(h, slot);
  if (!c) return fail(SIP_ERR_ARG, "checkpoint slot out of range");
  out->iteration = c->iter;
  out->refinements = c->refinements;
  out->restarts = c->restarts;
  out->mode = c->mode;
  out->nrhs = c->nrhs;
  out->transpose = c->transpose;
  return SIP_OK;
}

int sip_cg_checkpoint_iterate(sip_handle* h, int slot, double* x_dev, void* stream) {
  if (!h || !x_dev) return fail(SIP_ERR_ARG, "null argument");
  const Checkpoint* c = checkpoint_at(h, slot);
  if (!c) return fail(SIP_ERR_ARG, "checkpoint slot out of range");
  cudaError_t e = cudaMemcpyAsync(x_dev, c->x, sizeof(double) * h->plan.ndof * c->nrhs, cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream);
  return e == cudaSuccess ? SIP_OK : cuda_fail(e, "checkpoint copy");
}

int sip_cg_checkpoint_replay(sip_handle* h, int slot, int iters, double* x_dev, void* stream) {
  NvtxRange range("sip_cg_checkpoint_replay");
  if (!h || !x_dev || iters < 0) return fail(SIP_ERR_ARG, "bad argument");
  if (h->p2p()) return fail(SIP_ERR_ARG, "CG needs the symmetric shared-rule operator (face_scheme SIP_FACES_SHARED)");
  const Checkpoint* cp = checkpoint_at(h, slot);
  if (!cp) return fail(SIP_ERR_ARG, "checkpoint slot out of range");
  const Checkpoint c = *cp;  // the ring is not touched, but keep the fields stable
  const int nrhs = c.nrhs;
  int rc = ensure_solver(h, nrhs);
  if (rc) return rc;
  cudaStream_t s = h->solve_stream;
  cudaStream_t user = (cudaStream_t)stream;
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, user);
  cudaStreamWaitEvent(s, ev, 0);
  const size_t n = (size_t)h->plan.ndof * nrhs;
  const bool fp64 = c.mode == SIP_CG_FP64;
  CgWork& W = fp64 ? h->cg64 : h->cg32;
  rc = ensure_cg(h, W, fp64 ? sizeof(double) : sizeof(float), nrhs);
  if (rc == SIP_OK) {
    const size_t es = fp64 ? sizeof(double) : sizeof(float);
    double* xit = fp64 ? (double*)W.x : h->x64;
    cudaMemcpyAsync(xit, c.x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(W.r, c.r, n * es, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(W.p, c.p, n * es, cudaMemcpyDeviceToDevice, s);
    std::copy(c.scal.begin(), c.scal.end(), h->scal_host);
    int zero = 0;
    cudaMemcpyAsync(W.status, &zero, sizeof(int), cudaMemcpyHostToDevice, s);
    rc = write_scal(h, W, nrhs, s);
    if (rc == SIP_OK && fp64) {
      // the FP64 recurrence, chunked and masked as during the solve
      int done = 0;
      rc = cg_loop<double>(h, W, nrhs, SIP_FP64, c.transpose, c.tol, iters, &done, s,
                           h->plan.opt.checkpoint_every, CkCtx{});
    } else if (rc == SIP_OK) {
      // the FP32 recurrence of the refined mode (FP64 iterate), in chunks
      const int chunk = std::max(1, h->plan.opt.check_every);
      W.xext = h->x64;
      for (int done = 0; done < iters && rc == SIP_OK; done += chunk)
        rc = run_iters<float>(h, W, nrhs, SIP_FP32, c.transpose, std::min(chunk, iters - done), s,
                              iters - done >= chunk);
      W.xext = nullptr;
    }
    if (rc == SIP_OK) cudaMemcpyAsync(x_dev, xit, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  cudaEventRecord(ev, s);
  cudaStreamWaitEvent(user, ev, 0);
  cudaError_t e = cudaStreamSynchronize(s);
  cudaEventDestroy(ev);
  if (rc) return rc;
  return e == cudaSuccess ? SIP_OK : cuda_fail(e, "checkpoint replay");
}

int sip_cg_replay(sip_handle* h, double* x, double* r, double* p, double* rr_host, int iters, void* stream) {
  if (!h || !x || !r || !p || !rr_host || iters < 0) return fail(SIP_ERR_ARG, "bad argument");
  if (h->p2p()) return fail(SIP_ERR_ARG, "CG needs the symmetric shared-rule operator (face_scheme SIP_FACES_SHARED)");
  int rc = ensure_solver(h, 1);
  if (rc) return rc;
  rc = ensure_cg(h, h->cg64, sizeof(double), 1);
  if (rc) return rc;
  CgWork& W = h->cg64;
  cudaStream_t s = h->solve_stream;
  cudaStream_t user = (cudaStream_t)stream;
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, user);
  cudaStreamWaitEvent(s, ev, 0);
  const size_t bytes = sizeof(double) * h->plan.ndof;
  cudaMemcpyAsync(W.x, x, bytes, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(W.r, r, bytes, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(W.p, p, bytes, cudaMemcpyDeviceToDevice, s);
  double* sc = h->scal_host;
  std::fill(sc, sc + kScal, 0.0);
  sc[S_RR] = *rr_host;
  sc[S_ACTIVE] = 1.0;
  int zero = 0;
  cudaMemcpyAsync(W.status, &zero, sizeof(int), cudaMemcpyHostToDevice, s);
  rc = write_scal(h, W, 1, s);
  if (rc == SIP_OK) rc = run_iters<double>(h, W, 1, SIP_FP64, 0, iters, s, false);
  if (rc == SIP_OK) {
    cudaMemcpyAsync(x, W.x, bytes, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(r, W.r, bytes, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(p, W.p, bytes, cudaMemcpyDeviceToDevice, s);
    int st = 0;
    rc = read_scal(h, W, 1, s, &st);
    if (rc == SIP_OK) *rr_host = h->scal_host[S_RR];
  }
  cudaEventRecord(ev, s);
  cudaStreamWaitEvent(user, ev, 0);
  cudaStreamSynchronize(s);
  cudaEventDestroy(ev);
  return rc;
}

int sip_set_kappa(sip_handle* h, const double* kappa, void* stream) {
  if (!h) return fail(SIP_ERR_ARG, "null handle");
  cudaStream_t s = (cudaStream_t)stream;
  for (auto* W : {&h->cg64, &h->cg32})
    if (W->graph) { cudaGraphExecDestroy(W->graph); W->graph = nullptr; }
  if (!kappa) { h->kappa_set = false; return SIP_OK; }
  const int64_t n = h->plan.nquad;
  cudaMemcpyAsync(h->gd.kappa, kappa, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  k_d2f<<<vgrid(n, 1), 256, 0, s>>>(h->gd.kappa, h->gf.kappa, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "set kappa");
  h->kappa_set = true;
  return SIP_OK;
}

int sip_grad_kappa(sip_handle* h, const double* ybar, const double* x, double* kbar, int accumulate, void* stream) {
  if (!h || !ybar || !x || !kbar) return fail(SIP_ERR_ARG, "null argument");
  AuxArgs a{};
  a.a = ybar;
  a.b = x;
  a.out = kbar;
  a.accumulate = accumulate;
  a.mode = 0;
  return launch_aux(h, a, (cudaStream_t)stream);
}

int sip_mass_dot(sip_handle* h, const double* av, const double* bv, double* out, void* stream) {
  if (!h || !av || !bv || !out) return fail(SIP_ERR_ARG, "null argument");
  int rc = ensure_solver(h, 1);
  if (rc) return rc;
  AuxArgs a{};
  a.a = av;
  a.b = bv;
  a.out = h->red;
  a.mode = 1;
  cudaStream_t s = (cudaStream_t)stream;
  rc = launch_aux(h, a, s);
  if (rc) return rc;
  // fixed-order final sum of the per-tile partials, straight into *out
  const int nt = (int)h->tiles_h[0].size();
  static_assert(S_RR == 0, "slot 0");
  // reuse k_final in "store" mode with a 1-RHS scalar block at h->red + nt
  k_final<<<1, kRedThreads, 0, s>>>(h->red, nt, h->red + nt, 0, 0, nullptr);
  cudaMemcpyAsync(out, h->red + nt, sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SIP_OK : cuda_fail(e, "mass dot");
}

int sip_iproduct(sip_handle* h, const double* f, double* b, void* stream) {
  if (!h || !f || !b) return fail(SIP_ERR_ARG, "null argument");
  AuxArgs a{};
  a.a = f;
  a.out = b;
  a.mode = 2;
  return launch_aux(h, a, (cudaStream_t)stream);
}

int sip_quad_points(sip_handle* h, double* xq, void* stream) {
  if (!h || !xq) return fail(SIP_ERR_ARG, "null argument");
  cudaError_t e = cudaMemcpyAsync(xq, h->xq, sizeof(double) * h->plan.nquad * h->plan.dim, cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream);
  return e == cudaSuccess ? SIP_OK : cuda_fail(e, "quad points");
}

int sip_work_model(const sip_handle* h, int precision, sip_work* out) {
  if (!h || !out) return fail(SIP_ERR_ARG, "null argument");
  const Plan& p = h->plan;
  const double es = precision == SIP_FP32 ? 4.0 : 8.0;
  double ft = 0.0, fm = 0.0;
  for (int64_t e = 0; e < p.E; ++e) {
    double a = 0.0, b = 0.0;
    element_flops(p, e, a, b);
    ft += a;
    fm += b;
  }
  out->flops_trace = ft;
  out->flops_main = fm;
  out->bytes_x = es * p.ndof;
  out->bytes_y = es * p.ndof;
  out->bytes_geometry = es * (p.vgeo.size() + p.fgeo.size() + p.f_tau.size());
  out->bytes_trace = 2.0 * es * 4.0 * p.trace_points;
  return SIP_OK;
}

}  // extern "C"
