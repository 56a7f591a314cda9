// sip_apply_static_scratch: the apply with its trace scratch in a file-scope
// device array instead of device memory from cudaMalloc.
//
// For callers that must not allocate device memory once they are running, for
// example a process whose device memory is entirely reserved by its own caching
// allocator, or a latency-critical loop that forbids cudaMalloc (which can also
// synchronise the device).  sip_apply allocates (and may re-grow) its trace
// buffer on the handle; this variant allocates nothing.  The paper has no
// counterpart: it is an interface convenience, not part of the method.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "handle.h"

namespace {

// 16 MiB per device, reserved by every GPU that loads the library until exit.
constexpr size_t kStaticTraceBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_trace_scratch[kStaticTraceBytes];

constexpr int kMaxDevices = 64;
void* g_trace_scratch_addr[kMaxDevices] = {};
std::mutex g_trace_scratch_mu;

}  // namespace

extern "C" int sip_apply_static_scratch(sip_handle* h, int precision, const void* x, void* y, int nrhs,
                                        void* stream) {
  if (!h || !x || !y) return sip::fail(SIP_ERR_ARG, "null handle or vector");
  if (nrhs < 1) return sip::fail(SIP_ERR_ARG, "nrhs must be >= 1");
  if (precision != SIP_FP64 && precision != SIP_FP32) return sip::fail(SIP_ERR_ARG, "precision");
  const size_t need = sip::apply_scratch_bytes(h, precision, nrhs, nullptr);
  if (need > kStaticTraceBytes)
    return sip::fail(SIP_ERR_ARG, "sip_apply_static_scratch: this mesh and nrhs need " + std::to_string(need) +
                                      " bytes of trace scratch, above the static limit of " +
                                      std::to_string(kStaticTraceBytes) + " bytes; use sip_apply");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sip::cuda_fail(e, "sip_apply_static_scratch: cudaGetDevice");
  if (dev != h->device) return sip::fail(SIP_ERR_ARG, "the handle was created on another device");
  if (dev < 0 || dev >= kMaxDevices) return sip::fail(SIP_ERR_ARG, "device index out of range");
  void* scratch = nullptr;
  {
    // set-up, once per device, with that device current: the host-side name of
    // the array is not a device address, so ask the runtime for the address
    std::lock_guard<std::mutex> lock(g_trace_scratch_mu);
    if (!g_trace_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_trace_scratch);
      if (e != cudaSuccess) return sip::cuda_fail(e, "sip_apply_static_scratch: cudaGetSymbolAddress");
      g_trace_scratch_addr[dev] = p;
    }
    scratch = g_trace_scratch_addr[dev];
  }
  // k_trace writes every scratch entry that k_main then reads, so the scratch
  // needs no clearing between calls.
  return sip::apply_any(h, precision, x, y, nrhs, (cudaStream_t)stream, 0, scratch);
}
