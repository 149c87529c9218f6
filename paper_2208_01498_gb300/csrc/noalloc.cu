// Contraction into a workspace that the library owns statically.
//
// Some callers cannot allocate device memory at the moment they need
// amplitudes: code inside a host framework whose caching allocator owns all
// device memory and must not be bypassed, latency-bound request handlers
// that may not call cudaMalloc/cudaFree (both can synchronise the whole
// device), or plugins whose host process forbids new allocations after
// start-up.
// tnc_contract_amplitudes_static serves them: it runs the same node program
// as tnc_contract_amplitudes, but its workspace is the file-scope array
// below, so the call itself allocates nothing (no cudaMalloc, no cudaFree, no
// allocating library routine).
//
// The array is kStaticWsBytes (64 MiB) and lives on every GPU that loads
// this library until the process exits.  Plans whose workspace is larger are
// rejected with TNC_ENOMEM.  All calls share the array and it keeps the
// contents of the last call; the executor clears what must start at zero (the
// staged bitstrings and the output) on every call.  Calls whose work overlaps
// on the GPU (two streams, or two host threads) race on the array and give
// wrong results: serialise them.
#include <cuda_runtime.h>

#include <mutex>

#include "tnc_internal.h"

namespace tnc {
int run_request(tnc_plan_t* plan, const uint8_t* host_bits, int batch, void* d_out, void* d_ws, size_t ws_bytes,
                void* stream);
}

namespace {

constexpr size_t kStaticWsBytes = (size_t)64 << 20;
constexpr int kMaxDevices = 64;

// The workspace.  In host code `g_static_ws` only names a host-side stand-in;
// its device address comes from cudaGetSymbolAddress (per device).
static __device__ __align__(256) unsigned char g_static_ws[kStaticWsBytes];

std::mutex g_mu;
void* g_ws_addr[kMaxDevices] = {};

// Device address of the array on device `dev` (which must be current); the
// first call on a device looks it up once.
int static_ws(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ws_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_ws);
    if (e != cudaSuccess) {
      tnc::set_error("tnc_contract_amplitudes_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return TNC_ECUDA;
    }
    g_ws_addr[dev] = ptr;
  }
  *out = g_ws_addr[dev];
  return TNC_OK;
}

}  // namespace

extern "C" int tnc_contract_amplitudes_static(tnc_plan_t* plan, const uint8_t* bits, int batch, void* d_out,
                                              void* stream) {
  if (!plan || !bits || !d_out) {
    tnc::set_error("tnc_contract_amplitudes_static: NULL argument");
    return TNC_EINVAL;
  }
  tnc::Plan& p = plan->p;
  if (p.prog.ws_bytes > kStaticWsBytes) {
    tnc::set_error("tnc_contract_amplitudes_static: the plan needs a %llu-byte workspace; the static workspace "
                   "holds %zu bytes (use tnc_contract_amplitudes with a caller workspace)",
                   (unsigned long long)p.prog.ws_bytes, kStaticWsBytes);
    return TNC_ENOMEM;
  }
  // the device is the one that owns the output
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, d_out) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    tnc::set_error("tnc_contract_amplitudes_static: d_out is not device memory");
    return TNC_EINVAL;
  }
  if (attr.device < 0 || attr.device >= kMaxDevices) {
    tnc::set_error("tnc_contract_amplitudes_static: device %d out of range", attr.device);
    return TNC_EINVAL;
  }
  cudaError_t e = cudaSetDevice(attr.device);
  if (e != cudaSuccess) {
    tnc::set_error("tnc_contract_amplitudes_static: cudaSetDevice: %s", cudaGetErrorString(e));
    return TNC_ECUDA;
  }
  // uploading the plan allocates: it must have happened before
  if (!p.d_base || p.device != attr.device) {
    tnc::set_error("tnc_contract_amplitudes_static: plan is not resident on device %d; call tnc_plan_upload "
                   "first (this entry point allocates nothing)",
                   attr.device);
    return TNC_ESTATE;
  }
  if (p.profiling) {
    tnc::set_error("tnc_contract_amplitudes_static: disable profiling first (it creates CUDA events)");
    return TNC_ESTATE;
  }
  void* ws = nullptr;
  int rc = static_ws(attr.device, &ws);
  if (rc != TNC_OK) return rc;
  return tnc::run_request(plan, bits, batch, d_out, ws, kStaticWsBytes, stream);
}
