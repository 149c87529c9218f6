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
//
// Set-up happens in tnc_plan_upload, which allocates anyway: for a plan
// whose workspace fits the array it loads every kernel of the library onto
// the device and resolves the array's device address there, once per device.
// With lazy module loading (the CUDA default) both would otherwise happen at
// the first use on that device, and both take device memory (the array
// itself is allocated when its module is loaded).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>

#include "devonce.cuh"
#include "tnc_internal.h"

namespace tnc {
int run_request(tnc_plan_t* plan, const uint8_t* host_bits, int batch, void* d_out, void* d_ws, size_t ws_bytes,
                void* stream);
}

namespace {

constexpr size_t kStaticWsBytes = (size_t)64 << 20;

// The workspace.  In host code `g_static_ws` only names a host-side stand-in;
// its device address comes from cudaGetSymbolAddress (per device).
static __device__ __align__(256) unsigned char g_static_ws[kStaticWsBytes];

std::mutex g_mu;
std::atomic<void*> g_ws_addr[tnc::kMaxDevices];
std::string g_setup_error[tnc::kMaxDevices];  // guarded by g_mu

}  // namespace

namespace tnc {

int preload_kernels_core();
int preload_kernels_tc();

size_t static_workspace_bytes() { return kStaticWsBytes; }

// Set-up of the static workspace on device `dev`, which must be current:
// every kernel loaded, the array's address resolved.  Called by
// tnc_plan_upload; idempotent.
int prepare_static_workspace(int dev) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("static workspace: device %d out of range", dev);
    return TNC_EINVAL;
  }
  if (g_ws_addr[dev].load(std::memory_order_acquire)) return TNC_OK;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_ws_addr[dev].load(std::memory_order_acquire)) return TNC_OK;
  int r = preload_kernels_core();
  if (!r) r = preload_kernels_tc();
  void* ptr = nullptr;
  cudaError_t e = r ? (cudaError_t)r : cudaGetSymbolAddress(&ptr, g_static_ws);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", r ? "loading the kernels" : "cudaGetSymbolAddress",
             cudaGetErrorString(e));
    g_setup_error[dev] = buf;
    set_error("static workspace set-up on device %d: %s", dev, buf);
    return TNC_ECUDA;
  }
  g_setup_error[dev].clear();
  g_ws_addr[dev].store(ptr, std::memory_order_release);
  return TNC_OK;
}

}  // namespace tnc

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
  if (attr.device < 0 || attr.device >= tnc::kMaxDevices) {
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
  // set up by tnc_plan_upload (this call only reads the cached address)
  void* ws = g_ws_addr[attr.device].load(std::memory_order_acquire);
  if (!ws) {
    std::lock_guard<std::mutex> lk(g_mu);
    tnc::set_error("tnc_contract_amplitudes_static: the static workspace of device %d is not set up (%s)",
                   attr.device,
                   g_setup_error[attr.device].empty() ? "tnc_plan_upload sets it up"
                                                      : g_setup_error[attr.device].c_str());
    return TNC_ESTATE;
  }
  return tnc::run_request(plan, bits, batch, d_out, ws, kStaticWsBytes, stream);
}
