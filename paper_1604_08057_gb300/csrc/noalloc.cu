// ov_apply_H_noalloc: H(mu) psi (or H^dagger psi) in FP64 without allocating
// device memory.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// apply the operator -- for example a process whose framework allocator has
// already reserved (almost) all device memory for its own pool, so a direct
// cudaMalloc would fail or fragment it; or a latency-sensitive inner loop
// (a molecular-dynamics or Langevin integrator applying H every step) that
// cannot afford the implicit device synchronisation of cudaMalloc/cudaFree;
// or a plug-in running inside a host application that forbids device
// allocations after start-up.  The context-based ov_apply_H allocates (and
// grows) its workspace on first use, which these callers cannot accept.
//
// The layout-conversion workspace lives instead in one file-scope device
// array of OV_NOALLOC_SCRATCH_BYTES bytes.  Every GPU that loads this library
// holds that array until the process exits.  Host code cannot use the name
// of a __device__ array as a device address (it is only a host-side stand-in
// for the symbol), so the device address is looked up with
// cudaGetSymbolAddress once per device, the first time the entry point runs
// on that device, and cached.
#include <cmath>
#include <mutex>

#include "ov.h"
#include "kernels.h"

using namespace ov;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[OV_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device (set-up on first use).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return OV_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return OV_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return OV_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return OV_OK;
}

bool aligned16(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" int ov_apply_H_noalloc(const int32_t dims[4], const void* U, double mu, double m_w, int32_t nsrc,
                                  const void* in, void* out, int32_t dagger, void* stream) {
  // a launch error left pending by earlier, unrelated work on this thread is
  // cleared here, so that the status returned below belongs to this call
  cudaGetLastError();
  if (!dims || !aligned16(U) || !aligned16(in) || !aligned16(out) || nsrc < 1 || nsrc > 4096)
    return OV_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 1 || dims[i] > 4096) return OV_ERR_INVALID_ARG;
  if (!(std::isfinite(mu) && std::isfinite(m_w)) || 2.0 * m_w + 8.0 == 0.0) return OV_ERR_INVALID_ARG;
  const int64_t V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
  // Every site costs at least 72 + 2 * 24 doubles (576 bytes) of scratch, so this
  // bound alone keeps V small enough that `need` below cannot overflow (V <= 58254,
  // nsrc <= 4096) and every grid size fits its launch type.
  if (V > (int64_t)(OV_NOALLOC_SCRATCH_BYTES / 576u)) return OV_ERR_SCRATCH_LIMIT;
  // scratch: internal links (72 V doubles), packed input and output (24 V doubles per source, padded)
  const int64_t vs = ((24 * V + 63) / 64) * 64;
  const int64_t need = (72 * V + 2 * (int64_t)nsrc * vs) * (int64_t)sizeof(double);
  if (need > (int64_t)OV_NOALLOC_SCRATCH_BYTES) return OV_ERR_SCRATCH_LIMIT;
  void* base = nullptr;
  const int st = scratch_address(&base);
  if (st != OV_OK) return st;
  double* links = static_cast<double*>(base);
  double* pin = links + 72 * V;
  double* pout = pin + (int64_t)nsrc * vs;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Lat<double> L{};
  L.g.nx = dims[0]; L.g.ny = dims[1]; L.g.nz = dims[2]; L.g.nt = dims[3]; L.g.V = V;
  L.kappa = 1.0 / (2.0 * m_w + 8.0);
  L.ef = std::exp(mu);
  L.efinv = std::exp(-mu);
  L.u = links;
  L.nsrc = nsrc;
  L.k = 1;
  L.vs = vs;
  // every scratch word read below is written first in the same call: nothing needs clearing
  pack_links<double>(static_cast<const double*>(U), links, V, s);
  pack_spinors<double>(static_cast<const double*>(in), pin, nsrc, V, vs, s);
  apply_h<double>(L, pin, pout, dagger, s);
  unpack_spinors<double>(pout, static_cast<double*>(out), nsrc, V, vs, s);
  if (cudaGetLastError() != cudaSuccess) return OV_ERR_CUDA;
  return OV_OK;
}
