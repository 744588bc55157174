// zbc_rmatvec_noalloc: the FP32 adjoint product Psi = Z^H Phi with no memory allocation.
//
// Some callers cannot allocate device memory when they need the product: real-time loops and
// embedded users whose memory is fixed up front, allocator hooks that must not re-enter the
// allocator, and code running while a stream is captured (cudaMalloc is not permitted there).
// zbc_rmatvec keeps its partial sums in a per-handle buffer that grows on demand; this variant
// instead uses one fixed scratch array compiled into the library (kScratchBytes = 16 MiB of
// device memory, held by every GPU that loads the library until the process exits).
//
// The array's host-side name is only a stand-in: its device address is taken once per device
// with cudaGetSymbolAddress, on the first call made while that device is current, and kept for
// the life of the process (a cudaDeviceReset would make it stale).  That first call should
// therefore happen before any stream capture begins.  Every call shares the array and it keeps
// the last call's contents; each call overwrites every entry it reads, so nothing needs
// clearing, but two calls that overlap on the GPU (different streams, different threads) race
// on it.
#include <mutex>

#include "zbc_internal.cuh"

namespace zbc {

int rmatvec_simt_scratch(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo,
                         float2* scratch, size_t scratch_bytes, cudaStream_t st);
int aca_post(const Handle& h, const float2* Psip, int p, float2* Psi, int64_t ldpsi, cudaStream_t st);

constexpr size_t kScratchBytes = (size_t)16 << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_noalloc_scratch[kScratchBytes / sizeof(float2)];

static std::mutex g_scratch_mu;
static float2* g_scratch_addr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (looked up once per device)
static int scratch_address(float2** out) {
  int dev = 0;
  ZBC_TRY_CUDA(cudaGetDevice(&dev));
  ZBC_CHECK_ARG(dev >= 0 && dev < kMaxDevices, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      set_error("cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
      return ZBC_ECUDA;
    }
    g_scratch_addr[dev] = (float2*)p;
  }
  *out = g_scratch_addr[dev];
  return ZBC_OK;
}

}  // namespace zbc

using namespace zbc;

extern "C" int zbc_rmatvec_noalloc(const zbc_handle* hh, const void* Phi, int64_t ldphi, int p, void* Psi,
                                   int64_t ldpsi, zbc_stream stream) {
  clear_error();
  ZBC_CHECK_ARG(hh && Phi && Psi, "zbc_rmatvec_noalloc: null argument");
  Handle& h = const_cast<zbc_handle*>(hh)->h;
  ZBC_CHECK_ARG(p >= 1 && p <= 1024, "p must be in [1, 1024] (got %d)", p);
  ZBC_CHECK_ARG(ldphi >= (int64_t)h.q * h.nv(), "ldphi < q*n_v");
  ZBC_CHECK_ARG(ldpsi >= h.m, "ldpsi (%lld) < m (%d)", (long long)ldpsi, h.m);
  // scratch use: one group of partial sums (q*M*p) at least, plus Psi' (M*p) for ACA storage
  const size_t aca_bytes = h.has_v ? sizeof(float2) * (size_t)h.M * p : 0;
  const size_t group_bytes = sizeof(float2) * (size_t)h.q * h.M * p;
  ZBC_CHECK_ARG(aca_bytes + group_bytes <= kScratchBytes,
                "zbc_rmatvec_noalloc: M*p = %d*%d needs %zu bytes of scratch, more than its fixed %zu bytes; use "
                "zbc_rmatvec or fewer right-hand sides per call",
                h.M, p, aca_bytes + group_bytes, kScratchBytes);
  float2* scratch = nullptr;
  ZBC_TRY(scratch_address(&scratch));
  float2* psi_p = (float2*)Psi;
  int64_t ldo = ldpsi;
  if (h.has_v) {
    psi_p = scratch + (kScratchBytes - aca_bytes) / sizeof(float2);
    ldo = h.M;
  }
  ZBC_TRY(rmatvec_simt_scratch(h, (const float2*)Phi, ldphi, p, psi_p, ldo, scratch, kScratchBytes - aca_bytes,
                               stream));
  if (h.has_v) return aca_post(h, psi_p, p, (float2*)Psi, ldpsi, stream);
  return ZBC_OK;
}
