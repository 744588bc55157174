// Internal definitions shared by the translation units of libzbc (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/zbc.h"

namespace zbc {

// ---------------------------------------------------------------------------------------------
// error reporting: thread-local message, status codes only across the ABI
// ---------------------------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

#define ZBC_TRY_CUDA(expr)                                                                  \
  do {                                                                                      \
    cudaError_t _e = (expr);                                                                \
    if (_e != cudaSuccess) {                                                                \
      ::zbc::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__,     \
                       __LINE__);                                                           \
      return _e == cudaErrorMemoryAllocation ? ZBC_ENOMEM : ZBC_ECUDA;                       \
    }                                                                                       \
  } while (0)

#define ZBC_CHECK_ARG(cond, ...)                                                            \
  do {                                                                                      \
    if (!(cond)) {                                                                          \
      ::zbc::set_error(__VA_ARGS__);                                                        \
      return ZBC_EINVAL;                                                                    \
    }                                                                                       \
  } while (0)

#define ZBC_TRY(expr)             \
  do {                            \
    int _s = (expr);              \
    if (_s != ZBC_OK) return _s;  \
  } while (0)

// ---------------------------------------------------------------------------------------------
// device workspace that grows on demand and is freed with its owner
// ---------------------------------------------------------------------------------------------
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  int ensure(size_t need);  // grow-only; contents are not preserved
  void release();
  ~DevBuf() { release(); }
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

// ---------------------------------------------------------------------------------------------
// the compressed coupling matrix
// ---------------------------------------------------------------------------------------------
// Tensor t = j*q + k.  Pool layout per tensor (complex64): core G[a + r1(b + r2 c)], then
// U1 (n1 x r1), U2 (n2 x r2), U3 (n3 x r3) column-major.
struct TensorDesc {
  int64_t off;        // offset of the core in the pool (complex64 elements)
  int32_t r1, r2, r3;
  float scale_log2;   // floor(log2 ||G||_F), used for the per-column scaling of the fp16 path
};

// bits of a handle's device error word (work_err), read and cleared by zbc_product_status
constexpr int kErrTimeout = 1;    // a bounded wait gave up; the kernel's output is incomplete
constexpr int kErrNonFinite = 2;  // a NaN or Inf was read from X or Phi

// polls of the bounded mbarrier waits in the product kernels
constexpr uint32_t kWaitPolls = 40000000u;

struct DecompCache;  // W = G x2 U2 x3 U3 and tile-blocked U1 per tensor, built lazily (decomp_cache.cu)
void cache_release(DecompCache* c);
int64_t cache_bytes(const DecompCache* c);  // device bytes held by a cache (0 for null)

struct Handle {
  int n1 = 0, n2 = 0, n3 = 0, q = 0;
  int M = 0;          // stored columns
  int m = 0;          // columns of Z
  bool has_v = false;
  std::vector<int32_t> ranks;      // 3*M*q
  std::vector<TensorDesc> desc;    // M*q
  int64_t pool_elems = 0;
  float2* d_pool = nullptr;        // complex64 cores + factors
  TensorDesc* d_desc = nullptr;    // device copy of desc
  float2* d_v = nullptr;           // m x M complex64 (ACA) or null
  int max_rank = 0;
  // per-handle workspaces of the product calls (not thread-safe: one call at a time)
  DevBuf work_partial;   // adjoint partial sums
  DevBuf work_x;         // X' = V^H X (ACA), scaled operands
  DevBuf work_misc;
  DevBuf work_xt;        // X^T of the forward products (s-chunk padded rows)
  DevBuf work_err;       // int: error bits kErrTimeout / kErrNonFinite set by the product kernels
  DevBuf work_phi;       // mode-1 adjoint: fp16 operand blocks of Phi and their exponents
  DecompCache* cache = nullptr;
  int cache_r = 0;                 // largest r1 rounded up to 2 (cache row stride bound)
  // autotuned choices per right-hand-side class (zbc_tune; -1 / 0 = untuned)
  static constexpr int kPClasses = 8;
  int8_t tune_fwd_prec[kPClasses] = {-1, -1, -1, -1, -1, -1, -1, -1};
  int8_t tune_fwd_warps[kPClasses] = {0, 0, 0, 0, 0, 0, 0, 0};
  int8_t tune_adj_warps[kPClasses] = {0, 0, 0, 0, 0, 0, 0, 0};
  int8_t tune_adj_prec[kPClasses] = {-1, -1, -1, -1, -1, -1, -1, -1};
  // polls allowed to the first stage wait of each consumer warp of the next FP32 SIMT adjoint
  // launch (zbc_test_wait_limit; reset after that launch); kWaitPolls otherwise
  uint32_t test_first_wait = kWaitPolls;
  ~Handle();
  int64_t nv() const { return (int64_t)n1 * n2 * n3; }
  int upload();          // copy desc to device (pool already on device)
};

int handle_append(Handle* h, const std::vector<int32_t>& ranks, const float2* d_pool_new,
                  int64_t new_elems, int ncols, cudaStream_t st);

// ---------------------------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {  // a*b + c
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__host__ __device__ __forceinline__ float2 cfma_conj(float2 a, float2 b, float2 c) {  // conj(a)*b + c
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__host__ __device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 zfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__host__ __device__ __forceinline__ double2 zfma_conj(double2 a, double2 b, double2 c) {  // conj(a)*b + c
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Raise Kernel's dynamic shared-memory limit to `bytes` on the current device, once per device
// (the attribute is per device; the flags are per kernel and safe across threads).
template <auto Kernel>
int set_smem_limit(int bytes) {
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  ZBC_TRY_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return ZBC_OK;
  ZBC_TRY_CUDA(cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.fetch_or(bit, std::memory_order_release);
  return ZBC_OK;
}

// right-hand-side class of p: 1, 2, 3-4, 5-8, 9-16, 17-32, 33-64, 65+
inline int rhs_class(int p) {
  int c = 0;
  while (c < 7 && p > (1 << c)) ++c;
  return c;
}

int sm_count();

// FP32 products on a handle's stored columns (products_simt.cu); warps = compute warps per CTA
// (6 or 9, anything else 9).  X / Phi are the M-row operands (after V^H for ACA storage).
int matvec_simt(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, int warps, cudaStream_t st);
int rmatvec_simt(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo, int warps,
                 cudaStream_t st);
// the adjoint with the mode-1 product on the tensor cores (products_mode1.cu)
int rmatvec_mode1(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo, cudaStream_t st);

// number of kernels this library has launched (all entry points), for launch accounting
void count_launch(int n = 1);

}  // namespace zbc

struct zbc_handle {
  zbc::Handle h;
};
