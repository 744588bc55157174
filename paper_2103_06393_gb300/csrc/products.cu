// zbc_matvec / zbc_rmatvec: argument checks, the ACA pre/post products (Sec. III.B), dispatch to
// the arithmetic form (FP32 SIMT or a tensor-core form), the autotuner and the product status.
#include <algorithm>
#include <cmath>

#include "decomp.cuh"
#include "zbc_internal.cuh"

namespace zbc {
int matvec_tc(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, zbc_precision prec,
              cudaStream_t st);
int matvec_tc2(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st);
int matvec_mode1(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st);
int matvec_dc(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st);
int aca_pre(const Handle& h, const float2* X, int64_t ldx, int p, float2* Xp, cudaStream_t st);
int aca_post(const Handle& h, const float2* Psip, int p, float2* Psi, int64_t ldpsi, cudaStream_t st);

// Y = Z X with an explicit form (prec != AUTO) and SIMT CTA shape
static int matvec_impl(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, zbc_precision prec,
                       int warps, cudaStream_t st) {
  const float2* Xe = X;
  int64_t ldxe = ldx;
  if (h.has_v) {
    ZBC_TRY(h.work_x.ensure(sizeof(float2) * (size_t)h.M * p));
    ZBC_TRY(aca_pre(h, X, ldx, p, (float2*)h.work_x.ptr, st));
    Xe = (const float2*)h.work_x.ptr;
    ldxe = h.M;
  }
  if (prec == ZBC_FP32_SIMT) return matvec_simt(h, Xe, ldxe, p, Y, ldy, warps, st);
  if (prec == ZBC_TC2) return matvec_tc2(h, Xe, ldxe, p, Y, ldy, st);
  if (prec == ZBC_TC_MODE1) return matvec_mode1(h, Xe, ldxe, p, Y, ldy, st);
  if (prec == ZBC_TC_DC) return matvec_dc(h, Xe, ldxe, p, Y, ldy, st);
  return matvec_tc(h, Xe, ldxe, p, Y, ldy, prec, st);
}

// Psi = Z^H Phi with an explicit form: FP32_SIMT (with `warps` compute warps) or TC_MODE1
static int rmatvec_impl(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* Psi, int64_t ldpsi,
                        zbc_precision prec, int warps, cudaStream_t st) {
  float2* out = Psi;
  int64_t ldo = ldpsi;
  if (h.has_v) {
    ZBC_TRY(h.work_x.ensure(sizeof(float2) * (size_t)h.M * p));
    out = (float2*)h.work_x.ptr;
    ldo = h.M;
  }
  if (prec == ZBC_TC_MODE1)
    ZBC_TRY(rmatvec_mode1(h, Phi, ldphi, p, out, ldo, st));
  else
    ZBC_TRY(rmatvec_simt(h, Phi, ldphi, p, out, ldo, warps, st));
  if (h.has_v) return aca_post(h, out, p, Psi, ldpsi, st);
  return ZBC_OK;
}
}  // namespace zbc

using namespace zbc;

extern "C" int zbc_matvec(const zbc_handle* hh, const void* X, int64_t ldx, int p, void* Y, int64_t ldy,
                          zbc_precision prec, zbc_stream stream) {
  clear_error();
  ZBC_CHECK_ARG(hh && X && Y, "zbc_matvec: null argument");
  Handle& h = const_cast<zbc_handle*>(hh)->h;
  ZBC_CHECK_ARG(p >= 1 && p <= 1024, "p must be in [1, 1024] (got %d)", p);
  ZBC_CHECK_ARG(ldx >= h.m, "ldx (%lld) < m (%d)", (long long)ldx, h.m);
  ZBC_CHECK_ARG(ldy >= (int64_t)h.q * h.nv(), "ldy < q*n_v");
  ZBC_CHECK_ARG(prec == ZBC_FP32_SIMT || prec == ZBC_TF32X3 || prec == ZBC_BF16X3 || prec == ZBC_AUTO ||
                    prec == ZBC_TC2 || prec == ZBC_TC_MODE1 || prec == ZBC_TC_DC,
                "unknown precision %d", (int)prec);
  const int cls = rhs_class(p);
  int warps = h.tune_fwd_warps[cls];
  if (prec == ZBC_AUTO)
    prec = h.tune_fwd_prec[cls] >= 0 ? (zbc_precision)h.tune_fwd_prec[cls] : (p >= 8 ? ZBC_BF16X3 : ZBC_FP32_SIMT);
  return matvec_impl(h, (const float2*)X, ldx, p, (float2*)Y, ldy, prec, warps, (cudaStream_t)stream);
}

extern "C" int zbc_rmatvec(const zbc_handle* hh, const void* Phi, int64_t ldphi, int p, void* Psi, int64_t ldpsi,
                           zbc_precision prec, zbc_stream stream) {
  clear_error();
  ZBC_CHECK_ARG(hh && Phi && Psi, "zbc_rmatvec: null argument");
  Handle& h = const_cast<zbc_handle*>(hh)->h;
  ZBC_CHECK_ARG(p >= 1 && p <= 1024, "p must be in [1, 1024] (got %d)", p);
  ZBC_CHECK_ARG(ldphi >= (int64_t)h.q * h.nv(), "ldphi < q*n_v");
  ZBC_CHECK_ARG(ldpsi >= h.m, "ldpsi (%lld) < m (%d)", (long long)ldpsi, h.m);
  ZBC_CHECK_ARG(prec == ZBC_FP32_SIMT || prec == ZBC_TF32X3 || prec == ZBC_BF16X3 || prec == ZBC_AUTO ||
                    prec == ZBC_TC2 || prec == ZBC_TC_MODE1 || prec == ZBC_TC_DC,
                "unknown precision %d", (int)prec);
  ZBC_CHECK_ARG(prec == ZBC_FP32_SIMT || prec == ZBC_AUTO || prec == ZBC_TC_MODE1,
                "the adjoint product's forms are ZBC_FP32_SIMT, ZBC_TC_MODE1 and ZBC_AUTO");
  const int cls = rhs_class(p);
  if (prec == ZBC_AUTO) prec = h.tune_adj_prec[cls] >= 0 ? (zbc_precision)h.tune_adj_prec[cls] : ZBC_FP32_SIMT;
  return rmatvec_impl(h, (const float2*)Phi, ldphi, p, (float2*)Psi, ldpsi, prec, h.tune_adj_warps[cls],
                      (cudaStream_t)stream);
}

// The per-handle operands of the forms that no tuned right-hand-side class selects (untuned
// classes fall back to BF16X3 or FP32_SIMT, which need none of them) are freed; a later call of
// such a form builds them again.  The decompression cache itself is kept.
static void release_unused_operands(Handle& h) {
  DecompCache* c = h.cache;
  if (!c) return;
  bool m1f = false, m1a = false, dc = false, tc2 = false;
  for (int i = 0; i < Handle::kPClasses; ++i) {
    m1f = m1f || h.tune_fwd_prec[i] == ZBC_TC_MODE1;
    dc = dc || h.tune_fwd_prec[i] == ZBC_TC_DC;
    tc2 = tc2 || h.tune_fwd_prec[i] == ZBC_TC2;
    m1a = m1a || h.tune_adj_prec[i] == ZBC_TC_MODE1;
  }
  if (c->mode1 && !m1f) mode1_fwd_release(c->mode1);
  if (c->mode1 && !m1f && !m1a) {
    mode1_release(c->mode1);
    c->mode1 = nullptr;
  }
  if (c->dc && !dc) {
    dc_release(c->dc);
    c->dc = nullptr;
  }
  if (!tc2) half_release(c);
}

extern "C" int zbc_tune(zbc_handle* hh, int p, zbc_stream stream, float* times_ms_host) {
  clear_error();
  ZBC_CHECK_ARG(hh, "zbc_tune: null handle");
  ZBC_CHECK_ARG(p >= 1 && p <= 1024, "p must be in [1, 1024] (got %d)", p);
  Handle& h = hh->h;
  const cudaStream_t st = (cudaStream_t)stream;
  const int64_t rows = (int64_t)h.q * h.nv();
  DevBuf X, Y, Phi, Psi;
  ZBC_TRY(X.ensure(sizeof(float2) * (size_t)h.m * p));
  ZBC_TRY(Psi.ensure(sizeof(float2) * (size_t)h.m * p));
  ZBC_TRY(Y.ensure(sizeof(float2) * (size_t)rows * p));
  ZBC_TRY(Phi.ensure(sizeof(float2) * (size_t)rows * p));
  ZBC_TRY_CUDA(cudaMemsetAsync(X.ptr, 0, X.bytes, st));
  ZBC_TRY_CUDA(cudaMemsetAsync(Phi.ptr, 0, Phi.bytes, st));
  cudaEvent_t e0, e1;
  ZBC_TRY_CUDA(cudaEventCreate(&e0));
  ZBC_TRY_CUDA(cudaEventCreate(&e1));
  struct Variant {
    bool fwd;
    zbc_precision prec;
    int warps;
  };
  constexpr int NV = 10, NF = 7;  // the first NF variants are forward forms
  const Variant vars[NV] = {{true, ZBC_FP32_SIMT, 6},  {true, ZBC_FP32_SIMT, 9},  {true, ZBC_TF32X3, 0},
                            {true, ZBC_BF16X3, 0},     {true, ZBC_TC2, 0},        {true, ZBC_TC_MODE1, 0},
                            {true, ZBC_TC_DC, 0},      {false, ZBC_FP32_SIMT, 6}, {false, ZBC_FP32_SIMT, 9},
                            {false, ZBC_TC_MODE1, 0}};
  // timing order: the tensor-core forms first, so that a slower form can be dropped after one
  // timed call once it is 1.5 times slower than the best of its direction so far
  const int order[NV] = {5, 6, 2, 3, 4, 0, 1, 9, 8, 7};
  float t[NV];
  float best[2] = {INFINITY, INFINITY};
  int status = ZBC_OK;
  for (int oi = 0; oi < NV && status == ZBC_OK; ++oi) {
    const int i = order[oi];
    const Variant& v = vars[i];
    auto run = [&]() {
      return v.fwd ? matvec_impl(h, (const float2*)X.ptr, h.m, p, (float2*)Y.ptr, rows, v.prec, v.warps, st)
                   : rmatvec_impl(h, (const float2*)Phi.ptr, rows, p, (float2*)Psi.ptr, h.m, v.prec, v.warps, st);
    };
    t[i] = INFINITY;
    if (run() != ZBC_OK) {  // a form that does not fit this handle is skipped
      clear_error();
      continue;
    }
    float sum = 0.f;
    int s = ZBC_OK, reps = 0;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < 2 && s == ZBC_OK && e == cudaSuccess; ++r) {
      e = cudaEventRecord(e0, st);
      s = run();
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      sum += ms;
      ++reps;
      if (ms > 1.5f * best[v.fwd ? 0 : 1]) break;
    }
    if (e != cudaSuccess) {
      set_error("zbc_tune: timing failed: %s", cudaGetErrorString(e));
      status = ZBC_ECUDA;
    } else if (s != ZBC_OK) {
      status = s;
    } else {
      t[i] = sum / (float)reps;
      best[v.fwd ? 0 : 1] = std::min(best[v.fwd ? 0 : 1], t[i]);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != ZBC_OK) return status;
  int bf = 0, ba = NF;
  for (int i = 1; i < NF; ++i)
    if (t[i] < t[bf]) bf = i;
  for (int i = NF + 1; i < NV; ++i)
    if (t[i] < t[ba]) ba = i;
  if (!(t[bf] < INFINITY) || !(t[ba] < INFINITY)) {
    set_error("zbc_tune: no product form fits this handle");
    return ZBC_EINVAL;
  }
  const int cls = rhs_class(p);
  h.tune_fwd_prec[cls] = (int8_t)vars[bf].prec;
  h.tune_fwd_warps[cls] = (int8_t)vars[bf].warps;
  h.tune_adj_prec[cls] = (int8_t)vars[ba].prec;
  // the SIMT CTA shape stays the faster of the two SIMT variants (zbc_rmatvec_noalloc uses it)
  h.tune_adj_warps[cls] = (int8_t)(t[NF + 1] < t[NF] ? 9 : 6);
  if (times_ms_host)
    for (int i = 0; i < NV; ++i) times_ms_host[i] = t[i];
  release_unused_operands(h);
  return ZBC_OK;
}

extern "C" int zbc_product_status(const zbc_handle* hh, zbc_stream stream) {
  clear_error();
  ZBC_CHECK_ARG(hh, "zbc_product_status: null handle");
  Handle& h = const_cast<zbc_handle*>(hh)->h;
  ZBC_TRY_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (!h.work_err.ptr) return ZBC_OK;  // no product has run yet
  int flag = 0;
  ZBC_TRY_CUDA(cudaMemcpy(&flag, h.work_err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
  if (!flag) return ZBC_OK;
  ZBC_TRY_CUDA(cudaMemset(h.work_err.ptr, 0, sizeof(int)));
  if (flag & kErrTimeout) {
    set_error("a product kernel gave up a bounded device wait; its output is incomplete%s",
              (flag & kErrNonFinite) ? " (and a NaN or Inf was read from X or Phi)" : "");
    return ZBC_ETIMEOUT;
  }
  set_error("a NaN or Inf was read from X or Phi; the products' outputs are not finite");
  return ZBC_ENAN;
}

extern "C" int zbc_test_wait_limit(zbc_handle* hh, uint32_t polls) {
  clear_error();
  ZBC_CHECK_ARG(hh, "zbc_test_wait_limit: null handle");
  hh->h.test_first_wait = polls;
  return ZBC_OK;
}
