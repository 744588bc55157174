// zbc_matvec / zbc_rmatvec: argument checks, the ACA pre/post products (Sec. III.B) and
// dispatch to the arithmetic form (FP32 SIMT or a tensor-core form).
#include "zbc_internal.cuh"

namespace zbc {
int matvec_simt(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st);
int rmatvec_simt(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo, cudaStream_t st);
int matvec_tc(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, zbc_precision prec,
              cudaStream_t st);
int rmatvec_tc(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo, zbc_precision prec,
               cudaStream_t st);
int aca_pre(const Handle& h, const float2* X, int64_t ldx, int p, float2* Xp, cudaStream_t st);
int aca_post(const Handle& h, const float2* Psip, int p, float2* Psi, int64_t ldpsi, cudaStream_t st);
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
  ZBC_CHECK_ARG(prec == ZBC_FP32_SIMT || prec == ZBC_TF32X3 || prec == ZBC_BF16X3, "unknown precision %d", (int)prec);
  const float2* Xe = (const float2*)X;
  int64_t ldxe = ldx;
  if (h.has_v) {
    ZBC_TRY(h.work_x.ensure(sizeof(float2) * (size_t)h.M * p));
    ZBC_TRY(aca_pre(h, (const float2*)X, ldx, p, (float2*)h.work_x.ptr, stream));
    Xe = (const float2*)h.work_x.ptr;
    ldxe = h.M;
  }
  if (prec == ZBC_FP32_SIMT) return matvec_simt(h, Xe, ldxe, p, (float2*)Y, ldy, stream);
  return matvec_tc(h, Xe, ldxe, p, (float2*)Y, ldy, prec, stream);
}

extern "C" int zbc_rmatvec(const zbc_handle* hh, const void* Phi, int64_t ldphi, int p, void* Psi, int64_t ldpsi,
                           zbc_precision prec, zbc_stream stream) {
  clear_error();
  ZBC_CHECK_ARG(hh && Phi && Psi, "zbc_rmatvec: null argument");
  Handle& h = const_cast<zbc_handle*>(hh)->h;
  ZBC_CHECK_ARG(p >= 1 && p <= 1024, "p must be in [1, 1024] (got %d)", p);
  ZBC_CHECK_ARG(ldphi >= (int64_t)h.q * h.nv(), "ldphi < q*n_v");
  ZBC_CHECK_ARG(ldpsi >= h.m, "ldpsi (%lld) < m (%d)", (long long)ldpsi, h.m);
  ZBC_CHECK_ARG(prec == ZBC_FP32_SIMT || prec == ZBC_TF32X3 || prec == ZBC_BF16X3, "unknown precision %d", (int)prec);
  float2* out = (float2*)Psi;
  int64_t ldo = ldpsi;
  if (h.has_v) {
    ZBC_TRY(h.work_x.ensure(sizeof(float2) * (size_t)h.M * p));
    out = (float2*)h.work_x.ptr;
    ldo = h.M;
  }
  int s = prec == ZBC_FP32_SIMT ? rmatvec_simt(h, (const float2*)Phi, ldphi, p, out, ldo, stream)
                                : rmatvec_tc(h, (const float2*)Phi, ldphi, p, out, ldo, prec, stream);
  if (s != ZBC_OK) return s;
  if (h.has_v) return aca_post(h, out, p, (float2*)Psi, ldpsi, stream);
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
  set_error("a product kernel gave up a bounded device wait; its output is incomplete");
  return ZBC_ETIMEOUT;
}
