// Tensor-core forms of Algorithms 1 and 2 (tcgen05, sm_103a).
#include "zbc_internal.cuh"

namespace zbc {

struct TcPack {
  int dummy;
};

void tc_release(TcPack* p) { delete p; }

int matvec_tc(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, zbc_precision prec,
              cudaStream_t st) {
  set_error("tensor-core product path not built yet");
  return ZBC_EINVAL;
}

int rmatvec_tc(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo, zbc_precision prec,
               cudaStream_t st) {
  set_error("tensor-core product path not built yet");
  return ZBC_EINVAL;
}

}  // namespace zbc
