// zbc_rank_widths: sketch widths for the randomized Tucker from the rank-predictor MLP
// (no counterpart in the paper).  The MLP predicts, per column, log(rank) for the 9
// (component, mode) pairs; the width used is ceil(exp(prediction)) + oversample, clamped to
// [2, n_mode].
#include <cmath>

#include "zbc_internal.cuh"

namespace zbc {
struct Mlp;
int mlp_forward_dev(const Mlp* M, const float* X, int B, float* out, cudaStream_t st);
}  // namespace zbc

struct zbc_mlp;
namespace zbc {
const Mlp* mlp_of(const zbc_mlp* z);
}

using namespace zbc;

extern "C" int zbc_rank_widths(const zbc_mlp* model, const float* features, int ncols, const zbc_grid* g,
                               int oversample, int32_t* widths_host, zbc_stream stream) {
  clear_error();
  ZBC_CHECK_ARG(model && features && g && widths_host && ncols >= 1, "zbc_rank_widths: bad argument");
  ZBC_CHECK_ARG(oversample >= 0 && oversample <= 64, "oversample must be in [0, 64]");
  float* out = nullptr;
  ZBC_TRY_CUDA(cudaMalloc(&out, sizeof(float) * 9 * (size_t)ncols));
  int s = mlp_forward_dev(mlp_of(model), features, ncols, out, stream);
  std::vector<float> h(9 * (size_t)ncols);
  if (s == ZBC_OK) {
    cudaError_t e = cudaMemcpyAsync(h.data(), out, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
      set_error("zbc_rank_widths: %s", cudaGetErrorString(e));
      s = ZBC_ECUDA;
    }
  }
  cudaFree(out);
  if (s != ZBC_OK) return s;
  const int n[3] = {g->n1, g->n2, g->n3};
  for (int j = 0; j < ncols; ++j)
    for (int k = 0; k < 3; ++k)
      for (int m = 0; m < 3; ++m) {
        const double pred = std::exp((double)h[9 * (size_t)j + 3 * k + m]);
        int w = (int)std::ceil(std::min(pred, 1e6)) + oversample;
        w = std::max(2, std::min(w, n[m]));
        widths_host[9 * (size_t)j + 3 * k + m] = w;
      }
  return ZBC_OK;
}
