// vsie_assemble_columns: columns of the coil-body coupling matrix (Sec. III.A; Eq. n6, Eq. nNt).
//
// Z[(k,v), e] = h^3 len_e [ (I + grad grad / k0^2) g(r_v - c_e) t_e ]_k with
// g = exp(-i k0 R)/(4 pi R) and, for x = k0 R and Rhat = (r_v - c_e)/R,
//   (I + grad grad/k0^2) g = g [ (1 - i/x - 1/x^2) I + (-1 + 3i/x + 3/x^2) Rhat Rhat^T ].
// One thread per voxel, one grid row per requested column; FP64 arithmetic throughout.
#include <cmath>

#include "zbc_internal.cuh"

namespace zbc {

template <typename OutT>
__global__ void __launch_bounds__(256) assemble_kernel(int n1, int n2, int n3, double h, double mask_r,
                                                       const double* __restrict__ centre,
                                                       const double* __restrict__ tangent,
                                                       const double* __restrict__ length, double k0,
                                                       const int32_t* __restrict__ cols, int m,
                                                       OutT* __restrict__ out, int64_t ld) {
  const int64_t nv = (int64_t)n1 * n2 * n3;
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int jj = blockIdx.y;
  const int e = cols[jj];
  if (v >= nv) return;
  const bool valid = e >= 0 && e < m;
  const int i1 = (int)(v % n1);
  const int i2 = (int)((v / n1) % n2);
  const int i3 = (int)(v / ((int64_t)n1 * n2));
  // voxel centre, same rounding as the definition ((i - (n-1)/2) * h)
  const double x = __dmul_rn((double)i1 - (n1 - 1) / 2.0, h);
  const double y = __dmul_rn((double)i2 - (n2 - 1) / 2.0, h);
  const double z = __dmul_rn((double)i3 - (n3 - 1) / 2.0, h);
  OutT* o = out + ld * jj + v;
  bool masked = false;
  if (mask_r > 0.0) masked = sqrt(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y))) > mask_r;
  if (!valid) masked = true;  // an out-of-range column index yields a zero column
  double re[3] = {0, 0, 0}, im[3] = {0, 0, 0};
  if (!masked) {
    const double Rx = x - centre[3 * e + 0], Ry = y - centre[3 * e + 1], Rz = z - centre[3 * e + 2];
    const double R = sqrt(Rx * Rx + Ry * Ry + Rz * Rz);
    const double iR = 1.0 / R;
    const double hx = Rx * iR, hy = Ry * iR, hz = Rz * iR;
    const double tx = tangent[3 * e + 0], ty = tangent[3 * e + 1], tz = tangent[3 * e + 2];
    const double kr = k0 * R, ikr = 1.0 / kr, ikr2 = ikr * ikr;
    double s, c;
    sincos(kr, &s, &c);
    const double scale = h * h * h * length[e] / (4.0 * M_PI * R);
    // g * scale = scale * (c - i s)
    const double gr = scale * c, gi = -scale * s;
    // a = (1 - 1/x^2) - i/x ; b = (-1 + 3/x^2) + 3i/x
    const double ar = 1.0 - ikr2, ai = -ikr;
    const double br = -1.0 + 3.0 * ikr2, bi = 3.0 * ikr;
    const double ht = hx * tx + hy * ty + hz * tz;
    const double tk[3] = {tx, ty, tz}, hk[3] = {hx, hy, hz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double ur = ar * tk[k] + br * hk[k] * ht;
      const double ui = ai * tk[k] + bi * hk[k] * ht;
      re[k] = gr * ur - gi * ui;
      im[k] = gr * ui + gi * ur;
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if constexpr (sizeof(OutT) == 16) {
      o[k * nv] = OutT{re[k], im[k]};
    } else {
      o[k * nv] = OutT{(float)re[k], (float)im[k]};
    }
  }
}

}  // namespace zbc

using namespace zbc;

extern "C" int vsie_assemble_columns(const zbc_grid* g, const zbc_segments* s, double freq_hz,
                                     const int32_t* cols, int ncols, int q, void* out, int64_t ld,
                                     zbc_dtype dt, zbc_stream stream) {
  clear_error();
  ZBC_CHECK_ARG(g && s && cols && out, "vsie_assemble_columns: null argument");
  ZBC_CHECK_ARG(q == 3, "q must be 3");
  ZBC_CHECK_ARG(g->n1 >= 1 && g->n2 >= 1 && g->n3 >= 1 && g->h > 0, "bad grid");
  ZBC_CHECK_ARG(s->m >= 1 && s->centre && s->tangent && s->length, "bad segments");
  ZBC_CHECK_ARG(ncols >= 0 && ncols <= 65535, "ncols must be in [0, 65535]");
  ZBC_CHECK_ARG(freq_hz > 0 && std::isfinite(freq_hz), "freq_hz must be positive");
  const int64_t nv = (int64_t)g->n1 * g->n2 * g->n3;
  ZBC_CHECK_ARG(ld >= 3 * nv, "ld (%lld) < q*n_v (%lld)", (long long)ld, (long long)(3 * nv));
  ZBC_CHECK_ARG(dt == ZBC_C64 || dt == ZBC_C128, "bad dtype");
  if (ncols == 0) return ZBC_OK;
  const double k0 = 2.0 * M_PI * freq_hz / 299792458.0;
  dim3 grid((unsigned)ceil_div(nv, 256), (unsigned)ncols);
  if (dt == ZBC_C128)
    assemble_kernel<double2><<<grid, 256, 0, stream>>>(g->n1, g->n2, g->n3, g->h, g->mask_radius, s->centre,
                                                       s->tangent, s->length, k0, cols, s->m,
                                                       (double2*)out, ld);
  else
    assemble_kernel<float2><<<grid, 256, 0, stream>>>(g->n1, g->n2, g->n3, g->h, g->mask_radius, s->centre,
                                                      s->tangent, s->length, k0, cols, s->m, (float2*)out,
                                                      ld);
  ZBC_TRY_CUDA(cudaGetLastError());
  return ZBC_OK;
}
