// vsie_assemble_columns(_op): columns of the coil-body coupling matrix (Sec. III.A; Eq. n6,
// Eq. nNt, Eq. nKt).  One thread per voxel, one grid row per requested column; FP64 arithmetic
// (green.cuh).
#include "green.cuh"

namespace zbc {

// Q = 3: piecewise-constant basis (rows k n_v + v); Q = 12: piecewise-linear (rows b n_v + v)
template <typename OutT, int Q>
__global__ void __launch_bounds__(256) assemble_kernel(GreenGeom G, const int32_t* __restrict__ cols,
                                                       OutT* __restrict__ out, int64_t ld) {
  const int64_t nv = (int64_t)G.n1 * G.n2 * G.n3;
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const int jj = blockIdx.y;
  double2 z[Q];
  if constexpr (Q == 12)
    pwl_entry(G, v, cols[jj], z);
  else if (G.op == 0 && G.nq == 1)
    green_entry(G, v, cols[jj], z);
  else
    segment_entry(G, v, cols[jj], z);
  OutT* o = out + ld * jj + v;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    if constexpr (sizeof(OutT) == 16) {
      o[k * nv] = z[k];
    } else {
      o[k * nv] = OutT{(float)z[k].x, (float)z[k].y};
    }
  }
}

GreenGeom make_green(const zbc_grid* g, const zbc_segments* s, double freq_hz) {
  GreenGeom G;
  G.n1 = g->n1;
  G.n2 = g->n2;
  G.n3 = g->n3;
  G.h = g->h;
  G.mask_r = g->mask_radius;
  G.mask_b = g->mask_box;
  G.k0 = wavenumber(freq_hz);
  G.centre = s->centre;
  G.tangent = s->tangent;
  G.length = s->length;
  G.m = s->m;
  G.op = 0;
  G.nq = 1;
  G.qx[0] = 0.0;
  G.qw[0] = 2.0;
  return G;
}

int assemble_columns_c128(const GreenGeom& G, const int32_t* cols, int ncols, double2* out, int64_t ld,
                          cudaStream_t st) {
  const int64_t nv = (int64_t)G.n1 * G.n2 * G.n3;
  dim3 grid((unsigned)ceil_div(nv, 256), (unsigned)ncols);
  assemble_kernel<double2, 3><<<grid, 256, 0, st>>>(G, cols, out, ld);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

}  // namespace zbc

using namespace zbc;

extern "C" int vsie_assemble_columns(const zbc_grid* g, const zbc_segments* s, double freq_hz,
                                     const int32_t* cols, int ncols, int q, void* out, int64_t ld,
                                     zbc_dtype dt, zbc_stream stream) {
  clear_error();
  ZBC_CHECK_ARG(q == 3, "q must be 3 (vsie_assemble_columns_op takes the piecewise-linear q = 12)");
  return vsie_assemble_columns_op(g, s, freq_hz, cols, ncols, q, ZBC_OP_N, 1, out, ld, dt, stream);
}

extern "C" int vsie_assemble_columns_op(const zbc_grid* g, const zbc_segments* s, double freq_hz,
                                        const int32_t* cols, int ncols, int q, zbc_operator op, int nq, void* out,
                                        int64_t ld, zbc_dtype dt, zbc_stream stream) {
  clear_error();
  ZBC_CHECK_ARG(g && s && cols && out, "vsie_assemble_columns: null argument");
  ZBC_CHECK_ARG(op == ZBC_OP_N || op == ZBC_OP_K, "unknown operator %d", (int)op);
  ZBC_CHECK_ARG(nq >= 1 && nq <= kMaxQuad, "nq must be in [1, %d]", kMaxQuad);
  ZBC_CHECK_ARG(q == 3 || q == 12, "q must be 3 (piecewise-constant) or 12 (piecewise-linear)");
  ZBC_CHECK_ARG(g->n1 >= 1 && g->n2 >= 1 && g->n3 >= 1 && g->h > 0, "bad grid");
  ZBC_CHECK_ARG(s->m >= 1 && s->centre && s->tangent && s->length, "bad segments");
  ZBC_CHECK_ARG(ncols >= 0 && ncols <= 65535, "ncols must be in [0, 65535]");
  ZBC_CHECK_ARG(freq_hz > 0 && std::isfinite(freq_hz), "freq_hz must be positive");
  const int64_t nv = (int64_t)g->n1 * g->n2 * g->n3;
  ZBC_CHECK_ARG(ld >= q * nv, "ld (%lld) < q*n_v (%lld)", (long long)ld, (long long)(q * nv));
  ZBC_CHECK_ARG(dt == ZBC_C64 || dt == ZBC_C128, "bad dtype");
  if (ncols == 0) return ZBC_OK;
  GreenGeom G = make_green(g, s, freq_hz);
  G.op = op == ZBC_OP_K ? 1 : 0;
  G.nq = nq;
  gauss_legendre(nq, G.qx, G.qw);
  dim3 grid((unsigned)ceil_div(nv, 256), (unsigned)ncols);
  if (q == 12) {
    if (dt == ZBC_C128)
      assemble_kernel<double2, 12><<<grid, 256, 0, stream>>>(G, cols, (double2*)out, ld);
    else
      assemble_kernel<float2, 12><<<grid, 256, 0, stream>>>(G, cols, (float2*)out, ld);
  } else if (dt == ZBC_C128) {
    assemble_kernel<double2, 3><<<grid, 256, 0, stream>>>(G, cols, (double2*)out, ld);
  } else {
    assemble_kernel<float2, 3><<<grid, 256, 0, stream>>>(G, cols, (float2*)out, ld);
  }
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}
