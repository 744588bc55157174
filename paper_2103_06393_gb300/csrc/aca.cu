// aca_compress: partially pivoted ACA of the coupling matrix (Sec. II.B.2) and its Tucker-based
// variant, Algorithm 3 (Sec. III.C), driven from the host with FP64 pivots, norms and test.
//
// Iteration k (Z ~ U V^H, u_l = columns of U, v_l = columns of V):
//   r = Z[i,:] - sum_l u_l[i] conj(v_l)          row residual (u_l[i] by element-wise Tucker
//                                                  evaluation in Algorithm 3)
//   j = argmax |r| over unused columns;  y = conj(r / r_j)
//   x = Z[:,j] - sum_l u_l conj(v_l[j])           column residual (Algorithm 1 on the
//                                                  compressed U in Algorithm 3)
//   s <- s + (|x||y|)^2 + 2 sum_l Re{(u_l^H x) conj(v_l^H y)}   (Frobenius norm of U V^H;
//                                                  u_l^H x by Algorithm 2 in Algorithm 3)
//   append x (dense, or as q HOSVD tensors at tolerance tucker_tol in Algorithm 3) and y;
//   stop when |x||y| <= tol sqrt(s); else i = argmax |x| over unused rows.
// Readings: ties go to the lowest index; used rows and columns are excluded from later
// pivots; the norm update carries the conjugate that the Frobenius identity needs; the
// start row is 0 and an all-zero residual row (a masked voxel) moves to the next unused row.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <set>

#include "green.cuh"

namespace zbc {

using cd = std::complex<double>;

GreenGeom make_green(const zbc_grid* g, const zbc_segments* s, double freq_hz);
int assemble_columns_c128(const GreenGeom& G, const int32_t* cols, int ncols, double2* out, int64_t ld,
                          cudaStream_t st);
int hosvd_compress(const void* cols, int64_t ld, int ncols, int n1, int n2, int n3, int q, zbc_dtype dt, double tol,
                   std::vector<int32_t>& ranks, float2** pool, int64_t* elems, double* max_err, int batch_cols,
                   cudaStream_t st);
int randomized_compress(const void* cols, int64_t ld, int ncols, int n1, int n2, int n3, int q, zbc_dtype dt,
                        double tol, const int32_t* widths, const float2* const* sketch, int lmax,
                        std::vector<int32_t>& ranks, float2** pool, int64_t* elems, zbc_compress_stats* stats,
                        cudaStream_t st);

// U's columns (complex128, ld N) in Tucker form: truncated HOSVD, or the fixed-width randomized
// range finder with the HOSVD as the fallback of each tensor that fails its check
static int compress_u(const void* cols, int64_t ld, int ncols, const zbc_grid* g, int q, double tol,
                      zbc_tucker_method method, const zbc_rank_model* model, int batch, std::vector<int32_t>& ranks,
                      float2** pool, int64_t* elems, double* max_err, int* fallbacks, cudaStream_t st) {
  if (method == ZBC_HOSVD)
    return hosvd_compress(cols, ld, ncols, g->n1, g->n2, g->n3, q, ZBC_C128, tol, ranks, pool, elems, max_err, batch,
                          st);
  std::vector<int32_t> widths(3 * (size_t)ncols * q, model->fixed_width);
  const float2* sk[3] = {(const float2*)model->sketch1, (const float2*)model->sketch2,
                         (const float2*)model->sketch3};
  zbc_compress_stats cs{};
  ZBC_TRY(randomized_compress(cols, ld, ncols, g->n1, g->n2, g->n3, q, ZBC_C128, tol, widths.data(), sk, model->lmax,
                              ranks, pool, elems, &cs, st));
  *max_err = std::max(*max_err, cs.max_rel_err);
  *fallbacks += cs.n_fallback;
  return ZBC_OK;
}

__global__ void aca_row_kernel(GreenGeom G, int64_t v, int k, double2* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= G.m) return;
  double2 z[3];
  green_entry(G, v, e, z);
  out[e] = z[k];
}

// t_l = G_l x1 U1_l[f1,:] x2 U2_l[f2,:] x3 U3_l[f3,:] for tensor (l, comp), one block per l
__global__ void __launch_bounds__(256) aca_eval_kernel(const float2* __restrict__ pool, const TensorDesc* __restrict__ desc,
                                                       int q, int comp, int n1, int n2, int n3, int f1, int f2, int f3,
                                                       double2* __restrict__ t) {
  const int l = blockIdx.x;
  const TensorDesc d = desc[(int64_t)l * q + comp];
  const float2* G = pool + d.off;
  const float2* U1 = G + (int64_t)d.r1 * d.r2 * d.r3;
  const float2* U2 = U1 + (int64_t)n1 * d.r1;
  const float2* U3 = U2 + (int64_t)n2 * d.r2;
  double sr = 0.0, si = 0.0;
  for (int o = threadIdx.x; o < d.r2 * d.r3; o += blockDim.x) {
    const int b = o % d.r2, c = o / d.r2;
    double ar = 0.0, ai = 0.0;
    for (int a = 0; a < d.r1; ++a) {
      const float2 gv = G[a + (int64_t)d.r1 * o];
      const float2 u = U1[f1 + (int64_t)n1 * a];
      ar += (double)gv.x * u.x - (double)gv.y * u.y;
      ai += (double)gv.x * u.y + (double)gv.y * u.x;
    }
    const float2 u2 = U2[f2 + (int64_t)n2 * b], u3 = U3[f3 + (int64_t)n3 * c];
    const double wr = (double)u2.x * u3.x - (double)u2.y * u3.y, wi = (double)u2.x * u3.y + (double)u2.y * u3.x;
    sr += ar * wr - ai * wi;
    si += ar * wi + ai * wr;
  }
  __shared__ double rs[256], is[256];
  rs[threadIdx.x] = sr;
  is[threadIdx.x] = si;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      rs[threadIdx.x] += rs[threadIdx.x + w];
      is[threadIdx.x] += is[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) t[l] = make_double2(rs[0], is[0]);
}

// x[r] -= sum_l U[r + N l] c_l
__global__ void aca_col_update_kernel(double2* __restrict__ x, const double2* __restrict__ U, int64_t N, int K,
                                      const double2* __restrict__ c) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  double2 acc = x[r];
  for (int l = 0; l < K; ++l) {
    const double2 u = U[r + N * l], cl = c[l];
    acc.x -= u.x * cl.x - u.y * cl.y;
    acc.y -= u.x * cl.y + u.y * cl.x;
  }
  x[r] = acc;
}

// t[l] = U[i + N l]
__global__ void aca_gather_row_kernel(const double2* __restrict__ U, int64_t N, int64_t i, int K, double2* __restrict__ t) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < K) t[l] = U[i + N * l];
}

// x[used[u]] = 0 (the current residual column is no longer needed once stored)
__global__ void aca_zero_rows_kernel(double2* __restrict__ x, const int64_t* __restrict__ used, int n) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) x[used[u]] = make_double2(0.0, 0.0);
}

// x[r] -= (double) y[r]
__global__ void aca_sub_c64_kernel(double2* __restrict__ x, const float2* __restrict__ y, int64_t N) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  x[r].x -= y[r].x;
  x[r].y -= y[r].y;
}

__global__ void aca_to_c64_kernel(const double2* __restrict__ x, float2* __restrict__ y, int64_t N) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  y[r] = make_float2((float)x[r].x, (float)x[r].y);
}

// partial[l * nb + b] = sum over block b's strided range of conj(U[r, l]) x[r]
__global__ void __launch_bounds__(256) aca_uhx_kernel(const double2* __restrict__ U, int64_t N,
                                                      const double2* __restrict__ x, double2* __restrict__ partial) {
  const int l = blockIdx.y;
  double sr = 0.0, si = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    const double2 u = U[r + N * l], v = x[r];
    sr += u.x * v.x + u.y * v.y;
    si += u.x * v.y - u.y * v.x;
  }
  __shared__ double rs[256], is[256];
  rs[threadIdx.x] = sr;
  is[threadIdx.x] = si;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      rs[threadIdx.x] += rs[threadIdx.x + w];
      is[threadIdx.x] += is[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(int64_t)l * gridDim.x + blockIdx.x] = make_double2(rs[0], is[0]);
}

// per block: sum |x|^2 and the (max |x|, lowest index) over its range; used rows read as 0
struct MaxIdx {
  double v;
  int64_t i;
};
__global__ void __launch_bounds__(256) aca_norm_argmax_kernel(const double2* __restrict__ x, int64_t N,
                                                              const int64_t* __restrict__ used, int nused,
                                                              double* __restrict__ norm_part,
                                                              MaxIdx* __restrict__ max_part) {
  double s = 0.0, best = -1.0;
  int64_t bi = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[r];
    const double a2 = v.x * v.x + v.y * v.y;
    s += a2;
    bool skip = false;
    for (int u = 0; u < nused; ++u) skip |= (used[u] == r);
    const double a = skip ? 0.0 : sqrt(a2);
    if (a > best) {
      best = a;
      bi = r;
    }
  }
  __shared__ double ss[256], bv[256];
  __shared__ int64_t bx[256];
  ss[threadIdx.x] = s;
  bv[threadIdx.x] = best;
  bx[threadIdx.x] = bi;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      ss[threadIdx.x] += ss[threadIdx.x + w];
      const double o = bv[threadIdx.x + w];
      const int64_t oi = bx[threadIdx.x + w];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bx[threadIdx.x])) {
        bv[threadIdx.x] = o;
        bx[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    norm_part[blockIdx.x] = ss[0];
    max_part[blockIdx.x] = MaxIdx{bv[0], bx[0]};
  }
}

namespace {
struct Dev {
  void* p = nullptr;
  ~Dev() {
    if (p) cudaFree(p);
  }
  int alloc(size_t b) {
    if (p) cudaFree(p);
    p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(b, 16));
    if (e != cudaSuccess) {
      set_error("cudaMalloc(%zu) failed in aca_compress", b);
      return ZBC_ENOMEM;
    }
    return ZBC_OK;
  }
};
}  // namespace

}  // namespace zbc

using namespace zbc;

extern "C" int aca_compress(const zbc_grid* g, const zbc_segments* s, double freq_hz, int q, double tol, int max_rank,
                            zbc_aca_mode mode, double tucker_tol, zbc_tucker_method method,
                            const zbc_rank_model* model, zbc_handle** out, zbc_aca_stats* stats,
                            int32_t* pivots_host, zbc_stream st) {
  clear_error();
  ZBC_CHECK_ARG(g && s && out, "aca_compress: null argument");
  ZBC_CHECK_ARG(q == 3, "q must be 3");
  ZBC_CHECK_ARG(g->n1 >= 2 && g->n2 >= 2 && g->n3 >= 2 && g->n1 % 2 == 0 && g->n2 % 2 == 0 && g->n3 % 2 == 0,
                "grid sizes must be even and >= 2");
  ZBC_CHECK_ARG(s->m >= 1 && s->centre && s->tangent && s->length, "bad segments");
  ZBC_CHECK_ARG(tol > 0 && tol < 1 && max_rank >= 1, "bad tol or max_rank");
  ZBC_CHECK_ARG(mode == ZBC_ACA_DENSE_U || mode == ZBC_ACA_ALG3, "bad mode");
  ZBC_CHECK_ARG(method == ZBC_HOSVD || method == ZBC_RANDOMIZED_FIXED,
                "U's columns are compressed by ZBC_HOSVD or ZBC_RANDOMIZED_FIXED (they are residual columns of Z, "
                "not single segments, so the rank predictor has no features for them)");
  if (method == ZBC_RANDOMIZED_FIXED) {
    ZBC_CHECK_ARG(model && model->sketch1 && model->sketch2 && model->sketch3, "RANDOMIZED_FIXED needs a rank model");
    ZBC_CHECK_ARG(model->fixed_width >= 1 && model->lmax >= 2 && model->lmax <= 64, "bad fixed_width or lmax");
  }
  if (!(tucker_tol > 0)) tucker_tol = 3.0 * tol;  // Algorithm 3 compresses U at 3 eps
  const GreenGeom G = make_green(g, s, freq_hz);
  const int m = s->m;
  const int64_t nv = (int64_t)g->n1 * g->n2 * g->n3;
  const int64_t N = (int64_t)q * nv;
  const int kmax = (int)std::min<int64_t>(std::min<int64_t>(N, m), max_rank);

  Dev d_row, d_col, d_col32, d_tmp32, d_U, d_c, d_t, d_part, d_norm, d_normz, d_max, d_used, d_cols;
  ZBC_TRY(d_row.alloc(sizeof(double2) * m));
  ZBC_TRY(d_col.alloc(sizeof(double2) * N));
  ZBC_TRY(d_col32.alloc(sizeof(float2) * N));
  ZBC_TRY(d_tmp32.alloc(sizeof(float2) * N));
  ZBC_TRY(d_c.alloc(sizeof(double2) * kmax));
  ZBC_TRY(d_t.alloc(sizeof(double2) * kmax));
  const int NB = 512;
  ZBC_TRY(d_part.alloc(sizeof(double2) * (size_t)NB * kmax));
  ZBC_TRY(d_norm.alloc(sizeof(double) * NB));
  ZBC_TRY(d_normz.alloc(sizeof(double) * NB));
  ZBC_TRY(d_max.alloc(sizeof(MaxIdx) * NB));
  ZBC_TRY(d_used.alloc(sizeof(int64_t) * (kmax + 1)));
  ZBC_TRY(d_cols.alloc(sizeof(int32_t)));
  int64_t ucap = 0;
  if (mode == ZBC_ACA_DENSE_U) {
    ucap = std::min<int64_t>(kmax, 64);
    ZBC_TRY(d_U.alloc(sizeof(double2) * N * ucap));
  }
  // Algorithm 3: the compressed U grows column by column in a handle
  zbc_handle* hh = new zbc_handle();
  hh->h.n1 = g->n1;
  hh->h.n2 = g->n2;
  hh->h.n3 = g->n3;
  hh->h.q = q;
  std::unique_ptr<zbc_handle> guard(hh);

  std::vector<std::vector<cd>> V;  // columns y
  std::set<int64_t> used_r;
  std::set<int> used_c;
  std::vector<int64_t> used_r_list;
  std::vector<int32_t> piv;
  double s2 = 0.0, max_terr = 0.0, last = 0.0;
  int64_t i = 0;
  bool converged = false;
  int restarts = 0, fallbacks = 0;
  std::vector<double2> hrow(m), ht(kmax);
  int K = 0;
  // ZBC_TRACE_ACA set: one line per iteration on stderr (progress of long compressions)
  const bool trace = std::getenv("ZBC_TRACE_ACA") != nullptr;
  const auto t_start = std::chrono::steady_clock::now();
  for (int k = 0; k < kmax; ++k) {
    std::vector<cd> r(m);
    while (true) {
      const int64_t v = i % nv;
      const int comp = (int)(i / nv);
      aca_row_kernel<<<ceil_div(m, 256), 256, 0, st>>>(G, v, comp, (double2*)d_row.p);
      count_launch();
      if (K > 0) {
        if (mode == ZBC_ACA_DENSE_U) {
          aca_gather_row_kernel<<<ceil_div(K, 256), 256, 0, st>>>((const double2*)d_U.p, N, i, K, (double2*)d_t.p);
          count_launch();
          ZBC_TRY_CUDA(cudaMemcpyAsync(ht.data(), d_t.p, sizeof(double2) * K, cudaMemcpyDeviceToHost, st));
        } else {
          const int f1 = (int)(v % g->n1), f2 = (int)((v / g->n1) % g->n2), f3 = (int)(v / ((int64_t)g->n1 * g->n2));
          aca_eval_kernel<<<K, 256, 0, st>>>(hh->h.d_pool, hh->h.d_desc, q, comp, g->n1, g->n2, g->n3, f1, f2, f3,
                                              (double2*)d_t.p);
          count_launch();
          ZBC_TRY_CUDA(cudaMemcpyAsync(ht.data(), d_t.p, sizeof(double2) * K, cudaMemcpyDeviceToHost, st));
        }
      }
      ZBC_TRY_CUDA(cudaMemcpyAsync(hrow.data(), d_row.p, sizeof(double2) * m, cudaMemcpyDeviceToHost, st));
      ZBC_TRY_CUDA(cudaStreamSynchronize(st));
      for (int e = 0; e < m; ++e) r[e] = cd(hrow[e].x, hrow[e].y);
      for (int l = 0; l < K; ++l) {
        const cd tl(ht[l].x, ht[l].y);
        for (int e = 0; e < m; ++e) r[e] -= tl * std::conj(V[l][e]);
      }
      used_r.insert(i);
      used_r_list.push_back(i);
      double mx = 0.0;
      for (int e = 0; e < m; ++e)
        if (!used_c.count(e)) mx = std::max(mx, std::abs(r[e]));
      if (mx > 0.0) break;
      // all-zero residual row: next unused row in index order
      ++restarts;
      int64_t nx = i + 1;
      while (nx < N && used_r.count(nx)) ++nx;
      if (nx >= N) {
        converged = true;
        break;
      }
      i = nx;
    }
    if (converged) break;
    int j = -1;
    double best = -1.0;
    for (int e = 0; e < m; ++e) {
      if (used_c.count(e)) continue;
      const double a = std::abs(r[e]);
      if (a > best) {
        best = a;
        j = e;
      }
    }
    const cd rj = r[j];
    std::vector<cd> y(m);
    for (int e = 0; e < m; ++e) y[e] = std::conj(r[e] / rj);
    // column residual
    ZBC_TRY_CUDA(cudaMemcpyAsync(d_cols.p, &j, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    ZBC_TRY(assemble_columns_c128(G, (const int32_t*)d_cols.p, 1, (double2*)d_col.p, N, st));
    // ||Z[:, j]||^2 (the scale of the terms the residual column is the difference of)
    aca_norm_argmax_kernel<<<NB, 256, 0, st>>>((const double2*)d_col.p, N, nullptr, 0, (double*)d_normz.p,
                                              (MaxIdx*)d_max.p);
    count_launch();
    std::vector<double> npz(NB);
    ZBC_TRY_CUDA(cudaMemcpyAsync(npz.data(), d_normz.p, sizeof(double) * NB, cudaMemcpyDeviceToHost, st));
    std::vector<double2> c(K);
    for (int l = 0; l < K; ++l) {
      const cd cl = std::conj(V[l][j]);
      c[l] = make_double2(cl.real(), cl.imag());
    }
    if (K > 0) {
      if (mode == ZBC_ACA_DENSE_U) {
        ZBC_TRY_CUDA(cudaMemcpyAsync(d_c.p, c.data(), sizeof(double2) * K, cudaMemcpyHostToDevice, st));
        aca_col_update_kernel<<<ceil_div(N, 256), 256, 0, st>>>((double2*)d_col.p, (const double2*)d_U.p, N, K,
                                                               (const double2*)d_c.p);
        count_launch();
      } else {
        std::vector<float2> c32(K);
        for (int l = 0; l < K; ++l) c32[l] = make_float2((float)c[l].x, (float)c[l].y);
        ZBC_TRY_CUDA(cudaMemcpyAsync(d_c.p, c32.data(), sizeof(float2) * K, cudaMemcpyHostToDevice, st));
        ZBC_TRY(matvec_simt(hh->h, (const float2*)d_c.p, K, 1, (float2*)d_tmp32.p, N, 9, st));
        aca_sub_c64_kernel<<<ceil_div(N, 256), 256, 0, st>>>((double2*)d_col.p, (const float2*)d_tmp32.p, N);
        count_launch();
      }
    }
    // norms and the cross terms of the Frobenius update
    aca_norm_argmax_kernel<<<NB, 256, 0, st>>>((const double2*)d_col.p, N, nullptr, 0, (double*)d_norm.p,
                                              (MaxIdx*)d_max.p);
    count_launch();
    std::vector<double> np(NB);
    ZBC_TRY_CUDA(cudaMemcpyAsync(np.data(), d_norm.p, sizeof(double) * NB, cudaMemcpyDeviceToHost, st));
    std::vector<cd> uhx(K);
    if (K > 0) {
      if (mode == ZBC_ACA_DENSE_U) {
        aca_uhx_kernel<<<dim3(NB, K), 256, 0, st>>>((const double2*)d_U.p, N, (const double2*)d_col.p,
                                                    (double2*)d_part.p);
        count_launch();
        std::vector<double2> part((size_t)NB * K);
        ZBC_TRY_CUDA(cudaMemcpyAsync(part.data(), d_part.p, sizeof(double2) * part.size(), cudaMemcpyDeviceToHost, st));
        ZBC_TRY_CUDA(cudaStreamSynchronize(st));
        for (int l = 0; l < K; ++l) {
          cd a = 0;
          for (int b = 0; b < NB; ++b) a += cd(part[(size_t)l * NB + b].x, part[(size_t)l * NB + b].y);
          uhx[l] = a;
        }
      } else {
        aca_to_c64_kernel<<<ceil_div(N, 256), 256, 0, st>>>((const double2*)d_col.p, (float2*)d_col32.p, N);
        count_launch();
        ZBC_TRY(rmatvec_simt(hh->h, (const float2*)d_col32.p, N, 1, (float2*)d_tmp32.p, K, 9, st));
        std::vector<float2> w(K);
        ZBC_TRY_CUDA(cudaMemcpyAsync(w.data(), d_tmp32.p, sizeof(float2) * K, cudaMemcpyDeviceToHost, st));
        ZBC_TRY_CUDA(cudaStreamSynchronize(st));
        for (int l = 0; l < K; ++l) uhx[l] = cd(w[l].x, w[l].y);
      }
    }
    ZBC_TRY_CUDA(cudaStreamSynchronize(st));
    double nx2 = 0.0, nz2 = 0.0;
    for (int b = 0; b < NB; ++b) nx2 += np[b];
    for (int b = 0; b < NB; ++b) nz2 += npz[b];
    double ny2 = 0.0;
    for (int e = 0; e < m; ++e) ny2 += std::norm(y[e]);
    const double nxy = std::sqrt(nx2) * std::sqrt(ny2);
    s2 += nxy * nxy;
    for (int l = 0; l < K; ++l) {
      cd vhy = 0;
      for (int e = 0; e < m; ++e) vhy += std::conj(V[l][e]) * y[e];
      s2 += 2.0 * (uhx[l] * std::conj(vhy)).real();
    }
    // append x and y
    if (mode == ZBC_ACA_DENSE_U) {
      if (K >= ucap) {
        const int64_t ncap = std::min<int64_t>(kmax, 2 * ucap);
        Dev nu;
        ZBC_TRY(nu.alloc(sizeof(double2) * N * ncap));
        ZBC_TRY_CUDA(cudaMemcpyAsync(nu.p, d_U.p, sizeof(double2) * N * K, cudaMemcpyDeviceToDevice, st));
        ZBC_TRY_CUDA(cudaStreamSynchronize(st));
        std::swap(nu.p, d_U.p);
        ucap = ncap;
      }
      ZBC_TRY_CUDA(cudaMemcpyAsync((double2*)d_U.p + N * K, d_col.p, sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
    } else {
      std::vector<int32_t> rk;
      float2* pool = nullptr;
      int64_t elems = 0;
      ZBC_TRY(compress_u(d_col.p, N, 1, g, q, tucker_tol, method, model, 1, rk, &pool, &elems, &max_terr, &fallbacks,
                         st));
      const int sa = handle_append(&hh->h, rk, pool, elems, 1, st);
      cudaFree(pool);
      if (sa != ZBC_OK) return sa;
      if (trace) {
        int rmax = 0;
        for (int v : rk) rmax = std::max(rmax, v);
        std::fprintf(stderr, "[aca] k %d i %lld j %d |x||y|/sqrt(s) %.3e |Z_j|/|x| %.3e max rank %d fallbacks %d %.1f ms\n",
                     K, (long long)i, j, nxy / std::sqrt(std::max(s2, 1e-300)), std::sqrt(nz2 / std::max(nx2, 1e-300)),
                     rmax, fallbacks,
                     std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count());
        std::fflush(stderr);
      }
    }
    V.push_back(y);
    used_c.insert(j);
    piv.push_back((int32_t)i);
    piv.push_back(j);
    ++K;
    last = nxy;
    if (nxy <= tol * std::sqrt(std::max(s2, 0.0))) {
      converged = true;
      break;
    }
    // next row pivot: argmax |x| over unused rows
    ZBC_TRY(d_used.alloc(sizeof(int64_t) * used_r_list.size()));
    ZBC_TRY_CUDA(cudaMemcpyAsync(d_used.p, used_r_list.data(), sizeof(int64_t) * used_r_list.size(),
                                 cudaMemcpyHostToDevice, st));
    aca_zero_rows_kernel<<<ceil_div((int64_t)used_r_list.size(), 256), 256, 0, st>>>(
        (double2*)d_col.p, (const int64_t*)d_used.p, (int)used_r_list.size());
    aca_norm_argmax_kernel<<<NB, 256, 0, st>>>((const double2*)d_col.p, N, nullptr, 0, (double*)d_norm.p,
                                              (MaxIdx*)d_max.p);
    count_launch(2);
    std::vector<MaxIdx> mp(NB);
    ZBC_TRY_CUDA(cudaMemcpyAsync(mp.data(), d_max.p, sizeof(MaxIdx) * NB, cudaMemcpyDeviceToHost, st));
    ZBC_TRY_CUDA(cudaStreamSynchronize(st));
    MaxIdx b = mp[0];
    for (int t = 1; t < NB; ++t)
      if (mp[t].v > b.v || (mp[t].v == b.v && mp[t].i < b.i)) b = mp[t];
    i = b.i;
  }
  if (K == 0) {
    set_error("aca_compress: the matrix is zero");
    return ZBC_EINVAL;
  }
  // dense U: compress its columns now (Sec. III.A, applied to the r_c columns of U)
  if (mode == ZBC_ACA_DENSE_U) {
    std::vector<int32_t> rk;
    float2* pool = nullptr;
    int64_t elems = 0;
    const int64_t per_col = (int64_t)q * nv * 16;
    const int batch = (int)std::max<int64_t>(1, std::min<int64_t>(K, ((int64_t)4 << 30) / per_col));
    ZBC_TRY(compress_u(d_U.p, N, K, g, q, tucker_tol, method, model, batch, rk, &pool, &elems, &max_terr, &fallbacks,
                       st));
    const int sa = handle_append(&hh->h, rk, pool, elems, K, st);
    cudaFree(pool);
    if (sa != ZBC_OK) return sa;
  }
  // V (m x r_c, complex64)
  std::vector<float2> vh((size_t)m * K);
  for (int l = 0; l < K; ++l)
    for (int e = 0; e < m; ++e) vh[(size_t)l * m + e] = make_float2((float)V[l][e].real(), (float)V[l][e].imag());
  Handle& h = hh->h;
  ZBC_TRY_CUDA(cudaMalloc(&h.d_v, sizeof(float2) * vh.size()));
  ZBC_TRY_CUDA(cudaMemcpy(h.d_v, vh.data(), sizeof(float2) * vh.size(), cudaMemcpyHostToDevice));
  h.has_v = true;
  h.m = m;
  if (h.cache) {
    cache_release(h.cache);
    h.cache = nullptr;
  }
  if (stats) {
    stats->rank = K;
    stats->converged = converged ? 1 : 0;
    stats->row_restarts = restarts;
    stats->max_tucker_rank = h.max_rank;
    stats->s2 = s2;
    stats->last_term = last;
    stats->max_tucker_err = max_terr;
    stats->tucker_fallbacks = fallbacks;
  }
  if (pivots_host) std::copy(piv.begin(), piv.end(), pivots_host);
  *out = guard.release();
  return ZBC_OK;
}
