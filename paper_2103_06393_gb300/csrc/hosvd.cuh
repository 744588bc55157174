// Job descriptors and kernels of the FP64 Tucker compressors (hosvd.cu), shared with the
// compression from fibres (cross.cu).  The kernels are defined in hosvd.cu.
#pragma once

#include <algorithm>
#include <vector>

#include "zbc_internal.cuh"

namespace zbc {

// element (x, c) of a mode unfolding sits at x*sx + (c % d1)*e1 + (c / d1)*e2
struct Unf {
  int64_t sx, d1, e1, e2;
  __device__ __forceinline__ int64_t at(int64_t x, int64_t c) const {
    return x * sx + (c % d1) * e1 + (c / d1) * e2;
  }
};

struct GramJob {
  const void* A;  // tensor base
  Unf u;
  int64_t C;      // columns of the unfolding
  int n;          // rows of the unfolding
  double2* G;     // n x n
};

struct RotJob {    // out(x, c) = sum_i conj(V[i + ldv*x]) A(i, c),  x < r, i < n
  const void* A;
  Unf u;
  int64_t C;
  int n, r, ldv;
  const double2* V;
  double2* out;
  Unf o;           // output placement of (x, c)
};

// Hermitian Jacobi eigensolver, one CTA per matrix (n even, in global memory).  On return H is
// diagonal (eigenvalues on the diagonal) and V holds the eigenvectors (columns).
struct JacJob {
  double2* H;
  double2* V;
  int n;
};

// U[:, a] = V1 * W[:, ord[a]]  (n x r), FP64
struct FacJob {
  const double2* V1;
  const double2* W;
  const int* ord;
  int n, r;
  double2* U;
};

// copy FP64 (src) -> complex64 (dst), several segments per job list
struct CopyJob {
  const double2* src;
  float2* dst;
  int64_t len;
};

template <typename T>
__device__ __forceinline__ double2 ld_z(const void* p, int64_t i) {
  if constexpr (sizeof(T) == 16) {
    return ((const double2*)p)[i];
  } else {
    float2 v = ((const float2*)p)[i];
    return make_double2(v.x, v.y);
  }
}

// G = A_(g) A_(g)^H for FP64 operands; grid (ceil(n/32), ceil(n/32), jobs)
void launch_gram_f64(const GramJob* jobs, dim3 grid, cudaStream_t st);
// out(x, c) = sum_i conj(V[i + ldv x]) A(i, c) for FP64 operands; grid (ceil(C/64), ceil(r/32), jobs)
void launch_rotate_f64(const RotJob* jobs, dim3 grid, cudaStream_t st);
// grid (jobs), 512 threads, dynamic smem jacobi_smem(n)
__global__ void jacobi_kernel(const JacJob* jobs, int max_sweeps, int* sweeps_out);
// grid (x, jobs), 256 threads
__global__ void factor_kernel(const FacJob* jobs);
// grid (x, jobs), 256 threads
__global__ void pack_kernel(const CopyJob* jobs);

inline size_t jacobi_smem(int n) { return (size_t)(n / 2) * (2 * sizeof(double) + sizeof(double2) + 2 * sizeof(int)); }

template <typename J>
static int upload_jobs(DevBuf& buf, const std::vector<J>& jobs, cudaStream_t st) {
  ZBC_TRY(buf.ensure(sizeof(J) * std::max<size_t>(1, jobs.size())));
  ZBC_TRY_CUDA(cudaMemcpyAsync(buf.ptr, jobs.data(), sizeof(J) * jobs.size(), cudaMemcpyHostToDevice, st));
  return ZBC_OK;
}

// Rank rule: smallest r >= 1 with sum_{i>r} lambda_i <= thr (lambda sorted descending, clamped >= 0)
inline int truncation_rank(const std::vector<double>& lam_desc, double thr) {
  const int n = (int)lam_desc.size();
  std::vector<double> tail(n + 1, 0.0);
  for (int i = n - 1; i >= 0; --i) tail[i] = tail[i + 1] + std::max(lam_desc[i], 0.0);
  for (int r = 1; r <= n; ++r)
    if (tail[r] <= thr) return r;
  return n;
}

}  // namespace zbc

// Append compressed columns (ranks 3 per tensor, packed complex64 pool, freed here) to *out, a
// new handle when *out is null; fills stats.n_tensors / max_rank and copies stats to stats_host.
int finish_compress(zbc_handle** out, const zbc_grid* g, int q, int ncols, const std::vector<int32_t>& ranks,
                    float2* pool, int64_t elems, zbc_compress_stats& stats, zbc_compress_stats* stats_host,
                    cudaStream_t stream);
// Arguments of the column compressors (null pointers, q, grid sizes even in [2, 1024], ncols,
// tol, dtype, ld, and a handle to append to that matches); ZBC_EINVAL with the message set.
int check_compress_args(const void* cols, int64_t ld, int ncols, const zbc_grid* g, int q, zbc_dtype in_dt,
                        double tol, zbc_handle** out);
