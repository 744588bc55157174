// tucker_compress: column-wise truncated HOSVD on the GPU in FP64 (Sec. II.B.1, Sec. III.A).
//
// Every column of Z is reshaped into q tensors (Fig. 2); each tensor A gets, per mode g,
// the left singular vectors of its unfolding A_(g) and the truncation rank
//   r_g = min { r >= 1 : sum_{i>r} sigma_i^2 <= (tol^2/3) ||A||_F^2 },
// then the core A x1 U1^H x2 U2^H x3 U3^H (De Lathauwer's truncated HOSVD, used by the paper
// at tolerance 1e-8 in Sec. IV.A and at 3*eps inside Algorithm 3).
//
// The singular pairs come from a two-pass Gram/Jacobi scheme in FP64:
//   pass 1  H1 = A_(g) A_(g)^H,           Jacobi  H1 = V1 L1 V1^H
//   pass 2  B  = V1^H A_(g),  H2 = B B^H,  Jacobi  H2 = W L W^H
//   U_g = V1 W (columns sorted by L, descending), sigma_i^2 = L_i.
// Pass 2 restores the accuracy a single Gram loses for small singular values: the rows of B
// are nearly orthogonal, and the Jacobi method recovers the eigenvalues of such a matrix to
// high relative accuracy.  The Jacobi solver uses parallel (round-robin) ordering: n/2
// disjoint rotations per round, applied as a row pass then a column pass.
#include <algorithm>
#include <cmath>
#include <numeric>

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

template <typename T>
__device__ __forceinline__ double2 ld_z(const void* p, int64_t i) {
  if constexpr (sizeof(T) == 16) {
    return ((const double2*)p)[i];
  } else {
    float2 v = ((const float2*)p)[i];
    return make_double2(v.x, v.y);
  }
}

// ---------------------------------------------------------------------------------------------
// Gram matrices G = A_(g) A_(g)^H, 32x32 output tiles, lower-triangle tiles only + mirror
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(const GramJob* jobs) {
  const GramJob jb = jobs[blockIdx.z];
  const int tx = blockIdx.x * 32, ty = blockIdx.y * 32;
  if (tx >= jb.n || ty >= jb.n || ty > tx) return;
  __shared__ double2 sa[16][33];
  __shared__ double2 sb[16][33];
  const int lx = threadIdx.x % 16, ly = threadIdx.x / 16;  // each thread: rows tx+2lx.., cols ty+2ly..
  double2 acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = make_double2(0, 0);
  for (int64_t c0 = 0; c0 < jb.C; c0 += 16) {
    for (int e = threadIdx.x; e < 16 * 32; e += 256) {
      const int cc = e / 32, xx = e % 32;
      const int64_t c = c0 + cc;
      double2 va = make_double2(0, 0), vb = make_double2(0, 0);
      if (c < jb.C) {
        if (tx + xx < jb.n) va = ld_z<T>(jb.A, jb.u.at(tx + xx, c));
        if (ty + xx < jb.n) vb = ld_z<T>(jb.A, jb.u.at(ty + xx, c));
      }
      sa[cc][xx] = va;
      sb[cc][xx] = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int cc = 0; cc < 16; ++cc) {
      double2 a0 = sa[cc][2 * lx], a1 = sa[cc][2 * lx + 1];
      double2 b0 = sb[cc][2 * ly], b1 = sb[cc][2 * ly + 1];
      // G[x,y] += A(x,c) conj(A(y,c))
      acc[0][0] = zfma_conj(b0, a0, acc[0][0]);
      acc[0][1] = zfma_conj(b1, a0, acc[0][1]);
      acc[1][0] = zfma_conj(b0, a1, acc[1][0]);
      acc[1][1] = zfma_conj(b1, a1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int x = tx + 2 * lx + a, y = ty + 2 * ly + b;
      if (x < jb.n && y < jb.n && y <= x) {
        jb.G[x + (int64_t)jb.n * y] = acc[a][b];
        jb.G[y + (int64_t)jb.n * x] = make_double2(acc[a][b].x, -acc[a][b].y);
      }
    }
}

// ---------------------------------------------------------------------------------------------
// out(x, c) = sum_i conj(V[i, x]) A(i, c): tiles of 32 x by 64 c, i in chunks of 16
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) rotate_kernel(const RotJob* jobs) {
  const RotJob jb = jobs[blockIdx.z];
  const int x0 = blockIdx.y * 32;
  const int64_t c0 = (int64_t)blockIdx.x * 64;
  if (x0 >= jb.r || c0 >= jb.C) return;
  __shared__ double2 sv[16][33];
  __shared__ double2 sa[16][65];
  const int lc = threadIdx.x % 32, lx = threadIdx.x / 32;  // thread: c = c0+lc, c0+lc+32; x = x0+lx+8k
  double2 acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = make_double2(0, 0);
  for (int i0 = 0; i0 < jb.n; i0 += 16) {
    for (int e = threadIdx.x; e < 16 * 32; e += 256) {
      const int ii = e / 32, xx = e % 32;
      double2 v = make_double2(0, 0);
      if (i0 + ii < jb.n && x0 + xx < jb.r) v = jb.V[(i0 + ii) + (int64_t)jb.ldv * (x0 + xx)];
      sv[ii][xx] = v;
    }
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int ii = e / 64, cc = e % 64;
      double2 v = make_double2(0, 0);
      if (i0 + ii < jb.n && c0 + cc < jb.C) v = ld_z<T>(jb.A, jb.u.at(i0 + ii, c0 + cc));
      sa[ii][cc] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int ii = 0; ii < 16; ++ii) {
      const double2 a0 = sa[ii][lc], a1 = sa[ii][lc + 32];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double2 v = sv[ii][lx + 8 * k];
        acc[k][0] = zfma_conj(v, a0, acc[k][0]);
        acc[k][1] = zfma_conj(v, a1, acc[k][1]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int x = x0 + lx + 8 * k;
      const int64_t c = c0 + lc + 32 * h;
      if (x < jb.r && c < jb.C) jb.out[jb.o.at(x, c)] = acc[k][h];
    }
}

// ---------------------------------------------------------------------------------------------
// Hermitian Jacobi eigensolver, one CTA per matrix (n even, in global memory).  On return H is
// diagonal (eigenvalues on the diagonal) and V holds the eigenvectors (columns).
// ---------------------------------------------------------------------------------------------
struct JacJob {
  double2* H;
  double2* V;
  int n;
};

__global__ void __launch_bounds__(512) jacobi_kernel(const JacJob* jobs, int max_sweeps, int* sweeps_out) {
  const JacJob jb = jobs[blockIdx.x];
  const int n = jb.n;
  double2* H = jb.H;
  double2* V = jb.V;
  extern __shared__ unsigned char smem_raw[];
  double* cs = (double*)smem_raw;            // n/2
  double* sn = cs + n / 2;                   // n/2
  double2* ph = (double2*)(sn + n / 2);      // n/2 : e^{i phi}
  int* pp = (int*)(ph + n / 2);              // n/2
  int* pq = pp + n / 2;                      // n/2
  __shared__ int nrot;
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    V[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  const double eps = 2.220446049250313e-16;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) nrot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < n - 1; ++rnd) {
      for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
        int p, q;
        if (i == 0) {
          p = n - 1;
          q = rnd;
        } else {
          p = (rnd + i) % (n - 1);
          q = (rnd - i + n - 1) % (n - 1);
        }
        const double a = H[p + (int64_t)n * p].x, b = H[q + (int64_t)n * q].x;
        const double2 c = H[p + (int64_t)n * q];
        const double ac = hypot(c.x, c.y);
        pp[i] = p;
        pq[i] = q;
        if (ac == 0.0 || ac <= eps * sqrt(fabs(a) * fabs(b))) {
          cs[i] = 1.0;
          sn[i] = 0.0;
          ph[i] = make_double2(1.0, 0.0);
        } else {
          const double zeta = (b - a) / (2.0 * ac);
          const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cc = 1.0 / sqrt(1.0 + t * t);
          cs[i] = cc;
          sn[i] = t * cc;
          ph[i] = make_double2(c.x / ac, c.y / ac);
          atomicAdd(&nrot, 1);
        }
      }
      __syncthreads();
      // row pass: rows p,q <- J^H rows
      for (int64_t e = threadIdx.x; e < (int64_t)(n / 2) * n; e += blockDim.x) {
        const int i = (int)(e % (n / 2)), x = (int)(e / (n / 2));
        if (sn[i] == 0.0) continue;
        const int p = pp[i], q = pq[i];
        const double c = cs[i], s = sn[i];
        const double2 f = ph[i];
        const double2 hp = H[p + (int64_t)n * x], hq = H[q + (int64_t)n * x];
        const double2 fq = zmul(f, hq);  // e^{i phi} H[q,x]
        H[p + (int64_t)n * x] = make_double2(c * hp.x - s * fq.x, c * hp.y - s * fq.y);
        H[q + (int64_t)n * x] = make_double2(s * hp.x + c * fq.x, s * hp.y + c * fq.y);
      }
      __syncthreads();
      // column pass: columns p,q <- columns J ; same on V
      for (int64_t e = threadIdx.x; e < (int64_t)(n / 2) * n; e += blockDim.x) {
        const int i = (int)(e % (n / 2)), x = (int)(e / (n / 2));
        if (sn[i] == 0.0) continue;
        const int p = pp[i], q = pq[i];
        const double c = cs[i], s = sn[i];
        const double2 fc = make_double2(ph[i].x, -ph[i].y);  // e^{-i phi}
        {
          const double2 hp = H[x + (int64_t)n * p], hq = H[x + (int64_t)n * q];
          const double2 gq = zmul(fc, hq);
          H[x + (int64_t)n * p] = make_double2(c * hp.x - s * gq.x, c * hp.y - s * gq.y);
          H[x + (int64_t)n * q] = make_double2(s * hp.x + c * gq.x, s * hp.y + c * gq.y);
        }
        {
          const double2 vp = V[x + (int64_t)n * p], vq = V[x + (int64_t)n * q];
          const double2 gq = zmul(fc, vq);
          V[x + (int64_t)n * p] = make_double2(c * vp.x - s * gq.x, c * vp.y - s * gq.y);
          V[x + (int64_t)n * q] = make_double2(s * vp.x + c * gq.x, s * vp.y + c * gq.y);
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
        if (sn[i] == 0.0) continue;
        const int p = pp[i], q = pq[i];
        H[p + (int64_t)n * q] = make_double2(0, 0);
        H[q + (int64_t)n * p] = make_double2(0, 0);
        H[p + (int64_t)n * p].y = 0.0;
        H[q + (int64_t)n * q].y = 0.0;
      }
      __syncthreads();
    }
    if (nrot == 0) break;
    __syncthreads();
  }
  if (threadIdx.x == 0 && sweeps_out) sweeps_out[blockIdx.x] = sweep;
}

// ||A||_F^2 partial sums: 64 blocks per tensor, deterministic host-side final sum
template <typename T>
__global__ void __launch_bounds__(256) norm2_kernel(const void* const* bases, int64_t nv, double* partial) {
  const int t = blockIdx.y;
  const void* A = bases[t];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = ld_z<T>(A, i);
    s += v.x * v.x + v.y * v.y;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(int64_t)t * gridDim.x + blockIdx.x] = red[0];
}

// U[:, a] = V1 * W[:, ord[a]]  (n x r), FP64
struct FacJob {
  const double2* V1;
  const double2* W;
  const int* ord;
  int n, r;
  double2* U;
};
__global__ void __launch_bounds__(256) factor_kernel(const FacJob* jobs) {
  const FacJob jb = jobs[blockIdx.y];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < jb.n * jb.r; e += gridDim.x * blockDim.x) {
    const int i = e % jb.n, a = e / jb.n;
    const int col = jb.ord[a];
    double2 s = make_double2(0, 0);
    for (int l = 0; l < jb.n; ++l) s = zfma(jb.V1[i + (int64_t)jb.n * l], jb.W[l + (int64_t)jb.n * col], s);
    jb.U[i + (int64_t)jb.n * a] = s;
  }
}

// copy FP64 (src) -> complex64 (dst), several segments per job list
struct CopyJob {
  const double2* src;
  float2* dst;
  int64_t len;
};
__global__ void __launch_bounds__(256) pack_kernel(const CopyJob* jobs) {
  const CopyJob jb = jobs[blockIdx.y];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < jb.len; e += (int64_t)gridDim.x * blockDim.x)
    jb.dst[e] = make_float2((float)jb.src[e].x, (float)jb.src[e].y);
}

// ---------------------------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------------------------
template <typename J>
static int upload_jobs(DevBuf& buf, const std::vector<J>& jobs, cudaStream_t st) {
  ZBC_TRY(buf.ensure(sizeof(J) * std::max<size_t>(1, jobs.size())));
  ZBC_TRY_CUDA(cudaMemcpyAsync(buf.ptr, jobs.data(), sizeof(J) * jobs.size(), cudaMemcpyHostToDevice, st));
  return ZBC_OK;
}

// Rank rule: smallest r >= 1 with sum_{i>r} lambda_i <= thr (lambda sorted descending, clamped >= 0)
static int truncation_rank(const std::vector<double>& lam_desc, double thr) {
  const int n = (int)lam_desc.size();
  std::vector<double> tail(n + 1, 0.0);
  for (int i = n - 1; i >= 0; --i) tail[i] = tail[i + 1] + std::max(lam_desc[i], 0.0);
  for (int r = 1; r <= n; ++r)
    if (tail[r] <= thr) return r;
  return n;
}

struct HosvdWork {
  DevBuf jobs_a, jobs_b, jobs_c, jobs_d;
  DevBuf H, V1, W, Bbuf, U, C1, C2, G, norm_part, ord, sweeps, base_ptrs;
};

// Compress tensors t = 0..T-1 (tensor t = column t/q, component t%q) of one batch.
// Appends ranks (3 per tensor) and writes the packed complex64 pool of the batch to *pool_out
// (device, allocated here, caller frees).
template <typename T>
static int hosvd_batch(const void* cols, int64_t ld, int ncols, int n1, int n2, int n3, int q, double tol,
                       HosvdWork& w, std::vector<int32_t>& ranks_out, float2** pool_out, int64_t* elems_out,
                       double* max_err_bound, cudaStream_t st) {
  const int64_t nv = (int64_t)n1 * n2 * n3;
  const int NT = ncols * q;
  const int n[3] = {n1, n2, n3};
  const int64_t C[3] = {nv / n1, nv / n2, nv / n3};
  const int nmax = std::max(n1, std::max(n2, n3));
  const int nmax_e = nmax + (nmax & 1);
  const Unf unf[3] = {{1, nv / n1, n1, 0}, {n1, n1, 1, (int64_t)n1 * n2}, {(int64_t)n1 * n2, (int64_t)n1 * n2, 1, 0}};
  const size_t eb = sizeof(T);
  std::vector<const void*> base(NT);
  for (int t = 0; t < NT; ++t) base[t] = (const char*)cols + ((int64_t)(t / q) * ld + (int64_t)(t % q) * nv) * eb;

  // ||A||^2
  ZBC_TRY(w.base_ptrs.ensure(sizeof(void*) * NT));
  ZBC_TRY_CUDA(cudaMemcpyAsync(w.base_ptrs.ptr, base.data(), sizeof(void*) * NT, cudaMemcpyHostToDevice, st));
  ZBC_TRY(w.norm_part.ensure(sizeof(double) * 64 * NT));
  norm2_kernel<T><<<dim3(64, NT), 256, 0, st>>>((const void* const*)w.base_ptrs.ptr, nv, (double*)w.norm_part.ptr);
  ZBC_TRY_CUDA(cudaGetLastError());
  std::vector<double> part(64 * (size_t)NT), norm2(NT, 0.0);
  ZBC_TRY_CUDA(cudaMemcpyAsync(part.data(), w.norm_part.ptr, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st));

  const size_t mat = (size_t)nmax_e * nmax_e;
  ZBC_TRY(w.H.ensure(sizeof(double2) * mat * NT));
  ZBC_TRY(w.V1.ensure(sizeof(double2) * mat * NT));
  ZBC_TRY(w.W.ensure(sizeof(double2) * mat * NT));
  ZBC_TRY(w.Bbuf.ensure(sizeof(double2) * (size_t)nv * NT));
  ZBC_TRY(w.U.ensure(sizeof(double2) * (size_t)(n1 + n2 + n3) * nmax * NT));
  ZBC_TRY(w.sweeps.ensure(sizeof(int) * NT));
  double2* Hb = (double2*)w.H.ptr;
  double2* V1b = (double2*)w.V1.ptr;
  double2* Wb = (double2*)w.W.ptr;
  double2* Bb = (double2*)w.Bbuf.ptr;
  double2* Ub = (double2*)w.U.ptr;
  const int64_t uoff[3] = {0, (int64_t)n1 * nmax, (int64_t)(n1 + n2) * nmax};
  const int64_t ustride = (int64_t)(n1 + n2 + n3) * nmax;

  std::vector<int> rk(3 * (size_t)NT);
  ZBC_TRY_CUDA(cudaStreamSynchronize(st));
  for (int t = 0; t < NT; ++t)
    for (int b = 0; b < 64; ++b) norm2[t] += part[(size_t)t * 64 + b];

  double worst = 0.0;
  std::vector<double> tails(NT, 0.0);
  for (int g = 0; g < 3; ++g) {
    const int ng = n[g], ne = ng + (ng & 1);
    // zero-padded H for odd n (pad row/column stays decoupled)
    if (ne != ng) ZBC_TRY_CUDA(cudaMemsetAsync(Hb, 0, sizeof(double2) * mat * NT, st));
    std::vector<GramJob> gj(NT);
    for (int t = 0; t < NT; ++t) gj[t] = GramJob{base[t], unf[g], C[g], ng, Hb + mat * t};
    // the Gram kernel writes an ng x ng block with leading dimension ng; pad handled by ld=ne below
    for (int t = 0; t < NT; ++t) gj[t].n = ng;
    ZBC_TRY(upload_jobs(w.jobs_a, gj, st));
    dim3 gg(ceil_div(ng, 32), ceil_div(ng, 32), NT);
    gram_kernel<T><<<gg, 256, 0, st>>>((const GramJob*)w.jobs_a.ptr);
    ZBC_TRY_CUDA(cudaGetLastError());
    if (ne != ng) {
      set_error("odd mode sizes are not supported by the GPU HOSVD (n=%d)", ng);
      return ZBC_EINVAL;
    }
    std::vector<JacJob> jj(NT);
    for (int t = 0; t < NT; ++t) jj[t] = JacJob{Hb + mat * t, V1b + mat * t, ne};
    ZBC_TRY(upload_jobs(w.jobs_b, jj, st));
    const size_t jsm = (size_t)(ne / 2) * (2 * sizeof(double) + sizeof(double2) + 2 * sizeof(int));
    jacobi_kernel<<<NT, 512, jsm, st>>>((const JacJob*)w.jobs_b.ptr, 60, (int*)w.sweeps.ptr);
    ZBC_TRY_CUDA(cudaGetLastError());
    // pass 2: B = V1^H A_(g)  (n x C, column-major), H2 = B B^H
    std::vector<RotJob> rj(NT);
    for (int t = 0; t < NT; ++t)
      rj[t] = RotJob{base[t], unf[g], C[g], ng, ng, ng, V1b + mat * t, Bb + (size_t)nv * t, Unf{1, C[g], ng, 0}};
    ZBC_TRY(upload_jobs(w.jobs_c, rj, st));
    rotate_kernel<T><<<dim3(ceil_div(C[g], 64), ceil_div(ng, 32), NT), 256, 0, st>>>((const RotJob*)w.jobs_c.ptr);
    ZBC_TRY_CUDA(cudaGetLastError());
    for (int t = 0; t < NT; ++t) gj[t] = GramJob{Bb + (size_t)nv * t, Unf{1, C[g], ng, 0}, C[g], ng, Hb + mat * t};
    ZBC_TRY(upload_jobs(w.jobs_a, gj, st));
    gram_kernel<double2><<<gg, 256, 0, st>>>((const GramJob*)w.jobs_a.ptr);
    ZBC_TRY_CUDA(cudaGetLastError());
    for (int t = 0; t < NT; ++t) jj[t] = JacJob{Hb + mat * t, Wb + mat * t, ne};
    ZBC_TRY(upload_jobs(w.jobs_b, jj, st));
    jacobi_kernel<<<NT, 512, jsm, st>>>((const JacJob*)w.jobs_b.ptr, 60, (int*)w.sweeps.ptr);
    ZBC_TRY_CUDA(cudaGetLastError());
    // eigenvalues -> host, rank rule, order
    std::vector<double2> Hh(mat * NT);
    ZBC_TRY_CUDA(cudaMemcpyAsync(Hh.data(), Hb, sizeof(double2) * mat * NT, cudaMemcpyDeviceToHost, st));
    ZBC_TRY_CUDA(cudaStreamSynchronize(st));
    std::vector<int> ord_all((size_t)NT * ng);
    std::vector<FacJob> fj(NT);
    for (int t = 0; t < NT; ++t) {
      std::vector<double> lam(ng);
      for (int i = 0; i < ng; ++i) lam[i] = Hh[mat * t + i + (size_t)ng * i].x;
      std::vector<int> ord(ng);
      std::iota(ord.begin(), ord.end(), 0);
      std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return lam[a] > lam[b]; });
      std::vector<double> ls(ng);
      for (int i = 0; i < ng; ++i) ls[i] = lam[ord[i]];
      const double thr = tol * tol / 3.0 * norm2[t];
      const int r = truncation_rank(ls, thr);
      rk[3 * t + g] = r;
      double tail = 0;
      for (int i = r; i < ng; ++i) tail += std::max(ls[i], 0.0);
      tails[t] += tail;
      for (int i = 0; i < ng; ++i) ord_all[(size_t)t * ng + i] = ord[i];
    }
    ZBC_TRY(w.ord.ensure(sizeof(int) * ord_all.size()));
    ZBC_TRY_CUDA(cudaMemcpyAsync(w.ord.ptr, ord_all.data(), sizeof(int) * ord_all.size(), cudaMemcpyHostToDevice, st));
    for (int t = 0; t < NT; ++t)
      fj[t] = FacJob{V1b + mat * t, Wb + mat * t, (const int*)w.ord.ptr + (size_t)t * ng, ng, rk[3 * t + g],
                     Ub + ustride * t + uoff[g]};
    ZBC_TRY(upload_jobs(w.jobs_d, fj, st));
    factor_kernel<<<dim3(ceil_div((int64_t)ng * nmax, 256), NT), 256, 0, st>>>((const FacJob*)w.jobs_d.ptr);
    ZBC_TRY_CUDA(cudaGetLastError());
    ZBC_TRY_CUDA(cudaStreamSynchronize(st));  // job buffers are reused by the next mode
  }
  for (int t = 0; t < NT; ++t)
    if (norm2[t] > 0) worst = std::max(worst, std::sqrt(tails[t] / norm2[t]));
  *max_err_bound = std::max(*max_err_bound, worst);

  // core = A x1 U1^H x2 U2^H x3 U3^H
  int r1max = 0, r2max = 0;
  for (int t = 0; t < NT; ++t) {
    r1max = std::max(r1max, rk[3 * t]);
    r2max = std::max(r2max, rk[3 * t + 1]);
  }
  const int64_t c1sz = (int64_t)r1max * n2 * n3, c2sz = (int64_t)r1max * r2max * n3;
  ZBC_TRY(w.C1.ensure(sizeof(double2) * c1sz * NT));
  ZBC_TRY(w.C2.ensure(sizeof(double2) * c2sz * NT));
  ZBC_TRY(w.G.ensure(sizeof(double2) * (size_t)nmax * nmax * nmax * 0 + sizeof(double2) * (size_t)r1max * r2max * nmax * NT));
  double2* C1 = (double2*)w.C1.ptr;
  double2* C2 = (double2*)w.C2.ptr;
  double2* Gc = (double2*)w.G.ptr;
  const int64_t gsz = (int64_t)r1max * r2max * nmax;
  std::vector<RotJob> rj(NT);
  int rmax1 = 0;
  for (int t = 0; t < NT; ++t) {
    const int r1 = rk[3 * t];
    rj[t] = RotJob{base[t], unf[0], C[0], n1, r1, n1, Ub + ustride * t + uoff[0], C1 + c1sz * t, Unf{1, C[0], r1, 0}};
    rmax1 = std::max(rmax1, r1);
  }
  ZBC_TRY(upload_jobs(w.jobs_c, rj, st));
  rotate_kernel<T><<<dim3(ceil_div(C[0], 64), ceil_div(rmax1, 32), NT), 256, 0, st>>>((const RotJob*)w.jobs_c.ptr);
  ZBC_TRY_CUDA(cudaGetLastError());
  int rmax2 = 0;
  for (int t = 0; t < NT; ++t) {
    const int r1 = rk[3 * t], r2 = rk[3 * t + 1];
    rj[t] = RotJob{C1 + c1sz * t, Unf{r1, r1, 1, (int64_t)r1 * n2}, (int64_t)r1 * n3, n2, r2, n2,
                   Ub + ustride * t + uoff[1], C2 + c2sz * t, Unf{r1, r1, 1, (int64_t)r1 * r2}};
    rmax2 = std::max(rmax2, r2);
  }
  ZBC_TRY(upload_jobs(w.jobs_d, rj, st));
  rotate_kernel<double2><<<dim3(ceil_div((int64_t)r1max * n3, 64), ceil_div(rmax2, 32), NT), 256, 0, st>>>(
      (const RotJob*)w.jobs_d.ptr);
  ZBC_TRY_CUDA(cudaGetLastError());
  int rmax3 = 0;
  std::vector<RotJob> rj3(NT);
  for (int t = 0; t < NT; ++t) {
    const int r1 = rk[3 * t], r2 = rk[3 * t + 1], r3 = rk[3 * t + 2];
    rj3[t] = RotJob{C2 + c2sz * t, Unf{(int64_t)r1 * r2, (int64_t)r1 * r2, 1, 0}, (int64_t)r1 * r2, n3, r3, n3,
                    Ub + ustride * t + uoff[2], Gc + gsz * t, Unf{(int64_t)r1 * r2, (int64_t)r1 * r2, 1, 0}};
    rmax3 = std::max(rmax3, r3);
  }
  ZBC_TRY(upload_jobs(w.jobs_b, rj3, st));
  rotate_kernel<double2><<<dim3(ceil_div((int64_t)r1max * r2max, 64), ceil_div(rmax3, 32), NT), 256, 0, st>>>(
      (const RotJob*)w.jobs_b.ptr);
  ZBC_TRY_CUDA(cudaGetLastError());

  // pack into complex64: core, U1, U2, U3 per tensor
  int64_t elems = 0;
  std::vector<int64_t> toff(NT);
  for (int t = 0; t < NT; ++t) {
    const int r1 = rk[3 * t], r2 = rk[3 * t + 1], r3 = rk[3 * t + 2];
    toff[t] = elems;
    elems += (int64_t)r1 * r2 * r3 + (int64_t)n1 * r1 + (int64_t)n2 * r2 + (int64_t)n3 * r3;
  }
  float2* pool = nullptr;
  ZBC_TRY_CUDA(cudaMalloc(&pool, sizeof(float2) * std::max<int64_t>(1, elems)));
  std::vector<CopyJob> cj;
  for (int t = 0; t < NT; ++t) {
    const int r1 = rk[3 * t], r2 = rk[3 * t + 1], r3 = rk[3 * t + 2];
    int64_t o = toff[t];
    cj.push_back(CopyJob{Gc + gsz * t, pool + o, (int64_t)r1 * r2 * r3});
    o += (int64_t)r1 * r2 * r3;
    cj.push_back(CopyJob{Ub + ustride * t + uoff[0], pool + o, (int64_t)n1 * r1});
    o += (int64_t)n1 * r1;
    cj.push_back(CopyJob{Ub + ustride * t + uoff[1], pool + o, (int64_t)n2 * r2});
    o += (int64_t)n2 * r2;
    cj.push_back(CopyJob{Ub + ustride * t + uoff[2], pool + o, (int64_t)n3 * r3});
  }
  int st_up = upload_jobs(w.jobs_a, cj, st);
  if (st_up != ZBC_OK) {
    cudaFree(pool);
    return st_up;
  }
  pack_kernel<<<dim3(16, (unsigned)cj.size()), 256, 0, st>>>((const CopyJob*)w.jobs_a.ptr);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(pool);
    set_error("HOSVD pack failed: %s", cudaGetErrorString(e));
    return ZBC_ECUDA;
  }
  for (int t = 0; t < NT; ++t)
    for (int g = 0; g < 3; ++g) ranks_out.push_back(rk[3 * t + g]);
  *pool_out = pool;
  *elems_out = elems;
  return ZBC_OK;
}

int hosvd_compress(const void* cols, int64_t ld, int ncols, int n1, int n2, int n3, int q, zbc_dtype dt,
                   double tol, std::vector<int32_t>& ranks, float2** pool, int64_t* elems, double* max_err,
                   int batch_cols, cudaStream_t st) {
  HosvdWork w;
  std::vector<float2*> pools;
  std::vector<int64_t> sizes;
  int status = ZBC_OK;
  for (int c0 = 0; c0 < ncols && status == ZBC_OK; c0 += batch_cols) {
    const int nc = std::min(batch_cols, ncols - c0);
    const size_t eb = dt == ZBC_C128 ? 16 : 8;
    const void* cptr = (const char*)cols + (size_t)c0 * ld * eb;
    float2* p = nullptr;
    int64_t e = 0;
    if (dt == ZBC_C128)
      status = hosvd_batch<double2>(cptr, ld, nc, n1, n2, n3, q, tol, w, ranks, &p, &e, max_err, st);
    else
      status = hosvd_batch<float2>(cptr, ld, nc, n1, n2, n3, q, tol, w, ranks, &p, &e, max_err, st);
    if (status == ZBC_OK) {
      pools.push_back(p);
      sizes.push_back(e);
    }
  }
  int64_t total = 0;
  for (auto s : sizes) total += s;
  if (status == ZBC_OK) {
    float2* all = nullptr;
    cudaError_t err = cudaMalloc(&all, sizeof(float2) * std::max<int64_t>(1, total));
    if (err != cudaSuccess) {
      set_error("cudaMalloc pool failed");
      status = ZBC_ENOMEM;
    } else {
      int64_t o = 0;
      for (size_t i = 0; i < pools.size(); ++i) {
        cudaMemcpyAsync(all + o, pools[i], sizeof(float2) * sizes[i], cudaMemcpyDeviceToDevice, st);
        o += sizes[i];
      }
      cudaStreamSynchronize(st);
      *pool = all;
      *elems = total;
    }
  }
  for (auto p : pools) cudaFree(p);
  return status;
}

}  // namespace zbc

using namespace zbc;

int randomized_compress_entry(const void* cols, int64_t ld, int ncols, const zbc_grid* g, int q, zbc_dtype in_dt,
                              double tol, zbc_tucker_method method, std::vector<int32_t>& ranks, float2** pool,
                              int64_t* elems, zbc_compress_stats* stats, cudaStream_t st);

extern "C" int tucker_compress(const void* cols, int64_t ld, int ncols, const zbc_grid* g, int q, zbc_dtype in_dt,
                               double tol, zbc_tucker_method method, zbc_handle** out,
                               zbc_compress_stats* stats_host, zbc_stream stream) {
  clear_error();
  ZBC_CHECK_ARG(cols && g && out, "tucker_compress: null argument");
  ZBC_CHECK_ARG(q == 3, "q must be 3");
  ZBC_CHECK_ARG(g->n1 >= 2 && g->n2 >= 2 && g->n3 >= 2 && g->n1 <= 1024 && g->n2 <= 1024 && g->n3 <= 1024,
                "grid sizes must be in [2, 1024]");
  ZBC_CHECK_ARG(g->n1 % 2 == 0 && g->n2 % 2 == 0 && g->n3 % 2 == 0, "grid sizes must be even");
  ZBC_CHECK_ARG(ncols >= 1, "ncols must be >= 1");
  ZBC_CHECK_ARG(tol > 0 && tol < 1, "tol must be in (0, 1)");
  ZBC_CHECK_ARG(in_dt == ZBC_C64 || in_dt == ZBC_C128, "bad dtype");
  const int64_t nv = (int64_t)g->n1 * g->n2 * g->n3;
  ZBC_CHECK_ARG(ld >= q * nv, "ld < q*n_v");
  if (*out) {
    const Handle& h0 = (*out)->h;
    ZBC_CHECK_ARG(h0.n1 == g->n1 && h0.n2 == g->n2 && h0.n3 == g->n3 && h0.q == q && !h0.has_v,
                  "append: grid/q mismatch or handle holds ACA storage");
  }
  std::vector<int32_t> ranks;
  float2* pool = nullptr;
  int64_t elems = 0;
  double max_err = 0.0;
  zbc_compress_stats stats{};
  int s;
  if (method == ZBC_HOSVD) {
    // batch so that the FP64 rotated-unfolding buffer stays near 4 GB
    const int64_t per_col = (int64_t)q * nv * 16;
    int batch = (int)std::max<int64_t>(1, std::min<int64_t>(ncols, ((int64_t)4 << 30) / per_col));
    s = hosvd_compress(cols, ld, ncols, g->n1, g->n2, g->n3, q, in_dt, tol, ranks, &pool, &elems, &max_err, batch,
                       stream);
    stats.max_rel_err = max_err;
  } else {
    s = randomized_compress_entry(cols, ld, ncols, g, q, in_dt, tol, method, ranks, &pool, &elems, &stats, stream);
  }
  if (s != ZBC_OK) return s;
  zbc_handle* hh = *out;
  const bool fresh = hh == nullptr;
  if (fresh) {
    hh = new zbc_handle();
    hh->h.n1 = g->n1;
    hh->h.n2 = g->n2;
    hh->h.n3 = g->n3;
    hh->h.q = q;
  }
  s = handle_append(&hh->h, ranks, pool, elems, ncols, stream);
  cudaFree(pool);
  if (s != ZBC_OK) {
    if (fresh) delete hh;
    return s;
  }
  *out = hh;
  stats.n_tensors = ncols * q;
  for (auto r : ranks) stats.max_rank = std::max(stats.max_rank, r);
  if (stats_host) *stats_host = stats;
  return ZBC_OK;
}
