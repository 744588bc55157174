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

#include "hosvd.cuh"

namespace zbc {

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
// Hermitian Jacobi eigensolver, one CTA per matrix (JacJob, hosvd.cuh)
// ---------------------------------------------------------------------------------------------
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

// U[:, a] = V1 * W[:, ord[a]]  (n x r), FP64 (FacJob, hosvd.cuh)
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

// copy FP64 (src) -> complex64 (dst), several segments per job list (CopyJob, hosvd.cuh)
__global__ void __launch_bounds__(256) pack_kernel(const CopyJob* jobs) {
  const CopyJob jb = jobs[blockIdx.y];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < jb.len; e += (int64_t)gridDim.x * blockDim.x)
    jb.dst[e] = make_float2((float)jb.src[e].x, (float)jb.src[e].y);
}

// launches of the FP64-operand forms for other translation units (hosvd.cuh)
void launch_gram_f64(const GramJob* jobs, dim3 grid, cudaStream_t st) {
  gram_kernel<double2><<<grid, 256, 0, st>>>(jobs);
}
void launch_rotate_f64(const RotJob* jobs, dim3 grid, cudaStream_t st) {
  rotate_kernel<double2><<<grid, 256, 0, st>>>(jobs);
}

// ---------------------------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------------------------
struct HosvdWork {
  DevBuf jobs_a, jobs_b, jobs_c, jobs_d;
  DevBuf H, V1, W, Bbuf, U, C1, C2, G, norm_part, ord, sweeps, base_ptrs;
  DevBuf skpart;  // partial sketches of the split sketch kernel
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

// ---------------------------------------------------------------------------------------------
// Randomized range-finder Tucker with fixed widths and an HOSVD fallback (not in the paper;
// Halko-Martinsson-Tropp range finder per mode as in the randomized HOSVD of Minster, Saibaba
// and Kilmer):  Y_g = A_(g) Omega_g[:, :w_g] (FP64 sketch),  Q_g = orth(Y_g) (FP64 Householder),
// C = A x1 Q1^H x2 Q2^H x3 Q3^H, e^2 = ||A||^2 - ||C||^2 (FP64).  If e^2 > tol^2 ||A||^2 the
// widths failed and the tensor is redone by HOSVD; otherwise C is truncated by HOSVD with the
// remaining budget (tol^2 ||A||^2 - e^2)/3 per mode, U_g = Q_g W_g.  Error <= tol ||A||_F.
// ---------------------------------------------------------------------------------------------
constexpr int kWmax = 64;  // largest sketch width

struct SketchJob {
  const void* A;
  Unf u;
  int64_t C;
  int n, w;
  const float2* Om;  // C x lmax, column-major
  int64_t ldo;
  double2* Y;        // n x w, ld n
};

// Y(x, l) = sum_c A(x, c) Omega(c, l) in FP64.  (An FP32 sketch measured e^2 ~ 1e-13 ||A||^2 of
// rounding noise on the 2 mm workloads, a sixth of the tol^2 = 1e-12 budget at tol 1e-6, which
// inflated ranks; in FP64 the noise floor is far below the budget.)
// Grid (x tiles of 32 rows, jobs, ksplit): with ksplit > 1 the unfolding's columns are cut into
// ksplit ranges of whole 16-column chunks (so one tensor's sketch spreads over many SMs) and each
// range's partial Y goes to part[(job * ksplit + z) * pstride + x + n l], summed in a fixed order
// by sketch_reduce_kernel.
template <typename T>
__global__ void __launch_bounds__(256) sketch_kernel(const SketchJob* jobs, int ksplit, double2* part,
                                                     int64_t pstride) {
  const SketchJob jb = jobs[blockIdx.y];
  const int x0 = blockIdx.x * 32;
  if (x0 >= jb.n) return;
  const int64_t chunk = ((jb.C + ksplit - 1) / ksplit + 15) / 16 * 16;
  const int64_t cbeg = (int64_t)blockIdx.z * chunk, cend = min(jb.C, cbeg + chunk);
  __shared__ double2 sa[16][33];
  __shared__ double2 so[16][kWmax + 1];
  const int lx = threadIdx.x % 32, lg = threadIdx.x / 32;
  double2 acc[kWmax / 8];
#pragma unroll
  for (int i = 0; i < kWmax / 8; ++i) acc[i] = make_double2(0.0, 0.0);
  for (int64_t c0 = cbeg; c0 < cend; c0 += 16) {
    for (int e = threadIdx.x; e < 16 * 32; e += 256) {
      const int cc = e / 32, xx = e % 32;
      const int64_t c = c0 + cc;
      double2 v = make_double2(0.0, 0.0);
      if (c < cend && x0 + xx < jb.n) v = ld_z<T>(jb.A, jb.u.at(x0 + xx, c));
      sa[cc][xx] = v;
    }
    for (int e = threadIdx.x; e < 16 * kWmax; e += 256) {
      const int cc = e / kWmax, l = e % kWmax;
      const int64_t c = c0 + cc;
      double2 v = make_double2(0.0, 0.0);
      if (c < cend && l < jb.w) {
        const float2 o = jb.Om[c + jb.ldo * l];
        v = make_double2(o.x, o.y);
      }
      so[cc][l] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int cc = 0; cc < 16; ++cc) {
      const double2 a = sa[cc][lx];
#pragma unroll
      for (int i = 0; i < kWmax / 8; ++i) acc[i] = zfma(a, so[cc][lg + 8 * i], acc[i]);
    }
    __syncthreads();
  }
  double2* out = ksplit > 1 ? part + ((int64_t)blockIdx.y * ksplit + blockIdx.z) * pstride : jb.Y;
#pragma unroll
  for (int i = 0; i < kWmax / 8; ++i) {
    const int l = lg + 8 * i;
    if (x0 + lx < jb.n && l < jb.w) out[(x0 + lx) + (int64_t)jb.n * l] = acc[i];
  }
}

// Y = sum over z of the ksplit partial sketches, in order z = 0, 1, ... (grid (x, jobs))
__global__ void __launch_bounds__(256) sketch_reduce_kernel(const SketchJob* jobs, int ksplit,
                                                            const double2* __restrict__ part, int64_t pstride) {
  const SketchJob jb = jobs[blockIdx.y];
  const int64_t ne = (int64_t)jb.n * jb.w;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int z = 0; z < ksplit; ++z) {
      const double2 v = part[((int64_t)blockIdx.y * ksplit + z) * pstride + e];
      s.x += v.x;
      s.y += v.y;
    }
    jb.Y[e] = s;
  }
}

// Householder QR of Y (n x w), keeping only Q (n x w, orthonormal columns).  The reflector
// vectors overwrite Y; H_k = I - 2 v v^H / |v|^2 maps column k to a multiple of e_k.
struct QrJob {
  double2* Y;
  int n, w;
  double2* Q;
};
__device__ __forceinline__ double2 block_sum2(double2 v, double2* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double2 s = make_double2(0, 0);
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    s.x += red[w].x;
    s.y += red[w].y;
  }
  return s;
}
__global__ void __launch_bounds__(256) qr_kernel(const QrJob* jobs) {
  const QrJob jb = jobs[blockIdx.x];
  const int n = jb.n, w = jb.w;
  double2* Y = jb.Y;
  __shared__ double vn2[kWmax];
  __shared__ double2 red[8];
  __shared__ double2 dots[kWmax];
  for (int k = 0; k < w; ++k) {
    double2 part = make_double2(0, 0);
    for (int r = k + threadIdx.x; r < n; r += blockDim.x) {
      const double2 y = Y[r + (int64_t)n * k];
      part.x += y.x * y.x + y.y * y.y;
    }
    const double nx2 = block_sum2(part, red).x;
    const double2 x0 = Y[k + (int64_t)n * k];
    const double ax0 = hypot(x0.x, x0.y);
    const double nx = sqrt(nx2);
    // v = x + e^{i arg x0} |x| e_k
    const double2 ph = ax0 > 0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1, 0);
    const double2 v0 = make_double2(x0.x + ph.x * nx, x0.y + ph.y * nx);
    const double v2 = nx2 - ax0 * ax0 + (v0.x * v0.x + v0.y * v0.y);
    __syncthreads();
    if (threadIdx.x == 0) {
      Y[k + (int64_t)n * k] = v0;
      vn2[k] = nx > 0 ? v2 : 0.0;
    }
    __syncthreads();
    if (vn2[k] == 0.0) continue;
    // apply H_k to columns j > k: y_j -= 2 v (v^H y_j) / |v|^2
    for (int j = k + 1; j < w; ++j) {
      double2 d = make_double2(0, 0);
      for (int r = k + threadIdx.x; r < n; r += blockDim.x) d = zfma_conj(Y[r + (int64_t)n * k], Y[r + (int64_t)n * j], d);
      const double2 s = block_sum2(d, red);
      const double f = 2.0 / vn2[k];
      for (int r = k + threadIdx.x; r < n; r += blockDim.x) {
        const double2 v = Y[r + (int64_t)n * k];
        double2& y = Y[r + (int64_t)n * j];
        y.x -= f * (v.x * s.x - v.y * s.y);
        y.y -= f * (v.x * s.y + v.y * s.x);
      }
      __syncthreads();
    }
  }
  // Q = H_0 ... H_{w-1} [e_0 .. e_{w-1}]
  double2* Q = jb.Q;
  for (int64_t e = threadIdx.x; e < (int64_t)n * w; e += blockDim.x) {
    const int r = (int)(e % n), c = (int)(e / n);
    Q[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = w - 1; k >= 0; --k) {
    if (vn2[k] == 0.0) continue;
    for (int c = k; c < w; ++c) {
      double2 d = make_double2(0, 0);
      for (int r = k + threadIdx.x; r < n; r += blockDim.x) d = zfma_conj(Y[r + (int64_t)n * k], Q[r + (int64_t)n * c], d);
      const double2 s = block_sum2(d, red);
      if (threadIdx.x == 0) dots[c] = s;
    }
    __syncthreads();
    const double f = 2.0 / vn2[k];
    for (int64_t e = threadIdx.x; e < (int64_t)(n - k) * (w - k); e += blockDim.x) {
      const int r = k + (int)(e % (n - k)), c = k + (int)(e / (n - k));
      const double2 v = Y[r + (int64_t)n * k], s = dots[c];
      double2& q = Q[r + (int64_t)n * c];
      q.x -= f * (v.x * s.x - v.y * s.y);
      q.y -= f * (v.x * s.y + v.y * s.x);
    }
    __syncthreads();
  }
}

struct NormJob {
  const double2* p;
  int64_t len;
};
__global__ void __launch_bounds__(256) norm_jobs_kernel(const NormJob* jobs, double* partial) {
  const NormJob jb = jobs[blockIdx.y];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < jb.len; i += (int64_t)gridDim.x * blockDim.x)
    s += jb.p[i].x * jb.p[i].x + jb.p[i].y * jb.p[i].y;
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// U[i, a] = sum_l Q[i + n l] W[l + lw ord[a]]   (Q n x w, W w x w eigenvectors with ld lw)
struct Fac2Job {
  const double2* Q;
  const double2* W;
  const int* ord;
  int n, w, lw, r;
  double2* U;
};
__global__ void __launch_bounds__(256) factor2_kernel(const Fac2Job* jobs) {
  const Fac2Job jb = jobs[blockIdx.y];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < jb.n * jb.r; e += gridDim.x * blockDim.x) {
    const int i = e % jb.n, a = e / jb.n;
    const int col = jb.ord[a];
    double2 s = make_double2(0, 0);
    for (int l = 0; l < jb.w; ++l) s = zfma(jb.Q[i + (int64_t)jb.n * l], jb.W[l + (int64_t)jb.lw * col], s);
    jb.U[i + (int64_t)jb.n * a] = s;
  }
}

__global__ void set_pad_kernel(double2* H, int ne, int w) {
  // decoupled pad row/column of an odd-size Gram: diagonal -1 so it sorts last
  if (threadIdx.x == 0 && w < ne) H[w + (int64_t)ne * w] = make_double2(-1.0, 0.0);
}

// One batch of tensors: randomized compression of those that pass; the others are listed in
// *fallback.  Per passing tensor t the packed complex64 data goes to out_pool[t] (device,
// allocated here) with elems out_elems[t].
template <typename T>
static int randomized_batch(const void* cols, int64_t ld, int ncols, int n1, int n2, int n3, int q, double tol,
                            const int32_t* widths, const float2* const* sketch, int lmax, HosvdWork& w,
                            std::vector<int32_t>& ranks_out, std::vector<int>& fallback, std::vector<float2*>& out_pool,
                            std::vector<int64_t>& out_elems, double* max_err, cudaStream_t st) {
  const int64_t nv = (int64_t)n1 * n2 * n3;
  const int NT = ncols * q;
  const int n[3] = {n1, n2, n3};
  const int64_t Cn[3] = {nv / n1, nv / n2, nv / n3};
  const Unf unf[3] = {{1, nv / n1, n1, 0}, {n1, n1, 1, (int64_t)n1 * n2}, {(int64_t)n1 * n2, (int64_t)n1 * n2, 1, 0}};
  const size_t eb = sizeof(T);
  std::vector<const void*> base(NT);
  for (int t = 0; t < NT; ++t) base[t] = (const char*)cols + ((int64_t)(t / q) * ld + (int64_t)(t % q) * nv) * eb;
  std::vector<int> wd(3 * (size_t)NT);
  // widths are even (the Jacobi solver pairs rows); an odd request is rounded up when room allows
  for (int t = 0; t < NT; ++t)
    for (int g = 0; g < 3; ++g) {
      const int cap = std::min({n[g], kWmax, lmax}) / 2 * 2;
      int wv = std::max(2, std::min((int)widths[3 * t + g], cap));
      if (wv & 1) wv = wv + 1 <= cap ? wv + 1 : wv - 1;
      wd[3 * t + g] = wv;
    }
  // ||A||^2
  ZBC_TRY(w.base_ptrs.ensure(sizeof(void*) * NT));
  ZBC_TRY_CUDA(cudaMemcpyAsync(w.base_ptrs.ptr, base.data(), sizeof(void*) * NT, cudaMemcpyHostToDevice, st));
  ZBC_TRY(w.norm_part.ensure(sizeof(double) * 64 * NT));
  norm2_kernel<T><<<dim3(64, NT), 256, 0, st>>>((const void* const*)w.base_ptrs.ptr, nv, (double*)w.norm_part.ptr);
  count_launch();
  std::vector<double> part(64 * (size_t)NT), norm2(NT, 0.0);
  ZBC_TRY_CUDA(cudaMemcpyAsync(part.data(), w.norm_part.ptr, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st));
  // sketches and Q factors: Qbuf[t] holds Q1 (n1 x w1), Q2, Q3
  const int64_t qstride = (int64_t)(n1 + n2 + n3) * kWmax;
  ZBC_TRY(w.U.ensure(sizeof(double2) * qstride * NT));       // Q factors
  ZBC_TRY(w.Bbuf.ensure(sizeof(double2) * qstride * NT));    // sketches Y (overwritten by reflectors)
  double2* Qb = (double2*)w.U.ptr;
  double2* Yb = (double2*)w.Bbuf.ptr;
  const int64_t qoff[3] = {0, (int64_t)n1 * kWmax, (int64_t)(n1 + n2) * kWmax};
  std::vector<SketchJob> sj;
  std::vector<QrJob> qj;
  for (int t = 0; t < NT; ++t)
    for (int g = 0; g < 3; ++g) {
      sj.push_back(SketchJob{base[t], unf[g], Cn[g], n[g], wd[3 * t + g], sketch[g], Cn[g],
                             Yb + qstride * t + qoff[g]});
      qj.push_back(QrJob{Yb + qstride * t + qoff[g], n[g], wd[3 * t + g], Qb + qstride * t + qoff[g]});
    }
  ZBC_TRY(upload_jobs(w.jobs_a, sj, st));
  const int nmax = std::max(n1, std::max(n2, n3));
  // split the unfolding's columns when the x tiles of all jobs fill fewer than 4 CTAs per SM
  const int64_t tiles = (int64_t)ceil_div(nmax, 32) * (int64_t)sj.size();
  const int ksplit = (int)std::max<int64_t>(1, std::min<int64_t>(32, (4 * sm_count() + tiles - 1) / tiles));
  const int64_t pstride = (int64_t)nmax * kWmax;
  if (ksplit > 1) ZBC_TRY(w.skpart.ensure(sizeof(double2) * pstride * ksplit * sj.size()));
  sketch_kernel<T><<<dim3(ceil_div(nmax, 32), (unsigned)sj.size(), ksplit), 256, 0, st>>>(
      (const SketchJob*)w.jobs_a.ptr, ksplit, (double2*)w.skpart.ptr, pstride);
  count_launch();
  if (ksplit > 1) {
    sketch_reduce_kernel<<<dim3(ceil_div(pstride, 256), (unsigned)sj.size()), 256, 0, st>>>(
        (const SketchJob*)w.jobs_a.ptr, ksplit, (const double2*)w.skpart.ptr, pstride);
    count_launch();
  }
  ZBC_TRY(upload_jobs(w.jobs_b, qj, st));
  qr_kernel<<<(unsigned)qj.size(), 256, 0, st>>>((const QrJob*)w.jobs_b.ptr);
  count_launch();
  ZBC_TRY_CUDA(cudaGetLastError());
  // C = A x1 Q1^H x2 Q2^H x3 Q3^H
  int w1m = 0, w2m = 0;
  for (int t = 0; t < NT; ++t) {
    w1m = std::max(w1m, wd[3 * t]);
    w2m = std::max(w2m, wd[3 * t + 1]);
  }
  const int64_t c1sz = (int64_t)w1m * n2 * n3, c2sz = (int64_t)w1m * w2m * n3, csz = (int64_t)w1m * w2m * kWmax;
  ZBC_TRY(w.C1.ensure(sizeof(double2) * c1sz * NT));
  ZBC_TRY(w.C2.ensure(sizeof(double2) * c2sz * NT));
  ZBC_TRY(w.G.ensure(sizeof(double2) * csz * NT));
  double2* C1 = (double2*)w.C1.ptr;
  double2* C2 = (double2*)w.C2.ptr;
  double2* Cc = (double2*)w.G.ptr;
  std::vector<RotJob> r1j(NT), r2j(NT), r3j(NT);
  for (int t = 0; t < NT; ++t) {
    const int a = wd[3 * t], b = wd[3 * t + 1], c = wd[3 * t + 2];
    r1j[t] = RotJob{base[t], unf[0], Cn[0], n1, a, n1, Qb + qstride * t + qoff[0], C1 + c1sz * t, Unf{1, Cn[0], a, 0}};
    r2j[t] = RotJob{C1 + c1sz * t, Unf{a, a, 1, (int64_t)a * n2}, (int64_t)a * n3, n2, b, n2, Qb + qstride * t + qoff[1],
                    C2 + c2sz * t, Unf{a, a, 1, (int64_t)a * b}};
    r3j[t] = RotJob{C2 + c2sz * t, Unf{(int64_t)a * b, (int64_t)a * b, 1, 0}, (int64_t)a * b, n3, c, n3,
                    Qb + qstride * t + qoff[2], Cc + csz * t, Unf{(int64_t)a * b, (int64_t)a * b, 1, 0}};
  }
  ZBC_TRY(upload_jobs(w.jobs_c, r1j, st));
  rotate_kernel<T><<<dim3(ceil_div(Cn[0], 64), ceil_div(w1m, 32), NT), 256, 0, st>>>((const RotJob*)w.jobs_c.ptr);
  ZBC_TRY(upload_jobs(w.jobs_d, r2j, st));
  rotate_kernel<double2><<<dim3(ceil_div((int64_t)w1m * n3, 64), ceil_div(w2m, 32), NT), 256, 0, st>>>(
      (const RotJob*)w.jobs_d.ptr);
  ZBC_TRY_CUDA(cudaStreamSynchronize(st));
  ZBC_TRY(upload_jobs(w.jobs_c, r3j, st));
  rotate_kernel<double2><<<dim3(ceil_div((int64_t)w1m * w2m, 64), 2, NT), 256, 0, st>>>((const RotJob*)w.jobs_c.ptr);
  count_launch(3);
  // ||C||^2 and the projection test
  std::vector<NormJob> nj(NT);
  for (int t = 0; t < NT; ++t) nj[t] = NormJob{Cc + csz * t, (int64_t)wd[3 * t] * wd[3 * t + 1] * wd[3 * t + 2]};
  ZBC_TRY(upload_jobs(w.jobs_d, nj, st));
  ZBC_TRY(w.sweeps.ensure(sizeof(double) * 16 * NT));
  norm_jobs_kernel<<<dim3(16, NT), 256, 0, st>>>((const NormJob*)w.jobs_d.ptr, (double*)w.sweeps.ptr);
  count_launch();
  std::vector<double> cpart(16 * (size_t)NT);
  ZBC_TRY_CUDA(cudaMemcpyAsync(cpart.data(), w.sweeps.ptr, sizeof(double) * cpart.size(), cudaMemcpyDeviceToHost, st));
  ZBC_TRY_CUDA(cudaStreamSynchronize(st));
  std::vector<double> budget(NT, -1.0);
  std::vector<int> pass;
  for (int t = 0; t < NT; ++t) {
    for (int b = 0; b < 64; ++b) norm2[t] += part[(size_t)t * 64 + b];
    double c2n = 0.0;
    for (int b = 0; b < 16; ++b) c2n += cpart[(size_t)t * 16 + b];
    const double e2 = std::max(norm2[t] - c2n, 0.0);
    budget[t] = tol * tol * norm2[t] - e2;
    if (budget[t] < 0.0 || norm2[t] == 0.0)
      fallback.push_back(t);
    else
      pass.push_back(t);
  }
  out_pool.assign(NT, nullptr);
  out_elems.assign(NT, 0);
  ranks_out.assign(3 * (size_t)NT, 0);
  if (pass.empty()) return ZBC_OK;
  // truncate C by HOSVD with per-mode threshold budget/3 (one-pass Gram + Jacobi on the small core)
  const int P = (int)pass.size();
  const int wme = kWmax;  // padded Gram size bound
  ZBC_TRY(w.H.ensure(sizeof(double2) * (size_t)wme * wme * P));
  ZBC_TRY(w.W.ensure(sizeof(double2) * (size_t)wme * wme * P * 3));
  double2* Hb = (double2*)w.H.ptr;
  double2* Wb = (double2*)w.W.ptr;
  std::vector<int> rk(3 * (size_t)P);
  std::vector<double> trunc_tail(P, 0.0);
  std::vector<int> ord_all;
  std::vector<int64_t> ord_off(3 * (size_t)P);
  for (int g = 0; g < 3; ++g) {
    std::vector<GramJob> gj(P);
    std::vector<JacJob> jj(P);
    std::vector<int> we(P);
    ZBC_TRY_CUDA(cudaMemsetAsync(Hb, 0, sizeof(double2) * (size_t)wme * wme * P, st));
    for (int pi = 0; pi < P; ++pi) {
      const int t = pass[pi];
      const int a = wd[3 * t], b = wd[3 * t + 1], c = wd[3 * t + 2];
      const int dims[3] = {a, b, c};
      const int wg = dims[g];
      we[pi] = wg + (wg & 1);
      const Unf cu[3] = {{1, (int64_t)b * c, a, 0}, {a, a, 1, (int64_t)a * b}, {(int64_t)a * b, (int64_t)a * b, 1, 0}};
      const int64_t Cg = (int64_t)a * b * c / wg;
      gj[pi] = GramJob{Cc + csz * t, cu[g], Cg, wg, Hb + (size_t)wme * wme * pi};
      jj[pi] = JacJob{Hb + (size_t)wme * wme * pi, Wb + (size_t)wme * wme * (3 * pi + g), we[pi]};
    }
    ZBC_TRY(upload_jobs(w.jobs_a, gj, st));
    gram_kernel<double2><<<dim3(2, 2, P), 256, 0, st>>>((const GramJob*)w.jobs_a.ptr);
    ZBC_TRY(upload_jobs(w.jobs_b, jj, st));
    const size_t jsm = (size_t)(wme / 2) * (2 * sizeof(double) + sizeof(double2) + 2 * sizeof(int));
    jacobi_kernel<<<P, 512, jsm, st>>>((const JacJob*)w.jobs_b.ptr, 60, nullptr);
    count_launch(2);
    std::vector<double2> Hh((size_t)wme * wme * P);
    ZBC_TRY_CUDA(cudaMemcpyAsync(Hh.data(), Hb, sizeof(double2) * Hh.size(), cudaMemcpyDeviceToHost, st));
    ZBC_TRY_CUDA(cudaStreamSynchronize(st));
    for (int pi = 0; pi < P; ++pi) {
      const int t = pass[pi];
      const int dims[3] = {wd[3 * t], wd[3 * t + 1], wd[3 * t + 2]};
      const int wg = dims[g], e = we[pi];
      std::vector<double> lam(e);
      for (int i = 0; i < e; ++i) lam[i] = Hh[(size_t)wme * wme * pi + i + (size_t)e * i].x;
      std::vector<int> ord(e);
      std::iota(ord.begin(), ord.end(), 0);
      std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return lam[x] > lam[y]; });
      std::vector<double> ls(wg);
      for (int i = 0; i < wg; ++i) ls[i] = lam[ord[i]];
      const int r = truncation_rank(ls, budget[t] / 3.0);
      for (int i = r; i < wg; ++i) trunc_tail[pi] += std::max(ls[i], 0.0);
      rk[3 * pi + g] = r;
      ord_off[3 * pi + g] = (int64_t)ord_all.size();
      for (int i = 0; i < r; ++i) ord_all.push_back(ord[i]);
    }
  }
  ZBC_TRY(w.ord.ensure(sizeof(int) * std::max<size_t>(1, ord_all.size())));
  ZBC_TRY_CUDA(cudaMemcpyAsync(w.ord.ptr, ord_all.data(), sizeof(int) * ord_all.size(), cudaMemcpyHostToDevice, st));
  // U_g = Q_g W_g (n_g x r_g) into Yb (reused)
  std::vector<Fac2Job> fj;
  for (int pi = 0; pi < P; ++pi) {
    const int t = pass[pi];
    for (int g = 0; g < 3; ++g) {
      const int wg = wd[3 * t + g];
      const int e = wg + (wg & 1);
      fj.push_back(Fac2Job{Qb + qstride * t + qoff[g], Wb + (size_t)wme * wme * (3 * pi + g),
                           (const int*)w.ord.ptr + ord_off[3 * pi + g], n[g], wg, e, rk[3 * pi + g],
                           Yb + qstride * t + qoff[g]});
    }
  }
  ZBC_TRY(upload_jobs(w.jobs_a, fj, st));
  factor2_kernel<<<dim3(ceil_div((int64_t)nmax * kWmax, 256), (unsigned)fj.size()), 256, 0, st>>>(
      (const Fac2Job*)w.jobs_a.ptr);
  // core G = C x1 W1^H x2 W2^H x3 W3^H  (W_g: the first r_g sorted eigenvectors, rows < w_g)
  // build compact W factors (w_g x r_g, ld w_g) by reusing factor2 with Q = identity is
  // avoided: the rotation reads W through ord directly via a gathered copy.
  std::vector<double2> Wh((size_t)wme * wme * P * 3);
  ZBC_TRY_CUDA(cudaMemcpyAsync(Wh.data(), Wb, sizeof(double2) * Wh.size(), cudaMemcpyDeviceToHost, st));
  ZBC_TRY_CUDA(cudaStreamSynchronize(st));
  std::vector<double2> Wc((size_t)wme * wme * P * 3);
  for (int pi = 0; pi < P; ++pi) {
    const int t = pass[pi];
    for (int g = 0; g < 3; ++g) {
      const int wg = wd[3 * t + g], e = wg + (wg & 1), r = rk[3 * pi + g];
      for (int a = 0; a < r; ++a) {
        const int col = ord_all[ord_off[3 * pi + g] + a];
        for (int l = 0; l < wg; ++l)
          Wc[(size_t)wme * wme * (3 * pi + g) + l + (size_t)wg * a] = Wh[(size_t)wme * wme * (3 * pi + g) + l + (size_t)e * col];
      }
    }
  }
  ZBC_TRY_CUDA(cudaMemcpyAsync(Wb, Wc.data(), sizeof(double2) * Wc.size(), cudaMemcpyHostToDevice, st));
  std::vector<RotJob> g1(P), g2(P), g3(P);
  int r1m = 0, r2m = 0, r3m = 0;
  for (int pi = 0; pi < P; ++pi) {
    const int t = pass[pi];
    const int a = wd[3 * t], b = wd[3 * t + 1], c = wd[3 * t + 2];
    const int ra = rk[3 * pi], rb = rk[3 * pi + 1], rc = rk[3 * pi + 2];
    r1m = std::max(r1m, ra);
    r2m = std::max(r2m, rb);
    r3m = std::max(r3m, rc);
    // C (a,b,c) -> T1 (ra,b,c) -> T2 (ra,rb,c) -> G (ra,rb,rc); T1 in C1, T2 in C2, G in C1 (after T1 consumed)
    g1[pi] = RotJob{Cc + csz * t, Unf{1, (int64_t)b * c, a, 0}, (int64_t)b * c, a, ra, a,
                    Wb + (size_t)wme * wme * (3 * pi), C1 + c1sz * t, Unf{1, (int64_t)b * c, ra, 0}};
    g2[pi] = RotJob{C1 + c1sz * t, Unf{ra, ra, 1, (int64_t)ra * b}, (int64_t)ra * c, b, rb, b,
                    Wb + (size_t)wme * wme * (3 * pi + 1), C2 + c2sz * t, Unf{ra, ra, 1, (int64_t)ra * rb}};
    g3[pi] = RotJob{C2 + c2sz * t, Unf{(int64_t)ra * rb, (int64_t)ra * rb, 1, 0}, (int64_t)ra * rb, c, rc, c,
                    Wb + (size_t)wme * wme * (3 * pi + 2), Cc + csz * t, Unf{(int64_t)ra * rb, (int64_t)ra * rb, 1, 0}};
  }
  ZBC_TRY(upload_jobs(w.jobs_b, g1, st));
  rotate_kernel<double2><<<dim3(ceil_div((int64_t)kWmax * kWmax, 64), ceil_div(r1m, 32), P), 256, 0, st>>>(
      (const RotJob*)w.jobs_b.ptr);
  ZBC_TRY(upload_jobs(w.jobs_c, g2, st));
  rotate_kernel<double2><<<dim3(ceil_div((int64_t)r1m * kWmax, 64), ceil_div(r2m, 32), P), 256, 0, st>>>(
      (const RotJob*)w.jobs_c.ptr);
  ZBC_TRY(upload_jobs(w.jobs_d, g3, st));
  rotate_kernel<double2><<<dim3(ceil_div((int64_t)r1m * r2m, 64), ceil_div(r3m, 32), P), 256, 0, st>>>(
      (const RotJob*)w.jobs_d.ptr);
  count_launch(4);
  // pack passing tensors into per-tensor complex64 buffers
  for (int pi = 0; pi < P; ++pi) {
    const int t = pass[pi];
    const int r1 = rk[3 * pi], r2 = rk[3 * pi + 1], r3 = rk[3 * pi + 2];
    const int64_t elems = (int64_t)r1 * r2 * r3 + (int64_t)n1 * r1 + (int64_t)n2 * r2 + (int64_t)n3 * r3;
    float2* pp = nullptr;
    ZBC_TRY_CUDA(cudaMalloc(&pp, sizeof(float2) * elems));
    out_pool[t] = pp;
    out_elems[t] = elems;
    ranks_out[3 * t] = r1;
    ranks_out[3 * t + 1] = r2;
    ranks_out[3 * t + 2] = r3;
    // certified bound: projection error e^2 plus the truncated tails of the core
    const double e2 = std::max(0.0, tol * tol * norm2[t] - budget[t]);
    *max_err = std::max(*max_err, std::sqrt((e2 + trunc_tail[pi]) / norm2[t]));
  }
  std::vector<CopyJob> cj;
  for (int pi = 0; pi < P; ++pi) {
    const int t = pass[pi];
    const int r1 = rk[3 * pi], r2 = rk[3 * pi + 1], r3 = rk[3 * pi + 2];
    float2* o = out_pool[t];
    cj.push_back(CopyJob{Cc + csz * t, o, (int64_t)r1 * r2 * r3});
    o += (int64_t)r1 * r2 * r3;
    cj.push_back(CopyJob{Yb + qstride * t + qoff[0], o, (int64_t)n1 * r1});
    o += (int64_t)n1 * r1;
    cj.push_back(CopyJob{Yb + qstride * t + qoff[1], o, (int64_t)n2 * r2});
    o += (int64_t)n2 * r2;
    cj.push_back(CopyJob{Yb + qstride * t + qoff[2], o, (int64_t)n3 * r3});
  }
  ZBC_TRY(upload_jobs(w.jobs_a, cj, st));
  pack_kernel<<<dim3(8, (unsigned)cj.size()), 256, 0, st>>>((const CopyJob*)w.jobs_a.ptr);
  count_launch();
  ZBC_TRY_CUDA(cudaGetLastError());
  ZBC_TRY_CUDA(cudaStreamSynchronize(st));
  return ZBC_OK;
}

int randomized_compress(const void* cols, int64_t ld, int ncols, int n1, int n2, int n3, int q, zbc_dtype dt,
                        double tol, const int32_t* widths, const float2* const* sketch, int lmax,
                        std::vector<int32_t>& ranks, float2** pool, int64_t* elems, zbc_compress_stats* stats,
                        cudaStream_t st) {
  const int64_t nv = (int64_t)n1 * n2 * n3;
  const size_t eb = dt == ZBC_C128 ? 16 : 8;
  const int T = ncols * q;
  std::vector<float2*> tpool(T, nullptr);
  std::vector<int64_t> telems(T, 0);
  std::vector<int32_t> trank(3 * (size_t)T, 0);
  std::vector<int> fb_all;
  double max_err = 0.0;
  HosvdWork w;
  int status = ZBC_OK;
  const int batch = std::max(1, std::min(ncols, 64));
  for (int c0 = 0; c0 < ncols && status == ZBC_OK; c0 += batch) {
    const int nc = std::min(batch, ncols - c0);
    const void* cptr = (const char*)cols + (size_t)c0 * ld * eb;
    std::vector<int32_t> rk;
    std::vector<int> fb;
    std::vector<float2*> op;
    std::vector<int64_t> oe;
    status = dt == ZBC_C128 ? randomized_batch<double2>(cptr, ld, nc, n1, n2, n3, q, tol, widths + 3 * (size_t)c0 * q,
                                                        sketch, lmax, w, rk, fb, op, oe, &max_err, st)
                            : randomized_batch<float2>(cptr, ld, nc, n1, n2, n3, q, tol, widths + 3 * (size_t)c0 * q,
                                                       sketch, lmax, w, rk, fb, op, oe, &max_err, st);
    if (status != ZBC_OK) break;
    for (int t = 0; t < nc * q; ++t) {
      const int tt = c0 * q + t;
      tpool[tt] = op[t];
      telems[tt] = oe[t];
      for (int g = 0; g < 3; ++g) trank[3 * tt + g] = rk[3 * t + g];
    }
    for (int t : fb) fb_all.push_back(c0 * q + t);
  }
  // HOSVD fallback on the failed tensors (gathered as single-tensor columns)
  if (status == ZBC_OK && !fb_all.empty()) {
    void* tmp = nullptr;
    const int nf = (int)fb_all.size();
    const int fb_batch = std::max(1, std::min(nf, (int)(((int64_t)2 << 30) / (nv * (int64_t)eb))));
    for (int f0 = 0; f0 < nf && status == ZBC_OK; f0 += fb_batch) {
      const int nb = std::min(fb_batch, nf - f0);
      if (cudaMalloc(&tmp, eb * nv * nb) != cudaSuccess) {
        set_error("fallback buffer allocation failed");
        status = ZBC_ENOMEM;
        break;
      }
      for (int i = 0; i < nb; ++i) {
        const int t = fb_all[f0 + i];
        cudaMemcpyAsync((char*)tmp + eb * nv * i, (const char*)cols + ((int64_t)(t / q) * ld + (int64_t)(t % q) * nv) * eb,
                        eb * nv, cudaMemcpyDeviceToDevice, st);
      }
      std::vector<int32_t> rk;
      float2* fp = nullptr;
      int64_t fe = 0;
      status = hosvd_compress(tmp, nv, nb, n1, n2, n3, 1, dt, tol, rk, &fp, &fe, &max_err, nb, st);
      cudaFree(tmp);
      if (status != ZBC_OK) break;
      int64_t o = 0;
      for (int i = 0; i < nb; ++i) {
        const int t = fb_all[f0 + i];
        const int r1 = rk[3 * i], r2 = rk[3 * i + 1], r3 = rk[3 * i + 2];
        const int64_t e = (int64_t)r1 * r2 * r3 + (int64_t)n1 * r1 + (int64_t)n2 * r2 + (int64_t)n3 * r3;
        float2* pp = nullptr;
        cudaMalloc(&pp, sizeof(float2) * e);
        cudaMemcpyAsync(pp, fp + o, sizeof(float2) * e, cudaMemcpyDeviceToDevice, st);
        o += e;
        tpool[t] = pp;
        telems[t] = e;
        trank[3 * t] = r1;
        trank[3 * t + 1] = r2;
        trank[3 * t + 2] = r3;
      }
      cudaStreamSynchronize(st);
      cudaFree(fp);
    }
  }
  if (status == ZBC_OK) {
    int64_t total = 0;
    for (auto e : telems) total += e;
    float2* all = nullptr;
    if (cudaMalloc(&all, sizeof(float2) * std::max<int64_t>(1, total)) != cudaSuccess) {
      set_error("pool allocation failed");
      status = ZBC_ENOMEM;
    } else {
      int64_t o = 0;
      for (int t = 0; t < T; ++t) {
        cudaMemcpyAsync(all + o, tpool[t], sizeof(float2) * telems[t], cudaMemcpyDeviceToDevice, st);
        o += telems[t];
      }
      cudaStreamSynchronize(st);
      *pool = all;
      *elems = total;
      ranks = trank;
      if (stats) {
        stats->n_fallback = (int)fb_all.size();
        stats->max_rel_err = max_err;
      }
    }
  }
  for (auto p : tpool)
    if (p) cudaFree(p);
  return status;
}

}  // namespace zbc

using namespace zbc;

// Append the compressed columns (ranks, packed pool) to *out (a new handle when *out is null).
int finish_compress(zbc_handle** out, const zbc_grid* g, int q, int ncols, const std::vector<int32_t>& ranks,
                           float2* pool, int64_t elems, zbc_compress_stats& stats, zbc_compress_stats* stats_host,
                           cudaStream_t stream) {
  zbc_handle* hh = *out;
  const bool fresh = hh == nullptr;
  if (fresh) {
    hh = new zbc_handle();
    hh->h.n1 = g->n1;
    hh->h.n2 = g->n2;
    hh->h.n3 = g->n3;
    hh->h.q = q;
  }
  const int s = handle_append(&hh->h, ranks, pool, elems, ncols, stream);
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

int check_compress_args(const void* cols, int64_t ld, int ncols, const zbc_grid* g, int q, zbc_dtype in_dt,
                               double tol, zbc_handle** out) {
  ZBC_CHECK_ARG(cols && g && out, "tucker_compress: null argument");
  ZBC_CHECK_ARG(q >= 1 && q <= 12, "q must be in [1, 12]");
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
  return ZBC_OK;
}

extern "C" int tucker_compress_randomized(const void* cols, int64_t ld, int ncols, const zbc_grid* g, int q,
                                          zbc_dtype in_dt, double tol, const int32_t* widths_host,
                                          const void* sketch1, const void* sketch2, const void* sketch3, int lmax,
                                          zbc_handle** out, zbc_compress_stats* stats_host, zbc_stream stream) {
  clear_error();
  ZBC_TRY(check_compress_args(cols, ld, ncols, g, q, in_dt, tol, out));
  ZBC_CHECK_ARG(widths_host && sketch1 && sketch2 && sketch3, "tucker_compress_randomized: null widths or sketch");
  ZBC_CHECK_ARG(lmax >= 2 && lmax <= 64, "lmax must be in [2, 64]");
  for (int i = 0; i < 3 * ncols * q; ++i)
    ZBC_CHECK_ARG(widths_host[i] >= 1, "widths must be >= 1 (entry %d is %d)", i, widths_host[i]);
  const float2* sk[3] = {(const float2*)sketch1, (const float2*)sketch2, (const float2*)sketch3};
  std::vector<int32_t> ranks;
  float2* pool = nullptr;
  int64_t elems = 0;
  zbc_compress_stats stats{};
  const int s = randomized_compress(cols, ld, ncols, g->n1, g->n2, g->n3, q, in_dt, tol, widths_host, sk, lmax, ranks,
                                    &pool, &elems, &stats, stream);
  if (s != ZBC_OK) return s;
  return finish_compress(out, g, q, ncols, ranks, pool, elems, stats, stats_host, stream);
}

extern "C" int tucker_compress(const void* cols, int64_t ld, int ncols, const zbc_grid* g, int q, zbc_dtype in_dt,
                               double tol, zbc_tucker_method method, const zbc_rank_model* model,
                               zbc_dtype store_dt, zbc_handle** out, zbc_compress_stats* stats_host,
                               zbc_stream stream) {
  clear_error();
  ZBC_CHECK_ARG(method == ZBC_HOSVD || method == ZBC_RANDOMIZED_LEARNED || method == ZBC_RANDOMIZED_FIXED,
                "unknown compression method %d", (int)method);
  ZBC_CHECK_ARG(store_dt == ZBC_C64,
                "only complex64 storage is provided (the product kernels compute in FP32 on complex64 tensors)");
  ZBC_TRY(check_compress_args(cols, ld, ncols, g, q, in_dt, tol, out));
  if (method != ZBC_HOSVD) {
    // the randomized range finder with the model's widths (HOSVD fallback per tensor)
    ZBC_CHECK_ARG(model, "the randomized methods need a zbc_rank_model");
    ZBC_CHECK_ARG(model->sketch1 && model->sketch2 && model->sketch3, "zbc_rank_model: null sketch");
    std::vector<int32_t> widths(3 * (size_t)ncols * q);
    if (method == ZBC_RANDOMIZED_FIXED) {
      ZBC_CHECK_ARG(model->fixed_width >= 1, "zbc_rank_model: fixed_width must be >= 1 (got %d)", model->fixed_width);
      std::fill(widths.begin(), widths.end(), model->fixed_width);
    } else {
      ZBC_CHECK_ARG(model->mlp && model->features, "zbc_rank_model: the learned method needs mlp and features");
      ZBC_CHECK_ARG(q == 3, "the rank predictor has outputs for q = 3 components only");
      ZBC_TRY(zbc_rank_widths(model->mlp, model->features, ncols, g, model->oversample, widths.data(), stream));
    }
    return tucker_compress_randomized(cols, ld, ncols, g, q, in_dt, tol, widths.data(), model->sketch1,
                                      model->sketch2, model->sketch3, model->lmax, out, stats_host, stream);
  }
  std::vector<int32_t> ranks;
  float2* pool = nullptr;
  int64_t elems = 0;
  double max_err = 0.0;
  zbc_compress_stats stats{};
  // batch so that the FP64 rotated-unfolding buffer stays near 4 GB
  const int64_t nv = (int64_t)g->n1 * g->n2 * g->n3;
  const int64_t per_col = (int64_t)q * nv * 16;
  int batch = (int)std::max<int64_t>(1, std::min<int64_t>(ncols, ((int64_t)4 << 30) / per_col));
  int s = hosvd_compress(cols, ld, ncols, g->n1, g->n2, g->n3, q, in_dt, tol, ranks, &pool, &elems, &max_err, batch,
                         stream);
  stats.max_rel_err = max_err;
  if (s != ZBC_OK) return s;
  return finish_compress(out, g, q, ncols, ranks, pool, elems, stats, stats_host, stream);
}
