// cross_tucker_compress / cross_tucker_assemble: Tucker compression of columns from a few of
// their fibres (3D cross-Tucker), in FP64 on the GPU.
//
// The paper offers this for tensors too large to assemble whole for the HOSVD (end of Sec. II.B.1
// and Sec. V, citing the linear-time Tucker approximation of Oseledets, Savostyanov and
// Tyrtyshnikov 2008): the factors come from fibres of the tensor only, so the entries evaluated
// and the memory grow linearly with the grid's side.  The steps, per tensor (all tensors of a
// batch advance together, one launch per step):
//   index sets I_g of each mode (I_2, I_3 start as s0 evenly spread indices);
//   a sweep visits g = 1, 2, 3 with a < b the other modes:
//     F_g = the mode-g fibres through I_a x I_b (gather_kernel: entries read from a dense column
//           or evaluated from the Green's function, never the whole column);
//     left singular pairs of F_g by the two-pass Gram / Jacobi scheme of the HOSVD (hosvd.cu);
//     r_g = the smallest r with sum_{i>r} s_i^2 <= ((tol/4)^2/3) ||F_g||_F^2, at most rmax;
//     I_g = the first min(r_g + over, n_g, |I_a||I_b|) rows chosen by greedy pivoting on the
//           leading singular vectors (pivot_kernel: Gaussian elimination, row of largest modulus);
//   after the sweeps the core interpolates the tensor on the cross J_g (first r_g pivots):
//     G = A[J_1, J_2, J_3] x1 M_1^-1 x2 M_2^-1 x3 M_3^-1,  M_g = U_g[J_g, :]
//   (inverse_kernel: Gauss-Jordan with partial pivoting; the mode products reuse the HOSVD's rotate kernel);
//   optional check fibres estimate the model's relative error (check_kernel): each stands for all
//   fibres of its mode, e^2 = mean_c n_a n_b ||fibre error||^2, reported as e / ||G||_F.
#include <cmath>
#include <numeric>

#include "green.cuh"
#include "hosvd.cuh"

namespace zbc {

GreenGeom make_green(const zbc_grid* g, const zbc_segments* s, double freq_hz);  // assemble.cu

constexpr int kXMaxW = 80;    // pivots per mode, at most (rmax 64 + oversampling 16)
constexpr int kXMaxN = 1024;  // mode size, at most

// where tensor t's entries come from: a dense column segment (base) or segment e, row block k
struct XSrc {
  const void* base;
  int e, k;
};

enum { kSrcDense = 0, kSrcGreen3 = 1, kSrcGreen12 = 2 };

template <int KIND, typename T>
__device__ __forceinline__ double2 src_entry(const GreenGeom& G, const XSrc& s, int64_t v) {
  if constexpr (KIND == kSrcDense) {
    return ld_z<T>(s.base, v);
  } else if constexpr (KIND == kSrcGreen3) {
    double2 z[3];
    if (G.op == 0 && G.nq == 1)
      green_entry(G, v, s.e, z);  // the same evaluation as the column assembly
    else
      segment_entry(G, v, s.e, z);
    return s.k == 0 ? z[0] : s.k == 1 ? z[1] : z[2];
  } else {
    double2 z[12];
    pwl_entry(G, v, s.e, z);
    double2 r = z[0];
#pragma unroll
    for (int b = 1; b < 12; ++b)
      if (s.k == b) r = z[b];
    return r;
  }
}

// out[x1 + m1 (x2 + m2 x3)] = A[L1[x1], L2[x2], L3[x3]]  (L_g null: the whole range, m_g = n_g)
struct GatherJob {
  XSrc src;
  const int32_t* L[3];
  int m[3];
  double2* out;
};

template <int KIND, typename T>
__global__ void __launch_bounds__(256) gather_kernel(const GatherJob* jobs, GreenGeom G) {
  const GatherJob jb = jobs[blockIdx.y];
  const int64_t total = (int64_t)jb.m[0] * jb.m[1] * jb.m[2];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int x1 = (int)(e % jb.m[0]);
    const int x2 = (int)((e / jb.m[0]) % jb.m[1]);
    const int x3 = (int)(e / ((int64_t)jb.m[0] * jb.m[1]));
    const int i1 = jb.L[0] ? jb.L[0][x1] : x1;
    const int i2 = jb.L[1] ? jb.L[1][x2] : x2;
    const int i3 = jb.L[2] ? jb.L[2][x3] : x3;
    const int64_t v = i1 + (int64_t)G.n1 * (i2 + (int64_t)G.n2 * i3);
    jb.out[e] = src_entry<KIND, T>(G, jb.src, v);
  }
}

// Greedy pivoting on the first w columns of U (n x w, leading dimension ld): step c takes the
// free row of largest |R[i, c]| (lowest index on ties) and eliminates column c from every row.
// One CTA per job; R (n x w) is the job's workspace.
struct PivJob {
  const double2* U;
  int n, w, ld;
  double2* R;
  int32_t* piv;
};

__device__ __forceinline__ bool better(double ma, int ia, double mb, int ib) {
  return ma > mb || (ma == mb && ia < ib);
}

__global__ void __launch_bounds__(256) pivot_kernel(const PivJob* jobs) {
  const PivJob jb = jobs[blockIdx.x];
  __shared__ unsigned char freerow[kXMaxN];
  __shared__ double2 prow[kXMaxW];
  __shared__ double bm[256];
  __shared__ int bi[256];
  const int n = jb.n, w = jb.w;
  for (int64_t e = threadIdx.x; e < (int64_t)n * w; e += blockDim.x) {
    const int i = (int)(e % n), c = (int)(e / n);
    jb.R[e] = jb.U[i + (int64_t)jb.ld * c];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) freerow[i] = 1;
  __syncthreads();
  for (int c = 0; c < w; ++c) {
    double m = -1.0;
    int mi = n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (!freerow[i]) continue;
      const double2 z = jb.R[i + (int64_t)n * c];
      const double a = hypot(z.x, z.y);
      if (better(a, i, m, mi)) {
        m = a;
        mi = i;
      }
    }
    bm[threadIdx.x] = m;
    bi[threadIdx.x] = mi;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (threadIdx.x < s && better(bm[threadIdx.x + s], bi[threadIdx.x + s], bm[threadIdx.x], bi[threadIdx.x])) {
        bm[threadIdx.x] = bm[threadIdx.x + s];
        bi[threadIdx.x] = bi[threadIdx.x + s];
      }
      __syncthreads();
    }
    const int p = bi[0];
    const double pm = bm[0];
    // p < n: w <= n rows are free at every step
    for (int cc = c + threadIdx.x; cc < w; cc += blockDim.x) prow[cc] = jb.R[p + (int64_t)n * cc];
    if (threadIdx.x == 0) {
      jb.piv[c] = p;
      freerow[p] = 0;
    }
    __syncthreads();
    if (pm > 0.0) {
      const double2 pv = prow[c];
      const double d = pv.x * pv.x + pv.y * pv.y;
      const double2 inv = make_double2(pv.x / d, -pv.y / d);
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 l = zmul(jb.R[i + (int64_t)n * c], inv);
        for (int cc = c; cc < w; ++cc) {
          const double2 r = jb.R[i + (int64_t)n * cc], q = zmul(l, prow[cc]);
          jb.R[i + (int64_t)n * cc] = make_double2(r.x - q.x, r.y - q.y);
        }
      }
    }
    __syncthreads();
  }
}

// V[i + r x] = conj(Minv[x, i]) for M[a, b] = U[J[a] + ld b] (r x r): Gauss-Jordan with partial
// pivoting on [M | I] in the job's workspace (r x 2r).  One CTA per job; a zero pivot (a singular
// M, which the pivoting rules out) sets *bad.
struct InvJob {
  const double2* U;
  int ld, r;
  const int32_t* J;
  double2* work;
  double2* V;
};

__global__ void __launch_bounds__(256) inverse_kernel(const InvJob* jobs, int* bad) {
  const InvJob jb = jobs[blockIdx.x];
  const int r = jb.r;
  double2* A = jb.work;  // A[a + r c], c < 2r
  __shared__ int sp;
  for (int e = threadIdx.x; e < 2 * r * r; e += blockDim.x) {
    const int a = e % r, c = e / r;
    A[e] = c < r ? jb.U[jb.J[a] + (int64_t)jb.ld * c] : make_double2(a == c - r ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int c = 0; c < r; ++c) {
    if (threadIdx.x == 0) {
      int p = c;
      double best = -1.0;
      for (int a = c; a < r; ++a) {
        const double m = hypot(A[a + r * c].x, A[a + r * c].y);
        if (m > best) {
          best = m;
          p = a;
        }
      }
      if (!(best > 0.0)) atomicOr(bad, 1);
      sp = best > 0.0 ? p : -1;
    }
    __syncthreads();
    const int p = sp;
    __syncthreads();      // every thread has read sp before thread 0 writes the next one
    if (p < 0) continue;  // uniform: sp is shared
    if (p != c)
      for (int cc = threadIdx.x; cc < 2 * r; cc += blockDim.x) {
        const double2 t = A[c + r * cc];
        A[c + r * cc] = A[p + r * cc];
        A[p + r * cc] = t;
      }
    __syncthreads();
    const double2 pv = A[c + r * c];
    const double d = pv.x * pv.x + pv.y * pv.y;
    const double2 inv = make_double2(pv.x / d, -pv.y / d);
    __syncthreads();
    for (int cc = threadIdx.x; cc < 2 * r; cc += blockDim.x) A[c + r * cc] = zmul(A[c + r * cc], inv);
    __syncthreads();
    // eliminate column c from the other rows: thread owns (a, cc) pairs with cc > c or the
    // identity half; the multiplier A[a, c] is read before column c itself is cleared
    for (int e = threadIdx.x; e < r * 2 * r; e += blockDim.x) {
      const int a = e % r, cc = e / r;
      if (a == c || cc == c) continue;
      const double2 f = A[a + r * c], q = zmul(f, A[c + r * cc]);
      A[a + r * cc] = make_double2(A[a + r * cc].x - q.x, A[a + r * cc].y - q.y);
    }
    __syncthreads();
    for (int a = threadIdx.x; a < r; a += blockDim.x)
      if (a != c) A[a + r * c] = make_double2(0.0, 0.0);
    __syncthreads();
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, x = e / r;
    const double2 m = A[x + r * (r + i)];  // Minv[x, i]
    jb.V[i + r * x] = make_double2(m.x, -m.y);
  }
}

// One check fibre of one tensor: the mode-g fibre through (ia, ib) of the model
// G x1 U1 x2 U2 x3 U3 against the tensor's entries; out[0] = sum |A - model|^2, out[1] = sum |A|^2.
struct ChkJob {
  XSrc src;
  const double2* G;      // r1 x r2 x r3
  const double2* U[3];   // n_g x (>= r_g), leading dimension n_g
  int r[3];
  int g, ia, ib;
  double* out;
};

template <int KIND, typename T>
__global__ void __launch_bounds__(256) check_kernel(const ChkJob* jobs, GreenGeom G) {
  const ChkJob jb = jobs[blockIdx.x];
  const int n[3] = {G.n1, G.n2, G.n3};
  const int g = jb.g, a = g == 0 ? 1 : 0, b = g == 2 ? 1 : 2;
  __shared__ double2 tv[64];
  __shared__ double r0[256], r1[256];
  // tv[x] = sum_{y, z} G[.., x, ..] U_a[ia, y] U_b[ib, z]  (x along mode g)
  const int r1s = jb.r[0], r2s = jb.r[1];
  for (int x = threadIdx.x; x < jb.r[g]; x += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int z = 0; z < jb.r[b]; ++z) {
      const double2 ub = jb.U[b][jb.ib + (int64_t)n[b] * z];
      for (int y = 0; y < jb.r[a]; ++y) {
        int idx[3];
        idx[g] = x;
        idx[a] = y;
        idx[b] = z;
        const double2 gv = jb.G[idx[0] + r1s * (idx[1] + r2s * idx[2])];
        acc = zfma(zmul(gv, jb.U[a][jb.ia + (int64_t)n[a] * y]), ub, acc);
      }
    }
    tv[x] = acc;
  }
  __syncthreads();
  double s0 = 0.0, s1 = 0.0;
  for (int i = threadIdx.x; i < n[g]; i += blockDim.x) {
    double2 m = make_double2(0.0, 0.0);
    for (int x = 0; x < jb.r[g]; ++x) m = zfma(jb.U[g][i + (int64_t)n[g] * x], tv[x], m);
    int id[3];
    id[g] = i;
    id[a] = jb.ia;
    id[b] = jb.ib;
    const int64_t v = id[0] + (int64_t)G.n1 * (id[1] + (int64_t)G.n2 * id[2]);
    const double2 ref = src_entry<KIND, T>(G, jb.src, v);
    const double dx = ref.x - m.x, dy = ref.y - m.y;
    s0 += dx * dx + dy * dy;
    s1 += ref.x * ref.x + ref.y * ref.y;
  }
  r0[threadIdx.x] = s0;
  r1[threadIdx.x] = s1;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      r0[threadIdx.x] += r0[threadIdx.x + s];
      r1[threadIdx.x] += r1[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    jb.out[0] = r0[0];
    jb.out[1] = r1[0];
  }
}

// eigenvalues on the diagonals of the Jacobi output: lam[t*ld + i] = H_t[i + n i].x
__global__ void __launch_bounds__(256) diag_kernel(const JacJob* jobs, double* lam, int ld) {
  const JacJob jb = jobs[blockIdx.x];
  for (int i = threadIdx.x; i < jb.n; i += blockDim.x) lam[(int64_t)blockIdx.x * ld + i] = jb.H[i + (int64_t)jb.n * i].x;
}

}  // namespace zbc

// ---------------------------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------------------------
namespace zbc {

struct CrossParams {
  int sweeps, s0, over, rmax;
};

struct CrossWork {
  DevBuf jobs_a, jobs_b, jobs_c, idx, F, B, H, V1, W, U[3], lam, ord, piv, R, C, C1, C2, G, Vinv, inv_work, chk,
      bad;
};

// s indices spread evenly over [0, n): floor((2l + 1) n / (2 s))
static std::vector<int32_t> spread_indices(int n, int s) {
  s = std::min(s, n);
  std::vector<int32_t> v(s);
  for (int l = 0; l < s; ++l) v[l] = (int32_t)(((int64_t)(2 * l + 1) * n) / (2 * s));
  return v;
}

static inline int other_a(int g) { return g == 0 ? 1 : 0; }
static inline int other_b(int g) { return g == 2 ? 1 : 2; }

// unfolding of mode g of a gathered tensor of sizes ms (layout x1 + ms0 (x2 + ms1 x3)); column c
// of mode g is (x_a, x_b) with x_a = c mod ms_a
static Unf gathered_unf(int g, const int* ms) {
  if (g == 0) return Unf{1, (int64_t)ms[1] * ms[2], ms[0], 0};
  if (g == 1) return Unf{ms[0], ms[0], 1, (int64_t)ms[0] * ms[1]};
  return Unf{(int64_t)ms[0] * ms[1], (int64_t)ms[0] * ms[1], 1, 0};
}

template <int KIND, typename T>
static int launch_gather(CrossWork& w, const std::vector<GatherJob>& jobs, int64_t max_elems, const GreenGeom& G,
                         cudaStream_t st) {
  ZBC_TRY(upload_jobs(w.jobs_c, jobs, st));
  const int bx = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(max_elems, 256), 4096));
  gather_kernel<KIND, T><<<dim3(bx, (unsigned)jobs.size()), 256, 0, st>>>((const GatherJob*)w.jobs_c.ptr, G);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

// Compress the tensors src[0..NT) (tensor t = column t/q, row block t%q).  Appends 3 ranks per
// tensor and writes the batch's packed complex64 pool to *pool_out (allocated here).
template <int KIND, typename T>
static int cross_batch(const std::vector<XSrc>& src, const GreenGeom& Gg, double tol, const CrossParams& P,
                       const std::vector<int32_t>& checks, CrossWork& w, std::vector<int32_t>& ranks_out,
                       float2** pool_out, int64_t* elems_out, double* max_chk, int64_t* entries, cudaStream_t st) {
  const int NT = (int)src.size();
  const int n[3] = {Gg.n1, Gg.n2, Gg.n3};
  const int nmax = std::max(n[0], std::max(n[1], n[2]));
  int Wg[3];
  for (int g = 0; g < 3; ++g) Wg[g] = std::min(P.rmax + P.over, n[g]);
  const size_t mat = (size_t)nmax * nmax;
  std::vector<std::vector<int32_t>> I[3];
  for (int g = 0; g < 3; ++g) I[g].assign(NT, spread_indices(n[g], P.s0));
  std::vector<int> rk(3 * (size_t)NT, 0), wk(3 * (size_t)NT, 0);

  for (int g = 0; g < 3; ++g) ZBC_TRY(w.U[g].ensure(sizeof(double2) * (size_t)n[g] * Wg[g] * NT));
  ZBC_TRY(w.H.ensure(sizeof(double2) * mat * NT));
  ZBC_TRY(w.V1.ensure(sizeof(double2) * mat * NT));
  ZBC_TRY(w.W.ensure(sizeof(double2) * mat * NT));
  ZBC_TRY(w.lam.ensure(sizeof(double) * (size_t)nmax * NT));
  ZBC_TRY(w.ord.ensure(sizeof(int) * (size_t)nmax * NT));
  ZBC_TRY(w.piv.ensure(sizeof(int32_t) * (size_t)kXMaxW * NT));
  ZBC_TRY(w.R.ensure(sizeof(double2) * (size_t)nmax * kXMaxW * NT));
  double2* Hb = (double2*)w.H.ptr;
  double2* V1b = (double2*)w.V1.ptr;
  double2* Wb = (double2*)w.W.ptr;
  auto Ut = [&](int g, int t) { return (double2*)w.U[g].ptr + (size_t)n[g] * Wg[g] * t; };

  for (int sweep = 0; sweep < P.sweeps; ++sweep) {
    for (int g = 0; g < 3; ++g) {
      const int a = other_a(g), b = other_b(g), ng = n[g];
      // index lists and fibre tensors
      std::vector<int32_t> hidx;
      std::vector<int64_t> offa(NT), offb(NT), foff(NT), fcnt(NT);
      int64_t ftot = 0, fmax = 0;
      for (int t = 0; t < NT; ++t) {
        offa[t] = (int64_t)hidx.size();
        hidx.insert(hidx.end(), I[a][t].begin(), I[a][t].end());
        offb[t] = (int64_t)hidx.size();
        hidx.insert(hidx.end(), I[b][t].begin(), I[b][t].end());
        fcnt[t] = (int64_t)I[a][t].size() * I[b][t].size();
        foff[t] = ftot;
        ftot += ng * fcnt[t];
        fmax = std::max(fmax, fcnt[t]);
      }
      ZBC_TRY(w.idx.ensure(sizeof(int32_t) * hidx.size()));
      ZBC_TRY_CUDA(cudaMemcpyAsync(w.idx.ptr, hidx.data(), sizeof(int32_t) * hidx.size(), cudaMemcpyHostToDevice, st));
      ZBC_TRY(w.F.ensure(sizeof(double2) * ftot));
      ZBC_TRY(w.B.ensure(sizeof(double2) * ftot));
      double2* Fb = (double2*)w.F.ptr;
      double2* Bb = (double2*)w.B.ptr;
      const int32_t* didx = (const int32_t*)w.idx.ptr;
      std::vector<GatherJob> gj(NT);
      std::vector<Unf> unf(NT);
      for (int t = 0; t < NT; ++t) {
        GatherJob j{};
        j.src = src[t];
        j.L[g] = nullptr;
        j.m[g] = ng;
        j.L[a] = didx + offa[t];
        j.m[a] = (int)I[a][t].size();
        j.L[b] = didx + offb[t];
        j.m[b] = (int)I[b][t].size();
        j.out = Fb + foff[t];
        gj[t] = j;
        unf[t] = gathered_unf(g, j.m);
      }
      ZBC_TRY((launch_gather<KIND, T>(w, gj, ng * fmax, Gg, st)));
      *entries += ftot;
      // left singular pairs of F: Gram, Jacobi, B = V1^H F, Gram of B, Jacobi (hosvd.cu)
      std::vector<GramJob> gr(NT);
      for (int t = 0; t < NT; ++t) gr[t] = GramJob{Fb + foff[t], unf[t], fcnt[t], ng, Hb + mat * t};
      ZBC_TRY(upload_jobs(w.jobs_a, gr, st));
      const dim3 gg(ceil_div(ng, 32), ceil_div(ng, 32), NT);
      launch_gram_f64((const GramJob*)w.jobs_a.ptr, gg, st);
      ZBC_TRY_CUDA(cudaGetLastError());
      std::vector<JacJob> jj(NT);
      for (int t = 0; t < NT; ++t) jj[t] = JacJob{Hb + mat * t, V1b + mat * t, ng};
      ZBC_TRY(upload_jobs(w.jobs_b, jj, st));
      jacobi_kernel<<<NT, 512, jacobi_smem(ng), st>>>((const JacJob*)w.jobs_b.ptr, 60, nullptr);
      ZBC_TRY_CUDA(cudaGetLastError());
      std::vector<RotJob> rj(NT);
      for (int t = 0; t < NT; ++t)
        rj[t] = RotJob{Fb + foff[t], unf[t], fcnt[t], ng, ng, ng, V1b + mat * t, Bb + foff[t], Unf{1, fcnt[t], ng, 0}};
      ZBC_TRY(upload_jobs(w.jobs_c, rj, st));
      launch_rotate_f64((const RotJob*)w.jobs_c.ptr, dim3(ceil_div(fmax, 64), ceil_div(ng, 32), NT), st);
      ZBC_TRY_CUDA(cudaGetLastError());
      for (int t = 0; t < NT; ++t) gr[t] = GramJob{Bb + foff[t], Unf{1, fcnt[t], ng, 0}, fcnt[t], ng, Hb + mat * t};
      ZBC_TRY(upload_jobs(w.jobs_a, gr, st));
      launch_gram_f64((const GramJob*)w.jobs_a.ptr, gg, st);
      ZBC_TRY_CUDA(cudaGetLastError());
      for (int t = 0; t < NT; ++t) jj[t] = JacJob{Hb + mat * t, Wb + mat * t, ng};
      ZBC_TRY(upload_jobs(w.jobs_b, jj, st));
      jacobi_kernel<<<NT, 512, jacobi_smem(ng), st>>>((const JacJob*)w.jobs_b.ptr, 60, nullptr);
      ZBC_TRY_CUDA(cudaGetLastError());
      diag_kernel<<<NT, 256, 0, st>>>((const JacJob*)w.jobs_b.ptr, (double*)w.lam.ptr, nmax);
      ZBC_TRY_CUDA(cudaGetLastError());
      count_launch(6);
      std::vector<double> lam((size_t)nmax * NT);
      ZBC_TRY_CUDA(cudaMemcpyAsync(lam.data(), w.lam.ptr, sizeof(double) * lam.size(), cudaMemcpyDeviceToHost, st));
      ZBC_TRY_CUDA(cudaStreamSynchronize(st));
      // ranks (the HOSVD rule on the fibres at tol / 4) and the pivot counts
      std::vector<int> ord_all((size_t)NT * ng);
      for (int t = 0; t < NT; ++t) {
        std::vector<int> ord(ng);
        std::iota(ord.begin(), ord.end(), 0);
        const double* l = lam.data() + (size_t)nmax * t;
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return l[x] > l[y]; });
        std::vector<double> ls(ng);
        double norm2 = 0.0;
        for (int i = 0; i < ng; ++i) {
          ls[i] = l[ord[i]];
          norm2 += std::max(ls[i], 0.0);
        }
        const double tq = 0.25 * tol;
        int r = truncation_rank(ls, tq * tq / 3.0 * norm2);
        r = (int)std::min<int64_t>(std::min(r, std::min(P.rmax, ng)), fcnt[t]);
        const int wv = (int)std::min<int64_t>(std::min(r + P.over, ng), fcnt[t]);
        rk[3 * t + g] = r;
        wk[3 * t + g] = wv;
        for (int i = 0; i < ng; ++i) ord_all[(size_t)t * ng + i] = ord[i];
      }
      ZBC_TRY_CUDA(cudaMemcpyAsync(w.ord.ptr, ord_all.data(), sizeof(int) * ord_all.size(), cudaMemcpyHostToDevice, st));
      std::vector<FacJob> fj(NT);
      for (int t = 0; t < NT; ++t)
        fj[t] = FacJob{V1b + mat * t, Wb + mat * t, (const int*)w.ord.ptr + (size_t)t * ng, ng, wk[3 * t + g], Ut(g, t)};
      ZBC_TRY(upload_jobs(w.jobs_a, fj, st));
      factor_kernel<<<dim3(ceil_div((int64_t)ng * Wg[g], 256), NT), 256, 0, st>>>((const FacJob*)w.jobs_a.ptr);
      ZBC_TRY_CUDA(cudaGetLastError());
      std::vector<PivJob> pj(NT);
      for (int t = 0; t < NT; ++t)
        pj[t] = PivJob{Ut(g, t), ng, wk[3 * t + g], ng, (double2*)w.R.ptr + (size_t)nmax * kXMaxW * t,
                       (int32_t*)w.piv.ptr + (size_t)kXMaxW * t};
      ZBC_TRY(upload_jobs(w.jobs_b, pj, st));
      pivot_kernel<<<NT, 256, 0, st>>>((const PivJob*)w.jobs_b.ptr);
      ZBC_TRY_CUDA(cudaGetLastError());
      count_launch(2);
      std::vector<int32_t> piv((size_t)kXMaxW * NT);
      ZBC_TRY_CUDA(cudaMemcpyAsync(piv.data(), w.piv.ptr, sizeof(int32_t) * piv.size(), cudaMemcpyDeviceToHost, st));
      ZBC_TRY_CUDA(cudaStreamSynchronize(st));
      for (int t = 0; t < NT; ++t)
        I[g][t].assign(piv.begin() + (size_t)kXMaxW * t, piv.begin() + (size_t)kXMaxW * t + wk[3 * t + g]);
    }
  }

  // the core: entries on the cross J_1 x J_2 x J_3, then x_g M_g^-1
  std::vector<int32_t> hidx;
  std::vector<int64_t> joff(3 * (size_t)NT), coff(NT), voff(3 * (size_t)NT);
  int64_t ctot = 0, vtot = 0, cmax = 0;
  int rmx[3] = {0, 0, 0};
  for (int t = 0; t < NT; ++t) {
    for (int g = 0; g < 3; ++g) {
      const int r = rk[3 * t + g];
      joff[3 * t + g] = (int64_t)hidx.size();
      hidx.insert(hidx.end(), I[g][t].begin(), I[g][t].begin() + r);
      voff[3 * t + g] = vtot;
      vtot += (int64_t)r * r;
      rmx[g] = std::max(rmx[g], r);
    }
    const int64_t cs = (int64_t)rk[3 * t] * rk[3 * t + 1] * rk[3 * t + 2];
    coff[t] = ctot;
    ctot += cs;
    cmax = std::max(cmax, cs);
  }
  ZBC_TRY(w.idx.ensure(sizeof(int32_t) * hidx.size()));
  ZBC_TRY_CUDA(cudaMemcpyAsync(w.idx.ptr, hidx.data(), sizeof(int32_t) * hidx.size(), cudaMemcpyHostToDevice, st));
  ZBC_TRY(w.C.ensure(sizeof(double2) * ctot));
  ZBC_TRY(w.C1.ensure(sizeof(double2) * ctot));
  ZBC_TRY(w.C2.ensure(sizeof(double2) * ctot));
  ZBC_TRY(w.G.ensure(sizeof(double2) * ctot));
  ZBC_TRY(w.Vinv.ensure(sizeof(double2) * vtot));
  ZBC_TRY(w.inv_work.ensure(sizeof(double2) * 2 * vtot));
  ZBC_TRY(w.bad.ensure(sizeof(int)));
  ZBC_TRY_CUDA(cudaMemsetAsync(w.bad.ptr, 0, sizeof(int), st));
  const int32_t* didx = (const int32_t*)w.idx.ptr;
  double2* Cb = (double2*)w.C.ptr;
  double2* C1 = (double2*)w.C1.ptr;
  double2* C2 = (double2*)w.C2.ptr;
  double2* Gc = (double2*)w.G.ptr;
  double2* Vb = (double2*)w.Vinv.ptr;
  {
    std::vector<GatherJob> gj(NT);
    for (int t = 0; t < NT; ++t) {
      GatherJob j{};
      j.src = src[t];
      for (int g = 0; g < 3; ++g) {
        j.L[g] = didx + joff[3 * t + g];
        j.m[g] = rk[3 * t + g];
      }
      j.out = Cb + coff[t];
      gj[t] = j;
    }
    ZBC_TRY((launch_gather<KIND, T>(w, gj, cmax, Gg, st)));
    *entries += ctot;
  }
  {
    std::vector<InvJob> ij(3 * (size_t)NT);
    for (int t = 0; t < NT; ++t)
      for (int g = 0; g < 3; ++g)
        ij[3 * t + g] = InvJob{Ut(g, t), n[g], rk[3 * t + g], didx + joff[3 * t + g],
                               (double2*)w.inv_work.ptr + 2 * voff[3 * t + g], Vb + voff[3 * t + g]};
    ZBC_TRY(upload_jobs(w.jobs_a, ij, st));
    inverse_kernel<<<3 * NT, 256, 0, st>>>((const InvJob*)w.jobs_a.ptr, (int*)w.bad.ptr);
    ZBC_TRY_CUDA(cudaGetLastError());
  }
  {
    // G = C x1 M1^-1 x2 M2^-1 x3 M3^-1 with the rotate kernel: out(x, c) = sum_i conj(V[i + r x]) A(i, c)
    std::vector<RotJob> r1j(NT), r2j(NT), r3j(NT);
    int64_t c1max = 0, c2max = 0, c3max = 0;
    for (int t = 0; t < NT; ++t) {
      const int r1 = rk[3 * t], r2 = rk[3 * t + 1], r3 = rk[3 * t + 2];
      const Unf u1{1, (int64_t)r2 * r3, r1, 0}, u2{r1, r1, 1, (int64_t)r1 * r2}, u3{(int64_t)r1 * r2, (int64_t)r1 * r2, 1, 0};
      r1j[t] = RotJob{Cb + coff[t], u1, (int64_t)r2 * r3, r1, r1, r1, Vb + voff[3 * t], C1 + coff[t], u1};
      r2j[t] = RotJob{C1 + coff[t], u2, (int64_t)r1 * r3, r2, r2, r2, Vb + voff[3 * t + 1], C2 + coff[t], u2};
      r3j[t] = RotJob{C2 + coff[t], u3, (int64_t)r1 * r2, r3, r3, r3, Vb + voff[3 * t + 2], Gc + coff[t], u3};
      c1max = std::max<int64_t>(c1max, (int64_t)r2 * r3);
      c2max = std::max<int64_t>(c2max, (int64_t)r1 * r3);
      c3max = std::max<int64_t>(c3max, (int64_t)r1 * r2);
    }
    ZBC_TRY(upload_jobs(w.jobs_b, r1j, st));
    launch_rotate_f64((const RotJob*)w.jobs_b.ptr, dim3(ceil_div(c1max, 64), ceil_div(rmx[0], 32), NT), st);
    ZBC_TRY_CUDA(cudaGetLastError());
    ZBC_TRY(upload_jobs(w.jobs_c, r2j, st));
    launch_rotate_f64((const RotJob*)w.jobs_c.ptr, dim3(ceil_div(c2max, 64), ceil_div(rmx[1], 32), NT), st);
    ZBC_TRY_CUDA(cudaGetLastError());
    ZBC_TRY(upload_jobs(w.jobs_a, r3j, st));
    launch_rotate_f64((const RotJob*)w.jobs_a.ptr, dim3(ceil_div(c3max, 64), ceil_div(rmx[2], 32), NT), st);
    ZBC_TRY_CUDA(cudaGetLastError());
    count_launch(4);
    int bad = 0;
    ZBC_TRY_CUDA(cudaMemcpyAsync(&bad, w.bad.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    ZBC_TRY_CUDA(cudaStreamSynchronize(st));  // the job buffers are reused below
    if (bad) {
      set_error("cross_tucker: singular cross submatrix (a factor lost rank)");
      return ZBC_ENAN;
    }
  }

  // check fibres: relative error of the model on them, per tensor
  const int nchk = (int)checks.size() / 3;
  if (nchk > 0) {
    std::vector<ChkJob> cj((size_t)NT * nchk);
    ZBC_TRY(w.chk.ensure(sizeof(double) * 2 * cj.size()));
    for (int t = 0; t < NT; ++t)
      for (int c = 0; c < nchk; ++c) {
        ChkJob j{};
        j.src = src[t];
        j.G = Gc + coff[t];
        for (int g = 0; g < 3; ++g) {
          j.U[g] = Ut(g, t);
          j.r[g] = rk[3 * t + g];
        }
        j.g = checks[3 * c];
        j.ia = checks[3 * c + 1];
        j.ib = checks[3 * c + 2];
        j.out = (double*)w.chk.ptr + 2 * ((size_t)t * nchk + c);
        cj[(size_t)t * nchk + c] = j;
        *entries += n[j.g];
      }
    ZBC_TRY(upload_jobs(w.jobs_b, cj, st));
    check_kernel<KIND, T><<<(unsigned)cj.size(), 256, 0, st>>>((const ChkJob*)w.jobs_b.ptr, Gg);
    ZBC_TRY_CUDA(cudaGetLastError());
    count_launch();
    std::vector<double> part(2 * cj.size());
    std::vector<double2> gh(ctot);
    ZBC_TRY_CUDA(cudaMemcpyAsync(part.data(), w.chk.ptr, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st));
    ZBC_TRY_CUDA(cudaMemcpyAsync(gh.data(), Gc, sizeof(double2) * ctot, cudaMemcpyDeviceToHost, st));
    ZBC_TRY_CUDA(cudaStreamSynchronize(st));
    // a uniformly drawn mode-g fibre stands for all n_a n_b of them:
    //   e^2 = (1/#checks) sum_c n_a n_b ||fibre error||^2 estimates ||A - model||_F^2,
    // relative to ||G||_F = ||model||_F (orthonormal factors)
    for (int t = 0; t < NT; ++t) {
      double num = 0.0, gn = 0.0;
      for (int c = 0; c < nchk; ++c) {
        const int gm = checks[3 * c];
        num += (double)n[other_a(gm)] * n[other_b(gm)] * part[2 * ((size_t)t * nchk + c)];
      }
      num /= nchk;
      const int64_t cs = (int64_t)rk[3 * t] * rk[3 * t + 1] * rk[3 * t + 2];
      for (int64_t i = 0; i < cs; ++i) gn += gh[coff[t] + i].x * gh[coff[t] + i].x + gh[coff[t] + i].y * gh[coff[t] + i].y;
      const double e = gn > 0.0 ? std::sqrt(num / gn) : (num == 0.0 ? 0.0 : INFINITY);
      *max_chk = std::max(*max_chk, e);
    }
  }

  // pack: core, U1, U2, U3 per tensor, complex64
  int64_t elems = 0;
  std::vector<int64_t> toff(NT);
  for (int t = 0; t < NT; ++t) {
    toff[t] = elems;
    elems += (int64_t)rk[3 * t] * rk[3 * t + 1] * rk[3 * t + 2];
    for (int g = 0; g < 3; ++g) elems += (int64_t)n[g] * rk[3 * t + g];
  }
  float2* pool = nullptr;
  ZBC_TRY_CUDA(cudaMalloc(&pool, sizeof(float2) * std::max<int64_t>(1, elems)));
  std::vector<CopyJob> pk;
  for (int t = 0; t < NT; ++t) {
    int64_t o = toff[t];
    const int64_t cs = (int64_t)rk[3 * t] * rk[3 * t + 1] * rk[3 * t + 2];
    pk.push_back(CopyJob{Gc + coff[t], pool + o, cs});
    o += cs;
    for (int g = 0; g < 3; ++g) {
      pk.push_back(CopyJob{Ut(g, t), pool + o, (int64_t)n[g] * rk[3 * t + g]});
      o += (int64_t)n[g] * rk[3 * t + g];
    }
  }
  int s_up = upload_jobs(w.jobs_c, pk, st);
  cudaError_t e = cudaSuccess;
  if (s_up == ZBC_OK) {
    pack_kernel<<<dim3(16, (unsigned)pk.size()), 256, 0, st>>>((const CopyJob*)w.jobs_c.ptr);
    count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (s_up != ZBC_OK || e != cudaSuccess) {
    cudaFree(pool);
    if (s_up != ZBC_OK) return s_up;
    set_error("cross_tucker pack failed: %s", cudaGetErrorString(e));
    return ZBC_ECUDA;
  }
  for (int t = 0; t < NT; ++t)
    for (int g = 0; g < 3; ++g) ranks_out.push_back(rk[3 * t + g]);
  *pool_out = pool;
  *elems_out = elems;
  return ZBC_OK;
}

}  // namespace zbc

using namespace zbc;

static int cross_params(const zbc_cross_params* p, CrossParams& P) {
  P = CrossParams{2, 8, 4, 64};
  if (p) {
    if (p->sweeps) P.sweeps = p->sweeps;
    if (p->s0) P.s0 = p->s0;
    P.over = p->over;
    if (p->rmax) P.rmax = p->rmax;
  }
  ZBC_CHECK_ARG(P.sweeps >= 1 && P.sweeps <= 16, "sweeps must be in [1, 16]");
  ZBC_CHECK_ARG(P.s0 >= 1 && P.s0 <= 64, "s0 must be in [1, 64]");
  ZBC_CHECK_ARG(P.over >= 0 && P.over <= 16, "over must be in [0, 16]");
  ZBC_CHECK_ARG(P.rmax >= 1 && P.rmax <= 64, "rmax must be in [1, 64]");
  return ZBC_OK;
}

static int cross_checks(const zbc_grid* g, const int32_t* checks_host, int nchecks, std::vector<int32_t>& out) {
  ZBC_CHECK_ARG(nchecks >= 0 && nchecks <= 4096, "nchecks must be in [0, 4096]");
  ZBC_CHECK_ARG(nchecks == 0 || checks_host, "checks_host is null");
  const int n[3] = {g->n1, g->n2, g->n3};
  out.assign(checks_host, checks_host + 3 * (size_t)nchecks);
  for (int c = 0; c < nchecks; ++c) {
    const int gm = out[3 * c];
    ZBC_CHECK_ARG(gm >= 0 && gm <= 2, "check %d: mode %d not in [0, 2]", c, gm);
    const int a = other_a(gm), b = other_b(gm);
    ZBC_CHECK_ARG(out[3 * c + 1] >= 0 && out[3 * c + 1] < n[a] && out[3 * c + 2] >= 0 && out[3 * c + 2] < n[b],
                  "check %d: fibre index out of range", c);
  }
  return ZBC_OK;
}

// columns per batch: tensors <= 16383 (pack grid) and a worst-case workspace near 16 GB
static int cross_batch_cols(const zbc_grid* g, int q, const CrossParams& P) {
  const int64_t nmax = std::max(g->n1, std::max(g->n2, g->n3));
  const int64_t W = std::min<int64_t>(P.rmax + P.over, nmax);
  const int64_t per_tensor =
      16 * (3 * nmax * nmax + 2 * nmax * W * W + (int64_t)(g->n1 + g->n2 + g->n3) * W + nmax * kXMaxW) + 64;
  const int64_t by_mem = std::max<int64_t>(1, ((int64_t)16 << 30) / per_tensor);
  return (int)std::max<int64_t>(1, std::min<int64_t>(by_mem, 16383) / q);
}

template <int KIND, typename T>
static int cross_run(const std::vector<XSrc>& src_all, int ncols, int q, const GreenGeom& G, double tol,
                     const CrossParams& P, const std::vector<int32_t>& checks, const zbc_grid* g, zbc_handle** out,
                     zbc_compress_stats* stats_host, zbc_cross_stats* xstats_host, cudaStream_t st) {
  CrossWork w;
  std::vector<int32_t> ranks;
  std::vector<float2*> pools;
  std::vector<int64_t> sizes;
  double max_chk = 0.0;
  int64_t entries = 0;
  int status = ZBC_OK;
  const int bc = cross_batch_cols(g, q, P);
  for (int c0 = 0; c0 < ncols && status == ZBC_OK; c0 += bc) {
    const int nc = std::min(bc, ncols - c0);
    std::vector<XSrc> src(src_all.begin() + (size_t)c0 * q, src_all.begin() + (size_t)(c0 + nc) * q);
    float2* p = nullptr;
    int64_t e = 0;
    status = cross_batch<KIND, T>(src, G, tol, P, checks, w, ranks, &p, &e, &max_chk, &entries, st);
    if (status == ZBC_OK) {
      pools.push_back(p);
      sizes.push_back(e);
    }
  }
  float2* all = nullptr;
  int64_t total = 0;
  for (auto s : sizes) total += s;
  if (status == ZBC_OK) {
    if (cudaMalloc(&all, sizeof(float2) * std::max<int64_t>(1, total)) != cudaSuccess) {
      set_error("cudaMalloc pool failed");
      status = ZBC_ENOMEM;
    } else {
      int64_t o = 0;
      for (size_t i = 0; i < pools.size() && status == ZBC_OK; ++i) {
        if (cudaMemcpyAsync(all + o, pools[i], sizeof(float2) * sizes[i], cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
          set_error("pool copy failed");
          status = ZBC_ECUDA;
        }
        o += sizes[i];
      }
      if (status == ZBC_OK && cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("pool copy failed");
        status = ZBC_ECUDA;
      }
    }
  }
  for (auto p : pools) cudaFree(p);
  if (status != ZBC_OK) {
    if (all) cudaFree(all);
    return status;
  }
  zbc_compress_stats stats{};
  stats.max_rel_err = checks.empty() ? -1.0 : max_chk;
  if (xstats_host) {
    xstats_host->entries = entries;
    xstats_host->max_check_err = checks.empty() ? -1.0 : max_chk;
  }
  return finish_compress(out, g, q, ncols, ranks, all, total, stats, stats_host, st);
}

extern "C" int cross_tucker_compress(const void* cols, int64_t ld, int ncols, const zbc_grid* g, int q,
                                     zbc_dtype in_dt, double tol, const zbc_cross_params* params,
                                     const int32_t* checks_host, int nchecks, zbc_handle** out,
                                     zbc_compress_stats* stats_host, zbc_cross_stats* xstats_host, zbc_stream stream) {
  clear_error();
  ZBC_TRY(check_compress_args(cols, ld, ncols, g, q, in_dt, tol, out));
  CrossParams P;
  ZBC_TRY(cross_params(params, P));
  std::vector<int32_t> checks;
  ZBC_TRY(cross_checks(g, checks_host, nchecks, checks));
  const int64_t nv = (int64_t)g->n1 * g->n2 * g->n3;
  const size_t eb = in_dt == ZBC_C128 ? 16 : 8;
  std::vector<XSrc> src((size_t)ncols * q);
  for (int j = 0; j < ncols; ++j)
    for (int k = 0; k < q; ++k) src[(size_t)j * q + k] = XSrc{(const char*)cols + ((int64_t)j * ld + k * nv) * eb, 0, 0};
  GreenGeom G{};
  G.n1 = g->n1;
  G.n2 = g->n2;
  G.n3 = g->n3;
  if (in_dt == ZBC_C128)
    return cross_run<kSrcDense, double2>(src, ncols, q, G, tol, P, checks, g, out, stats_host, xstats_host, stream);
  return cross_run<kSrcDense, float2>(src, ncols, q, G, tol, P, checks, g, out, stats_host, xstats_host, stream);
}

extern "C" int cross_tucker_assemble(const zbc_grid* g, const zbc_segments* s, double freq_hz,
                                     const int32_t* cols_host, int ncols, int q, zbc_operator op, int nq, double tol,
                                     const zbc_cross_params* params, const int32_t* checks_host, int nchecks,
                                     zbc_handle** out, zbc_compress_stats* stats_host, zbc_cross_stats* xstats_host,
                                     zbc_stream stream) {
  clear_error();
  ZBC_CHECK_ARG(g && s && cols_host && out, "cross_tucker_assemble: null argument");
  ZBC_CHECK_ARG(op == ZBC_OP_N || op == ZBC_OP_K, "unknown operator %d", (int)op);
  ZBC_CHECK_ARG(nq >= 1 && nq <= kMaxQuad, "nq must be in [1, %d]", kMaxQuad);
  ZBC_CHECK_ARG(q == 3 || q == 12, "q must be 3 (piecewise-constant) or 12 (piecewise-linear)");
  ZBC_CHECK_ARG(g->n1 >= 2 && g->n2 >= 2 && g->n3 >= 2 && g->n1 <= 1024 && g->n2 <= 1024 && g->n3 <= 1024,
                "grid sizes must be in [2, 1024]");
  ZBC_CHECK_ARG(g->n1 % 2 == 0 && g->n2 % 2 == 0 && g->n3 % 2 == 0, "grid sizes must be even");
  ZBC_CHECK_ARG(g->h > 0, "bad grid");
  ZBC_CHECK_ARG(s->m >= 1 && s->centre && s->tangent && s->length, "bad segments");
  ZBC_CHECK_ARG(ncols >= 1, "ncols must be >= 1");
  ZBC_CHECK_ARG(tol > 0 && tol < 1, "tol must be in (0, 1)");
  ZBC_CHECK_ARG(freq_hz > 0 && std::isfinite(freq_hz), "freq_hz must be positive");
  for (int j = 0; j < ncols; ++j)
    ZBC_CHECK_ARG(cols_host[j] >= 0 && cols_host[j] < s->m, "cols_host[%d] = %d not in [0, m)", j, cols_host[j]);
  if (*out) {
    const Handle& h0 = (*out)->h;
    ZBC_CHECK_ARG(h0.n1 == g->n1 && h0.n2 == g->n2 && h0.n3 == g->n3 && h0.q == q && !h0.has_v,
                  "append: grid/q mismatch or handle holds ACA storage");
  }
  CrossParams P;
  ZBC_TRY(cross_params(params, P));
  std::vector<int32_t> checks;
  ZBC_TRY(cross_checks(g, checks_host, nchecks, checks));
  GreenGeom G = make_green(g, s, freq_hz);
  G.op = op == ZBC_OP_K ? 1 : 0;
  G.nq = nq;
  gauss_legendre(nq, G.qx, G.qw);
  std::vector<XSrc> src((size_t)ncols * q);
  for (int j = 0; j < ncols; ++j)
    for (int k = 0; k < q; ++k) src[(size_t)j * q + k] = XSrc{nullptr, cols_host[j], k};
  if (q == 12)
    return cross_run<kSrcGreen12, double2>(src, ncols, q, G, tol, P, checks, g, out, stats_host, xstats_host, stream);
  return cross_run<kSrcGreen3, double2>(src, ncols, q, G, tol, P, checks, g, out, stats_host, xstats_host, stream);
}
