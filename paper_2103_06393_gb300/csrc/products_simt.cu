// Plain complex-FP32 forms of Algorithm 1 (Y = Z X) and Algorithm 2 (Psi = Z^H Phi) on CUDA
// cores (Sec. III.B), plus the ACA pre/post products X' = V^H X and Psi = V Psi'.
//
// The decompressed column never reaches HBM: a CTA decompresses its voxel tile column by
// column and either accumulates Y^k[v,s] += Z[v,j] X[j,s] in registers (Algorithm 1) or
// reduces sum_v conj(Z[v,j]) Phi^k[v,s] over the tile (Algorithm 2) into a per-CTA
// accumulator that a second kernel sums in a fixed order.  The per-column inputs arrive through
// the bulk-copy stage pipeline of stage.cuh: warps 0 .. ntask-1 compute (one task of 32 i1 x
// kUQ i2 each), warp ntask copies (and, in Algorithm 2, sums the warps' per-column results).
#include <algorithm>

#include "stage.cuh"

namespace zbc {

// NT = compute warps per CTA at most (template): 6 (7 warps with the copy warp, up to 255
// registers per thread) or 9 (10 warps, 168 registers); chosen per call (zbc_tune), default 9
constexpr size_t kSmemBudget = 220 * 1024;
constexpr int kAdjStages = 4;  // adjoint stage ring depth (the per-column sums take the rest; 6 or 8
                               // measured no faster)

// ---------------------------------------------------------------------------------------------
// warp reduce-scatter of NV floats per lane: afterwards lane l holds the warp sum of value index
// (l >> (5 - log2 NV)); 31 shuffles for NV = 32 instead of 160 for independent butterflies.
// ---------------------------------------------------------------------------------------------
template <int NV>
struct Log2 {
  static constexpr int v = NV == 1 ? 0 : NV == 2 ? 1 : NV == 4 ? 2 : NV == 8 ? 3 : NV == 16 ? 4 : 5;
};

template <int NV>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[NV], int lane) {
  constexpr int LOG = Log2<NV>::v;
  static_assert((1 << LOG) == NV, "NV must be a power of two <= 32");
#pragma unroll
  for (int step = 0; step < LOG; ++step) {
    const int o = 16 >> step;
    const int c = NV >> step;  // live values
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < c / 2; ++i) {
      const float send = upper ? v[i] : v[i + c / 2];
      const float keep = upper ? v[i + c / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  float r = v[0];
#pragma unroll
  for (int o = 16 >> LOG; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

// X^T[j][s] = X[j, s] for s < p, zero up to the row stride pst (a whole number of s-chunks)
__global__ void __launch_bounds__(256) transpose_x_kernel(const float2* __restrict__ X, int64_t ldx, int M, int p,
                                                          int pst, float2* __restrict__ XT, int* __restrict__ err) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * pst) return;
  const int j = (int)(e / pst), s = (int)(e % pst);
  const float2 v = s < p ? X[j + ldx * s] : make_float2(0.f, 0.f);
  if (!(isfinite(v.x) && isfinite(v.y))) atomicOr(err, kErrNonFinite);
  XT[e] = v;
}

int transpose_rhs(Handle& h, const float2* X, int64_t ldx, int p, int chunk, const float2** XT, int* pst,
                  cudaStream_t st) {
  *pst = (ceil_div(p, chunk) * chunk + 1) / 2 * 2;
  ZBC_TRY(h.work_xt.ensure(sizeof(float2) * (size_t)h.M * *pst));
  float2* xt = (float2*)h.work_xt.ptr;
  transpose_x_kernel<<<ceil_div((int64_t)h.M * *pst, 256), 256, 0, st>>>(X, ldx, h.M, p, *pst, xt,
                                                                          (int*)h.work_err.ptr);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  *XT = xt;
  return ZBC_OK;
}

// ---------------------------------------------------------------------------------------------
// Algorithm 1: one CTA per (voxel tile, component k, s-chunk); items = the M stored columns
// ---------------------------------------------------------------------------------------------
template <int PS, int NT>
__global__ void __launch_bounds__(32 * (NT + 1), 1)
    matvec_simt_kernel(const float2* __restrict__ cache, const CacheDesc* __restrict__ cdesc, Geo g, int q, int M,
                       StageLayout SL, int S, const float2* __restrict__ XT, int pst, int p,
                       float2* __restrict__ Y, int64_t ldy, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[kMaxStages], empty[kMaxStages];
  __shared__ int meta[kMaxStages];
  __shared__ volatile int abort_flag;
  const int k = blockIdx.y;
  const int s0 = blockIdx.z * PS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ncw = g.ntask;
  const int B1p = (g.B1 + 1) / 2 * 2;
  int i1_0, i2_0, i3;
  g.tile(blockIdx.x, i1_0, i2_0, i3);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], ncw);
    }
    abort_flag = 0;
  }
  __syncthreads();

  if (warp == ncw) {
    // ---------------- producer ----------------
    if (lane == 0) {
      const uint32_t xb = StageLayout::r16(8u * PS);
      int issued = 0;
      for (int c = 0; c < M; ++c) {
        const int st = c % S;
        if (c >= S && (abort_flag || !tc::mbar_wait(&empty[st], ((c / S) - 1) & 1))) {
          abort_flag = 1;
          break;
        }
        const CacheDesc d = cdesc[(int64_t)c * q + k];
        issue_item(smem + (size_t)st * SL.stride, SL, &full[st], &meta[st], cache, d, g, B1p, i1_0, i2_0, i3,
                   XT + (int64_t)c * pst + s0, xb);
        issued = c + 1;
      }
      if (abort_flag)  // let the copies in flight land before the CTA exits
        for (int c = std::max(0, issued - S); c < issued; ++c) tc::mbar_wait(&full[c % S], (c / S) & 1);
    }
  } else {
    // ---------------- consumers ----------------
    int i1, u0;
    bool ok;
    g.task(i1_0, warp, lane, i1, u0, ok);
    const int il = ok ? i1 - i1_0 : 0;
    float2 acc[kUQ][PS];
#pragma unroll
    for (int l = 0; l < kUQ; ++l)
#pragma unroll
      for (int i = 0; i < PS; ++i) acc[l][i] = make_float2(0.f, 0.f);
    for (int c = 0; c < M; ++c) {
      const int st = c % S;
      // warp-uniform decisions: the warp shuffles below need every lane
      if (__any_sync(0xffffffffu, abort_flag != 0)) break;
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&full[st], (c / S) & 1))) {
        if (lane == 0) abort_flag = 1;
        break;
      }
      const unsigned char* sb = smem + (size_t)st * SL.stride;
      float2 z[kUQ];
      last_mode_staged((const float2*)(sb + SL.u1), B1p, il, (const float2*)(sb + SL.w), meta[st], u0, z);
      if constexpr (PS == 1) {
        const float2 x = *(const float2*)(sb + SL.x);
#pragma unroll
        for (int l = 0; l < kUQ; ++l) acc[l][0] = cfma(z[l], x, acc[l][0]);
      } else {
        const float4* xs = (const float4*)(sb + SL.x);
#pragma unroll
        for (int i = 0; i < PS / 2; ++i) {
          const float4 x = xs[i];
#pragma unroll
          for (int l = 0; l < kUQ; ++l) {
            acc[l][2 * i] = cfma(z[l], make_float2(x.x, x.y), acc[l][2 * i]);
            acc[l][2 * i + 1] = cfma(z[l], make_float2(x.z, x.w), acc[l][2 * i + 1]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive1(&empty[st]);
    }
    if (ok && !abort_flag) {
      const int64_t nv = (int64_t)g.n1 * g.n2 * g.n3;
#pragma unroll
      for (int l = 0; l < kUQ; ++l) {
        const int i2 = i2_0 + u0 + l;
        if (u0 + l >= g.NU || i2 >= g.n2) continue;
        const int64_t v = i1 + (int64_t)g.n1 * (i2 + (int64_t)g.n2 * i3);
        float2* y = Y + k * nv + v;
#pragma unroll
        for (int i = 0; i < PS; ++i)
          if (s0 + i < p) y[ldy * (s0 + i)] = acc[l][i];
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag) atomicOr(err, kErrTimeout);
}

// ---------------------------------------------------------------------------------------------
// Algorithm 2: grid (G, q * jblocks, s-chunks).  The (tile, column) items of one j-block are
// split into G equal contiguous ranges, one per CTA; a CTA's partial sums go to
// partial[(cta * q + k)][s][j] (M x p), summed over the G CTAs by reduce_partials_kernel.
// Per item, each consumer warp reduces its voxels' sum_v conj(Z[v,j]) Phi[v,s] with a warp
// reduce-scatter into the stage's red[warp][NV]; the producer warp adds the warps' values in
// warp order into pacc[j][NV] (fixed order: results are reproducible) before it reuses the stage.
// ---------------------------------------------------------------------------------------------
// Bounded wait on an mbarrier phase that also gives up once another warp of the CTA has set
// *abort_flag (checked between slices of 1024 polls; kWaitPolls polls in all).
__device__ __forceinline__ bool wait_or_abort(uint64_t* mbar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t done = 0; done < kWaitPolls; done += 1024u) {
    if (*abort_flag) return false;
    if (tc::mbar_wait(mbar, parity, 1024u)) return true;
  }
  return false;
}

// first_wait: polls allowed to each consumer warp's wait for its first stage (kWaitPolls, or the
// test limit of zbc_test_wait_limit, which makes that wait give up and the CTA abort).  Non-finite
// Phi values set kErrNonFinite in err.
template <int PS, int NT>
__global__ void __launch_bounds__(32 * (NT + 1), 1)
    rmatvec_simt_kernel(const float2* __restrict__ cache, const CacheDesc* __restrict__ cdesc, Geo g, int q, int M,
                        int MJ, StageLayout SL, int S, const float2* __restrict__ Phi, int64_t ldphi, int p,
                        float2* __restrict__ partial, int* __restrict__ err, uint32_t first_wait) {
  constexpr int NV = 2 * PS;
  constexpr int NH = PS > 8 ? 2 : 1;  // halves of the right-hand sides
  constexpr int PSH = PS / NH, NVH = 2 * PSH;
  constexpr int SHH = 5 - Log2<NVH>::v;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[kMaxStages], empty[kMaxStages];
  __shared__ int meta[kMaxStages];
  __shared__ volatile int abort_flag;
  float* pacc = (float*)(smem + (size_t)S * SL.stride);  // [MJ][NV]
  const int k = blockIdx.y % q;
  const int jb0 = (blockIdx.y / q) * MJ;
  const int nj = min(M, jb0 + MJ) - jb0;
  const int s0 = blockIdx.z * PS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ncw = g.ntask;
  const int B1p = (g.B1 + 1) / 2 * 2;
  const int64_t N = (int64_t)g.ntiles() * nj;
  const int64_t c0 = N * blockIdx.x / gridDim.x;
  const int nitems = (int)(N * (blockIdx.x + 1) / gridDim.x - c0);
  for (int e = threadIdx.x; e < nj * NV; e += blockDim.x) pacc[e] = 0.f;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], ncw);
    }
    abort_flag = 0;
  }
  __syncthreads();

  if (warp == ncw) {
    // ---------------- producer and reducer ----------------
    // item c (local) -> global index c0 + c -> (tile (c0 + c) / nj, column jb0 + (c0 + c) % nj)
    auto reduce = [&](int c) {
      const int jl = (int)((c0 + c) % nj);
      const float* red = (const float*)(smem + (size_t)(c % S) * SL.stride + SL.red);
      if (lane < NV) {
        float sum = 0.f;
        for (int w = 0; w < ncw; ++w) sum += red[w * NV + lane];
        pacc[jl * NV + lane] += sum;
      }
    };
    int t = (int)(c0 / (nj > 0 ? nj : 1)), jl = (int)(c0 % (nj > 0 ? nj : 1));
    int issued = 0;
    for (int c = 0; c < nitems; ++c) {
      const int st = c % S;
      if (c >= S) {
        bool bad = abort_flag != 0;
        if (!bad) bad = !wait_or_abort(&empty[st], ((c / S) - 1) & 1, &abort_flag);
        if (__any_sync(0xffffffffu, bad)) {
          if (lane == 0) abort_flag = 1;
          break;
        }
        reduce(c - S);
        __syncwarp();
      }
      if (lane == 0) {
        int i1_0, i2_0, i3;
        g.tile(t, i1_0, i2_0, i3);
        const CacheDesc d = cdesc[(int64_t)(jb0 + jl) * q + k];
        issue_item(smem + (size_t)st * SL.stride, SL, &full[st], &meta[st], cache, d, g, B1p, i1_0, i2_0, i3,
                   nullptr, 0u);
      }
      issued = c + 1;
      if (++jl == nj) {
        jl = 0;
        ++t;
      }
    }
    if (!__any_sync(0xffffffffu, abort_flag != 0)) {
      for (int c = std::max(0, nitems - S); c < nitems; ++c) {
        bool bad = abort_flag != 0;
        if (!bad) bad = !wait_or_abort(&empty[c % S], (c / S) & 1, &abort_flag);
        if (__any_sync(0xffffffffu, bad)) {
          if (lane == 0) abort_flag = 1;
          break;
        }
        reduce(c);
      }
    }
    if (abort_flag && lane == 0)  // let the copies in flight land before the CTA exits
      for (int c = std::max(0, issued - S); c < issued; ++c) tc::mbar_wait(&full[c % S], (c / S) & 1);
  } else {
    // ---------------- consumers ----------------
    const int64_t nv = (int64_t)g.n1 * g.n2 * g.n3;
    int t = (int)(c0 / (nj > 0 ? nj : 1)), jl = (int)(c0 % (nj > 0 ? nj : 1));
    int tcur = -1, il = 0, u0 = 0;
    bool okl[kUQ];
    bool finite = true;
    float2 ph[kUQ][PS];
    for (int c = 0; c < nitems; ++c) {
      const int st = c % S;
      if (t != tcur) {
        // the task's Phi values on this tile (zero outside the grid)
        tcur = t;
        int i1_0, i2_0, i3, i1;
        bool ok;
        g.tile(t, i1_0, i2_0, i3);
        g.task(i1_0, warp, lane, i1, u0, ok);
        il = ok ? i1 - i1_0 : 0;
#pragma unroll
        for (int l = 0; l < kUQ; ++l) {
          const int i2 = i2_0 + u0 + l;
          okl[l] = ok && (u0 + l) < g.NU && i2 < g.n2;
          const int64_t v = i1 + (int64_t)g.n1 * (i2 + (int64_t)g.n2 * i3);
#pragma unroll
          for (int i = 0; i < PS; ++i) {
            ph[l][i] = (okl[l] && s0 + i < p) ? Phi[k * nv + v + ldphi * (s0 + i)] : make_float2(0.f, 0.f);
            finite = finite && isfinite(ph[l][i].x) && isfinite(ph[l][i].y);
          }
        }
      }
      if (++jl == nj) {
        jl = 0;
        ++t;
      }
      // warp-uniform decisions: the warp shuffles below need every lane
      if (__any_sync(0xffffffffu, abort_flag != 0)) break;
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&full[st], (c / S) & 1, c == 0 ? first_wait : kWaitPolls))) {
        if (lane == 0) abort_flag = 1;
        break;
      }
      unsigned char* sb = smem + (size_t)st * SL.stride;
      float2 z[kUQ];
      last_mode_staged((const float2*)(sb + SL.u1), B1p, il, (const float2*)(sb + SL.w), meta[st], u0, z);
      // the contraction in halves of at most 8 right-hand sides: two reduce-scatters of 16 values
      // take as many shuffles as one of 32 and need half the registers
#pragma unroll
      for (int hf = 0; hf < NH; ++hf) {
        float vals[NVH];
#pragma unroll
        for (int i = 0; i < PSH; ++i) {
          float re = 0.f, im = 0.f;
#pragma unroll
          for (int l = 0; l < kUQ; ++l) {
            const float2 zz = okl[l] ? z[l] : make_float2(0.f, 0.f);
            const float2 f = ph[l][hf * PSH + i];
            re = fmaf(zz.x, f.x, fmaf(zz.y, f.y, re));
            im = fmaf(zz.x, f.y, fmaf(-zz.y, f.x, im));
          }
          vals[2 * i] = re;
          vals[2 * i + 1] = im;
        }
        const float r = warp_reduce_scatter<NVH>(vals, lane);
        if ((lane & ((1 << SHH) - 1)) == 0)
          ((float*)(sb + SL.red))[warp * NV + hf * NVH + (lane >> SHH)] = r;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive1(&empty[st]);
    }
    if (!finite) atomicOr(err, kErrNonFinite);
  }
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag) atomicOr(err, kErrTimeout);
  float2* out = partial + (int64_t)(blockIdx.x * q + k) * M * p;
  for (int e = threadIdx.x; e < nj * PS; e += blockDim.x) {
    const int j = e % nj, i = e / nj;
    if (s0 + i < p) out[(jb0 + j) + (int64_t)M * (s0 + i)] = make_float2(pacc[j * NV + 2 * i], pacc[j * NV + 2 * i + 1]);
  }
}

// Psi'[j, s] = sum_{g} partial[g][s][j], fixed order
__global__ void __launch_bounds__(256) reduce_partials_kernel(const float2* __restrict__ partial, int ng, int M, int p,
                                                              float2* __restrict__ out, int64_t ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)M * p) return;
  const int j = (int)(e % M), s = (int)(e / M);
  float2 acc = make_float2(0.f, 0.f);
  for (int g = 0; g < ng; ++g) {
    const float2 v = partial[(int64_t)g * M * p + e];
    acc.x += v.x;
    acc.y += v.y;
  }
  out[j + ldo * s] = acc;
}

// out = op(V) * B:  conj=1 -> V^H B (V is m x M, out M x p); conj=0 -> V B (out m x p)
__global__ void __launch_bounds__(256) small_gemm_kernel(const float2* __restrict__ V, int m, int Mc, int conj,
                                                         const float2* __restrict__ B, int64_t ldb, int p,
                                                         float2* __restrict__ out, int64_t ldo) {
  const int rows = conj ? Mc : m;
  const int K = conj ? m : Mc;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * p) return;
  const int r = (int)(e % rows), s = (int)(e / rows);
  float2 acc = make_float2(0.f, 0.f);
  if (conj) {
    for (int i = 0; i < K; ++i) acc = cfma_conj(V[i + (int64_t)m * r], B[i + ldb * s], acc);
  } else {
    for (int i = 0; i < K; ++i) acc = cfma(V[r + (int64_t)m * i], B[i + ldb * s], acc);
  }
  out[r + ldo * s] = acc;
}

int aca_pre(const Handle& h, const float2* X, int64_t ldx, int p, float2* Xp, cudaStream_t st) {
  const int64_t n = (int64_t)h.M * p;
  small_gemm_kernel<<<ceil_div(n, 256), 256, 0, st>>>(h.d_v, h.m, h.M, 1, X, ldx, p, Xp, h.M);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}
int aca_post(const Handle& h, const float2* Psip, int p, float2* Psi, int64_t ldpsi, cudaStream_t st) {
  const int64_t n = (int64_t)h.m * p;
  small_gemm_kernel<<<ceil_div(n, 256), 256, 0, st>>>(h.d_v, h.m, h.M, 0, Psip, h.M, p, Psi, ldpsi);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}



int reduce_partials(const float2* partial, int ng, int M, int p, float2* out, int64_t ldo, cudaStream_t st) {
  reduce_partials_kernel<<<ceil_div((int64_t)M * p, 256), 256, 0, st>>>(partial, ng, M, p, out, ldo);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}


// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
template <int PS, int NT>
static int launch_matvec(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  ZBC_TRY(build_decomp_cache(h, st));
  const Geo g = make_geo(h.n1, h.n2, h.n3, 0, NT);
  const int R = h.cache_r;
  const int B1p = tile_b1p(h.n1);
  const int schunks = ceil_div(p, PS);
  const float2* XT;
  int pst;
  ZBC_TRY(transpose_rhs(h, X, ldx, p, PS, &XT, &pst, st));
  const StageLayout SL = StageLayout::make(R, B1p, g.NUp, 8 * PS, 0);
  const int S = (int)std::min<size_t>(kMaxStages, kSmemBudget / SL.stride);
  ZBC_CHECK_ARG(S >= 2, "rank %d too large for the FP32 SIMT path", R);
  const size_t sm = (size_t)S * SL.stride;
  ZBC_TRY((set_smem_limit<matvec_simt_kernel<PS, NT>>((int)kSmemBudget)));
  dim3 grid(g.ntiles(), h.q, schunks);
  matvec_simt_kernel<PS, NT><<<grid, 32 * (g.ntask + 1), sm, st>>>(h.cache->data, h.cache->d_desc, g, h.q, h.M, SL, S,
                                                               XT, pst, p, Y, ldy, (int*)h.work_err.ptr);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

// Algorithm 2 with the partial sums in `scratch` (scratch_bytes) or, when scratch is null, in
// the handle's workspace (grown as needed).
template <int PS, int NT>
static int launch_rmatvec(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo,
                          float2* scratch, size_t scratch_bytes, cudaStream_t st) {
  if (!scratch) ZBC_TRY(build_decomp_cache(h, st));
  const Geo g = make_geo(h.n1, h.n2, h.n3, 0, NT);
  const int R = h.cache_r;
  const int B1p = tile_b1p(h.n1);
  constexpr int NV = 2 * PS;
  const StageLayout SL = StageLayout::make(R, B1p, g.NUp, 0, 4 * NV * g.ntask);
  // stages first (4, or as many as fit), the rest of shared memory holds the j-block's sums
  const int S = (int)std::min<size_t>(kAdjStages, kSmemBudget / SL.stride);
  ZBC_CHECK_ARG(S >= 2, "rank %d too large for the FP32 SIMT adjoint", R);
  const size_t left = kSmemBudget - (size_t)S * SL.stride;
  const int MJmax = (int)std::min<size_t>(h.M, left / (sizeof(float) * NV));
  ZBC_CHECK_ARG(MJmax >= 1, "rank %d too large for the FP32 SIMT adjoint", R);
  const int jblocks = ceil_div(h.M, MJmax);
  const int MJ = ceil_div(h.M, jblocks);  // balanced j-blocks
  const int schunks = ceil_div(p, PS);
  const size_t per_group = sizeof(float2) * (size_t)h.q * h.M * p;
  int G = std::max(1, sm_count() / std::max(1, h.q * jblocks * schunks));
  G = std::min(G, std::max(1, g.ntiles()));
  if (scratch) {
    const size_t gmax = scratch_bytes / per_group;
    ZBC_CHECK_ARG(gmax >= 1, "scratch of %zu bytes cannot hold one partial-sum group (%zu bytes)", scratch_bytes,
                  per_group);
    G = (int)std::min<size_t>(G, gmax);
  } else {
    ZBC_TRY(h.work_partial.ensure(per_group * G));
    scratch = (float2*)h.work_partial.ptr;
  }
  const size_t sm = (size_t)S * SL.stride + sizeof(float) * (size_t)MJ * NV;
  ZBC_TRY((set_smem_limit<rmatvec_simt_kernel<PS, NT>>((int)kSmemBudget)));
  dim3 grid(G, h.q * jblocks, schunks);
  rmatvec_simt_kernel<PS, NT><<<grid, 32 * (g.ntask + 1), sm, st>>>(h.cache->data, h.cache->d_desc, g, h.q, h.M, MJ, SL,
                                                                S, Phi, ldphi, p, scratch, (int*)h.work_err.ptr,
                                                                h.test_first_wait);
  h.test_first_wait = kWaitPolls;  // a test limit applies to one launch
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return reduce_partials(scratch, G * h.q, h.M, p, out, ldo, st);
}

template <int NT>
static int rmatvec_dispatch(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo,
                            float2* scratch, size_t scratch_bytes, cudaStream_t st) {
  if (p == 1) return launch_rmatvec<1, NT>(h, Phi, ldphi, p, out, ldo, scratch, scratch_bytes, st);
  if (p == 2) return launch_rmatvec<2, NT>(h, Phi, ldphi, p, out, ldo, scratch, scratch_bytes, st);
  if (p <= 4) return launch_rmatvec<4, NT>(h, Phi, ldphi, p, out, ldo, scratch, scratch_bytes, st);
  if (p <= 8) return launch_rmatvec<8, NT>(h, Phi, ldphi, p, out, ldo, scratch, scratch_bytes, st);
  return launch_rmatvec<16, NT>(h, Phi, ldphi, p, out, ldo, scratch, scratch_bytes, st);
}

template <int NT>
static int matvec_dispatch(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  if (p == 1) return launch_matvec<1, NT>(h, X, ldx, p, Y, ldy, st);
  if (p == 2) return launch_matvec<2, NT>(h, X, ldx, p, Y, ldy, st);
  if (p <= 4) return launch_matvec<4, NT>(h, X, ldx, p, Y, ldy, st);
  if (p <= 8) return launch_matvec<8, NT>(h, X, ldx, p, Y, ldy, st);
  return launch_matvec<16, NT>(h, X, ldx, p, Y, ldy, st);
}

int rmatvec_simt_scratch(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo,
                         float2* scratch, size_t scratch_bytes, cudaStream_t st) {
  if (!h.cache) {
    set_error("the handle's decompression cache is not built: call zbc_matvec or zbc_rmatvec on it once first");
    return ZBC_EINVAL;
  }
  if (h.tune_adj_warps[rhs_class(p)] == 6)
    return rmatvec_dispatch<6>(h, Phi, ldphi, p, out, ldo, scratch, scratch_bytes, st);
  return rmatvec_dispatch<9>(h, Phi, ldphi, p, out, ldo, scratch, scratch_bytes, st);
}

// warps: compute warps per CTA, 6 or 9 (anything else: 9)
int matvec_simt(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, int warps, cudaStream_t st) {
  if (warps == 6) return matvec_dispatch<6>(h, X, ldx, p, Y, ldy, st);
  return matvec_dispatch<9>(h, X, ldx, p, Y, ldy, st);
}

int rmatvec_simt(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo, int warps,
                 cudaStream_t st) {
  if (warps == 6) return rmatvec_dispatch<6>(h, Phi, ldphi, p, out, ldo, nullptr, 0, st);
  return rmatvec_dispatch<9>(h, Phi, ldphi, p, out, ldo, nullptr, 0, st);
}

}  // namespace zbc
