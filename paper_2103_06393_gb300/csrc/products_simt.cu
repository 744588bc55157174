// Plain complex-FP32 forms of Algorithm 1 (Y = Z X) and Algorithm 2 (Psi = Z^H Phi) on CUDA
// cores (Sec. III.B), plus the ACA pre/post products X' = V^H X and Psi = V Psi'.
//
// The decompressed column never reaches HBM: a CTA decompresses its voxel tile column by
// column (chunked front end in decomp.cuh) and either accumulates Y^k[v,s] += Z[v,j] X[j,s]
// in registers (Algorithm 1) or reduces sum_v conj(Z[v,j]) Phi^k[v,s] over the tile
// (Algorithm 2) into a per-CTA accumulator that a second kernel sums in a fixed order.
#include <algorithm>

#include "decomp.cuh"

namespace zbc {

// ---------------------------------------------------------------------------------------------
// Algorithm 1: one task (32 i1 x kUQ u) per warp
// ---------------------------------------------------------------------------------------------
template <int PS>
__global__ void __launch_bounds__(kThreads, 1)
    matvec_simt_kernel(const float2* __restrict__ cache, const CacheDesc* __restrict__ cdesc, Geo g, int q, int M,
                       int R, const float2* __restrict__ X, int64_t ldx, int p, float2* __restrict__ Y,
                       int64_t ldy) {
  extern __shared__ __align__(16) unsigned char smem[];
  // two front-end buffers (chunk c uses buffer c & 1), so one barrier per chunk suffices
  const FrontEnd2 fe(smem, R, g.NUp, kChunk * PS);
  const int k = blockIdx.y;
  const int s0 = blockIdx.z * PS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tid = threadIdx.x, nthr = blockDim.x;
  int i1_0, i2_0, i3;
  g.tile(blockIdx.x, i1_0, i2_0, i3);
  const bool active = warp < g.ntask;
  int i1 = 0, u0 = 0;
  bool ok = false;
  if (active) g.task(i1_0, warp, lane, i1, u0, ok);
  float2 acc[kUQ][PS];
#pragma unroll
  for (int l = 0; l < kUQ; ++l)
#pragma unroll
    for (int i = 0; i < PS; ++i) acc[l][i] = make_float2(0.f, 0.f);
  WPrefetch pf;
  pf.load(cache, cdesc, g, R, q, k, 0, min(kChunk, M), i2_0, i3, tid, nthr);
  for (int j0 = 0, c = 0; j0 < M; j0 += kChunk, ++c) {
    const int jc = min(kChunk, M - j0);
    const int b = c & 1;
    const ChunkSmem cs = fe.cs(b);
    float2* xs = fe.xs(b);
    for (int e = tid; e < jc * PS; e += nthr) {
      const int jj = e / PS, i = e % PS;
      xs[e] = (s0 + i < p) ? X[(j0 + jj) + ldx * (s0 + i)] : make_float2(0.f, 0.f);
    }
    pf.store(cs, g, R, jc, tid, nthr);
    __syncthreads();
    if (j0 + kChunk < M)
      pf.load(cache, cdesc, g, R, q, k, j0 + kChunk, min(kChunk, M - j0 - kChunk), i2_0, i3, tid, nthr);
    if (active) {
      for (int jj = 0; jj < jc; ++jj) {
        const CacheDesc d = cs.cd[jj];
        float2 z[kUQ];
        last_mode4(cache + d.uoff + (int64_t)i1 * d.r1p, d.r1, ok, cs.W + (size_t)jj * R * g.NUp, g.NUp, u0, z);
#pragma unroll
        for (int i = 0; i < PS; ++i) {
          const float2 x = xs[jj * PS + i];
#pragma unroll
          for (int l = 0; l < kUQ; ++l) acc[l][i] = cfma(z[l], x, acc[l][i]);
        }
      }
    }
  }
  if (!active || !ok) return;
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

// ---------------------------------------------------------------------------------------------
// Algorithm 2: per-CTA partial sums over its tiles, partial[(cta*q+k)][s][j] (M x p)
// ---------------------------------------------------------------------------------------------
template <int PS>
__global__ void __launch_bounds__(kThreads, 1)
    rmatvec_simt_kernel(const float2* __restrict__ cache, const CacheDesc* __restrict__ cdesc, Geo g, int q, int M,
                        int R, int MJ, const float2* __restrict__ Phi, int64_t ldphi, int p,
                        float2* __restrict__ partial) {
  constexpr int NV = 2 * PS;
  constexpr int SH = 5 - Log2<NV>::v;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nw = blockDim.x >> 5;
  const FrontEnd2 fe(smem, R, g.NUp, 0);   // chunk c uses buffer c & 1
  float* red = (float*)fe.end();            // [kChunk][nw][NV]
  float* pacc = red + kChunk * nw * NV;     // [MJ][NV]
  const int k = blockIdx.y % q;
  const int jb0 = (blockIdx.y / q) * MJ;
  const int jb1 = min(M, jb0 + MJ);
  const int s0 = blockIdx.z * PS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int64_t nv = (int64_t)g.n1 * g.n2 * g.n3;
  const bool active = warp < g.ntask;
  for (int e = threadIdx.x; e < (jb1 - jb0) * NV; e += blockDim.x) pacc[e] = 0.f;
  int c = 0;
  for (int t = blockIdx.x; t < g.ntiles(); t += gridDim.x) {
    int i1_0, i2_0, i3;
    g.tile(t, i1_0, i2_0, i3);
    int i1 = 0, u0 = 0;
    bool ok = false;
    if (active) g.task(i1_0, warp, lane, i1, u0, ok);
    float2 ph[kUQ][PS];
#pragma unroll
    for (int l = 0; l < kUQ; ++l) {
      const int i2 = i2_0 + u0 + l;
      const bool okl = ok && (u0 + l) < g.NU && i2 < g.n2;
      const int64_t v = i1 + (int64_t)g.n1 * (i2 + (int64_t)g.n2 * i3);
#pragma unroll
      for (int i = 0; i < PS; ++i)
        ph[l][i] = (okl && s0 + i < p) ? Phi[k * nv + v + ldphi * (s0 + i)] : make_float2(0.f, 0.f);
    }
    WPrefetch pf;
    pf.load(cache, cdesc, g, R, q, k, jb0, min(kChunk, jb1 - jb0), i2_0, i3, tid, nthr);
    for (int j0 = jb0; j0 < jb1; j0 += kChunk, ++c) {
      const int jc = min(kChunk, jb1 - j0);
      const ChunkSmem cs = fe.cs(c & 1);
      pf.store(cs, g, R, jc, tid, nthr);
      __syncthreads();
      if (j0 + kChunk < jb1)
        pf.load(cache, cdesc, g, R, q, k, j0 + kChunk, min(kChunk, jb1 - j0 - kChunk), i2_0, i3, tid, nthr);
      for (int jj = 0; jj < jc; ++jj) {
        const CacheDesc d = cs.cd[jj];
        float2 z[kUQ];
        last_mode4(cache + d.uoff + (int64_t)i1 * d.r1p, d.r1, ok && active, cs.W + (size_t)jj * R * g.NUp, g.NUp,
                   u0, z);
        float vals[NV];
#pragma unroll
        for (int i = 0; i < PS; ++i) {
          float re = 0.f, im = 0.f;
#pragma unroll
          for (int l = 0; l < kUQ; ++l) {
            re = fmaf(z[l].x, ph[l][i].x, fmaf(z[l].y, ph[l][i].y, re));
            im = fmaf(z[l].x, ph[l][i].y, fmaf(-z[l].y, ph[l][i].x, im));
          }
          vals[2 * i] = re;
          vals[2 * i + 1] = im;
        }
        const float r = warp_reduce_scatter<NV>(vals, lane);
        if ((lane & ((1 << SH) - 1)) == 0) red[(jj * nw + warp) * NV + (lane >> SH)] = r;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < jc * NV; e += blockDim.x) {
        const int jj = e / NV, i = e % NV;
        float tsum = 0.f;
        for (int w = 0; w < nw; ++w) tsum += red[(jj * nw + w) * NV + i];
        pacc[(j0 + jj - jb0) * NV + i] += tsum;
      }
    }
  }
  __syncthreads();
  float2* out = partial + (int64_t)(blockIdx.x * q + k) * M * p;
  for (int e = threadIdx.x; e < (jb1 - jb0) * PS; e += blockDim.x) {
    const int jl = e % (jb1 - jb0), i = e / (jb1 - jb0);
    if (s0 + i < p) out[(jb0 + jl) + (int64_t)M * (s0 + i)] = make_float2(pacc[jl * NV + 2 * i], pacc[jl * NV + 2 * i + 1]);
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

template <int PS>
static int launch_matvec(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  ZBC_TRY(build_decomp_cache(h, st));
  const int R = h.cache_r;
  Geo g = make_geo(h.n1, h.n2, h.n3, R, 8);
  const int nthr = 32 * std::max(4, g.ntask);
  const size_t sm = 2 * FrontEnd2::buf_bytes(R, g.NUp, kChunk * PS);
  static bool attr_set = false;
  if (!attr_set) {
    ZBC_TRY_CUDA(cudaFuncSetAttribute(matvec_simt_kernel<PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    attr_set = true;
  }
  ZBC_CHECK_ARG(sm <= 220 * 1024, "rank %d too large for the FP32 SIMT path", R);
  dim3 grid(g.ntiles(), h.q, ceil_div(p, PS));
  matvec_simt_kernel<PS><<<grid, nthr, sm, st>>>(h.cache->data, h.cache->d_desc, g, h.q, h.M, R, X, ldx, p, Y,
                                                     ldy);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

template <int PS>
static int launch_rmatvec(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo,
                          cudaStream_t st) {
  ZBC_TRY(build_decomp_cache(h, st));
  const int R = h.cache_r;
  Geo g = make_geo(h.n1, h.n2, h.n3, R, 8);
  const int NV = 2 * PS;
  const int nthr = 32 * std::max(4, g.ntask);
  const size_t base = 2 * FrontEnd2::buf_bytes(R, g.NUp, 0) + sizeof(float) * kChunk * (nthr / 32) * NV;
  // j-block so that the per-CTA accumulator stays within the shared-memory budget
  const size_t budget = 220 * 1024 - base;
  const int MJ = std::max(kChunk, std::min(h.M, (int)(budget / (NV * sizeof(float))) / kChunk * kChunk));
  const int jblocks = ceil_div(h.M, MJ);
  const int schunks = ceil_div(p, PS);
  const int target = 2 * sm_count();
  int G = std::max(1, target / std::max(1, h.q * jblocks * schunks));
  G = std::min(G, g.ntiles());
  const size_t sm = base + sizeof(float) * (size_t)MJ * NV;
  static bool attr_set = false;
  if (!attr_set) {
    ZBC_TRY_CUDA(cudaFuncSetAttribute(rmatvec_simt_kernel<PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    attr_set = true;
  }
  ZBC_CHECK_ARG(sm <= 220 * 1024, "rank %d too large for the FP32 SIMT adjoint", R);
  ZBC_TRY(h.work_partial.ensure(sizeof(float2) * (size_t)G * h.q * h.M * p));
  float2* partial = (float2*)h.work_partial.ptr;
  dim3 grid(G, h.q * jblocks, schunks);
  rmatvec_simt_kernel<PS><<<grid, nthr, sm, st>>>(h.cache->data, h.cache->d_desc, g, h.q, h.M, R, MJ, Phi, ldphi,
                                                  p, partial);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return reduce_partials(partial, G * h.q, h.M, p, out, ldo, st);
}

// The same adjoint with caller-provided scratch for the partial sums and no allocation at all:
// the decompression cache must already exist, and the number of partial-sum groups is capped
// so that they fit scratch_bytes.
template <int PS>
static int launch_rmatvec_scratch(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo,
                                  float2* scratch, size_t scratch_bytes, cudaStream_t st) {
  const int R = h.cache_r;
  Geo g = make_geo(h.n1, h.n2, h.n3, R, 8);
  const int NV = 2 * PS;
  const int nthr = 32 * std::max(4, g.ntask);
  const size_t base = 2 * FrontEnd2::buf_bytes(R, g.NUp, 0) + sizeof(float) * kChunk * (nthr / 32) * NV;
  const size_t budget = 220 * 1024 - base;
  const int MJ = std::max(kChunk, std::min(h.M, (int)(budget / (NV * sizeof(float))) / kChunk * kChunk));
  const int jblocks = ceil_div(h.M, MJ);
  const int schunks = ceil_div(p, PS);
  const size_t per_group = sizeof(float2) * (size_t)h.q * h.M * p;
  const int gmax = (int)std::min<size_t>(scratch_bytes / per_group, 1 << 20);
  ZBC_CHECK_ARG(gmax >= 1, "scratch of %zu bytes cannot hold one partial-sum group (%zu bytes)", scratch_bytes,
                per_group);
  int G = std::max(1, 2 * sm_count() / std::max(1, h.q * jblocks * schunks));
  G = std::min(std::min(G, g.ntiles()), gmax);
  const size_t sm = base + sizeof(float) * (size_t)MJ * NV;
  ZBC_CHECK_ARG(sm <= 220 * 1024, "rank %d too large for the FP32 SIMT adjoint", R);
  ZBC_TRY_CUDA(cudaFuncSetAttribute(rmatvec_simt_kernel<PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
  dim3 grid(G, h.q * jblocks, schunks);
  rmatvec_simt_kernel<PS><<<grid, nthr, sm, st>>>(h.cache->data, h.cache->d_desc, g, h.q, h.M, R, MJ, Phi, ldphi,
                                                  p, scratch);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return reduce_partials(scratch, G * h.q, h.M, p, out, ldo, st);
}

int rmatvec_simt_scratch(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo,
                         float2* scratch, size_t scratch_bytes, cudaStream_t st) {
  if (!h.cache) {
    set_error("the handle's decompression cache is not built: call zbc_matvec or zbc_rmatvec on it once first");
    return ZBC_EINVAL;
  }
  if (p == 1) return launch_rmatvec_scratch<1>(h, Phi, ldphi, p, out, ldo, scratch, scratch_bytes, st);
  if (p == 2) return launch_rmatvec_scratch<2>(h, Phi, ldphi, p, out, ldo, scratch, scratch_bytes, st);
  if (p <= 4) return launch_rmatvec_scratch<4>(h, Phi, ldphi, p, out, ldo, scratch, scratch_bytes, st);
  if (p <= 8) return launch_rmatvec_scratch<8>(h, Phi, ldphi, p, out, ldo, scratch, scratch_bytes, st);
  return launch_rmatvec_scratch<16>(h, Phi, ldphi, p, out, ldo, scratch, scratch_bytes, st);
}

int matvec_simt(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  if (p == 1) return launch_matvec<1>(h, X, ldx, p, Y, ldy, st);
  if (p == 2) return launch_matvec<2>(h, X, ldx, p, Y, ldy, st);
  if (p <= 4) return launch_matvec<4>(h, X, ldx, p, Y, ldy, st);
  if (p <= 8) return launch_matvec<8>(h, X, ldx, p, Y, ldy, st);
  return launch_matvec<16>(h, X, ldx, p, Y, ldy, st);
}

int rmatvec_simt(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo, cudaStream_t st) {
  if (p == 1) return launch_rmatvec<1>(h, Phi, ldphi, p, out, ldo, st);
  if (p == 2) return launch_rmatvec<2>(h, Phi, ldphi, p, out, ldo, st);
  if (p <= 4) return launch_rmatvec<4>(h, Phi, ldphi, p, out, ldo, st);
  if (p <= 8) return launch_rmatvec<8>(h, Phi, ldphi, p, out, ldo, st);
  return launch_rmatvec<16>(h, Phi, ldphi, p, out, ldo, st);
}

}  // namespace zbc
