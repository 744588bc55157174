// Plain complex-FP32 forms of Algorithm 1 (Y = Z X) and Algorithm 2 (Psi = Z^H Phi) on CUDA
// cores (Sec. III.B), plus the ACA pre/post products X' = V^H X and Psi = V Psi'.
//
// A CTA owns a voxel tile of 32 (i1) x 8 (i2) x 2 (i3) = 512 voxels of one component k and
// walks all stored columns j.  For each j it decompresses the tile in shared memory,
// contracting the core with U3 first, then U2, then U1 (i1 last, so a warp's 32 lanes hold
// 32 consecutive voxels and the stores of Y are coalesced):
//   P[a,b,i3] = sum_c G[a,b,c] U3[i3,c];  W[a,i2,i3] = sum_b P[a,b,i3] U2[i2,b];
//   Z[i1,i2,i3] = sum_a U1[i1,a] W[a,i2,i3]
// and then either accumulates Y^k[v,s] += Z[v] X[j,s] in registers (Algorithm 1) or reduces
// sum_v conj(Z[v]) Phi^k[v,s] over the tile (Algorithm 2).  The decompressed column never
// reaches HBM.
#include <algorithm>

#include "zbc_internal.cuh"

namespace zbc {

constexpr int TB1 = 32, TB2 = 8, TB3 = 2;
constexpr int NPAIR = TB2 * TB3;  // (i2,i3) pairs per tile = 16; a thread owns pairs w and w+8

struct TileGeom {
  int n1, n2, n3, t1, t2, t3;  // tiles per axis
  __device__ __forceinline__ void tile(int idx, int& b1, int& b2, int& b3) const {
    b1 = (idx % t1) * TB1;
    b2 = ((idx / t1) % t2) * TB2;
    b3 = (idx / (t1 * t2)) * TB3;
  }
};

// shared-memory layout for one column j of the tile (RMAX = largest rank in the handle)
struct SimtSmem {
  float2* u1;  // [RMAX][32]
  float2* u2;  // [RMAX][8]
  float2* u3;  // [RMAX][2]
  float2* P;   // [RMAX][RMAX][2]
  float2* W;   // [RMAX][16]
  float2* xs;  // [32]
  __device__ static size_t bytes(int R) {
    return sizeof(float2) * ((size_t)R * 32 + R * 8 + R * 2 + (size_t)R * R * 2 + R * 16 + 32);
  }
  __device__ __forceinline__ void carve(unsigned char* base, int R) {
    u1 = (float2*)base;
    u2 = u1 + R * 32;
    u3 = u2 + R * 8;
    P = u3 + R * 2;
    W = P + R * R * 2;
    xs = W + R * 16;
  }
};
static size_t simt_smem_bytes(int R) {
  return sizeof(float2) * ((size_t)R * 32 + R * 8 + R * 2 + (size_t)R * R * 2 + R * 16 + 32);
}

// Decompress the tile of tensor d into z0 (pair w) and z1 (pair w+8) of this thread.
// Precondition: u1/u2/u3 loaded for this tensor.  Contains two __syncthreads.
__device__ __forceinline__ void decompress_tile(const float2* __restrict__ G, const TensorDesc& d,
                                                const SimtSmem& s, int lane, int warp, float2& z0,
                                                float2& z1) {
  const int r1 = d.r1, r2 = d.r2, r3 = d.r3;
  // P[a][b][l3] = sum_c G[a + r1(b + r2 c)] U3[l3][c]
  const int np = r1 * r2 * TB3;
  for (int o = threadIdx.x; o < np; o += blockDim.x) {
    const int l3 = o % TB3, ab = o / TB3;
    const int a = ab % r1, b = ab / r1;
    float2 acc = make_float2(0.f, 0.f);
    const float2* g = G + a + r1 * b;
    for (int c = 0; c < r3; ++c) acc = cfma(__ldg(g + (int64_t)r1 * r2 * c), s.u3[c * TB3 + l3], acc);
    s.P[(a * r2 + b) * TB3 + l3] = acc;
  }
  __syncthreads();
  // W[a][pair] = sum_b P[a][b][l3] U2[l2][b], pair = l2 + 8*l3
  const int nw = r1 * NPAIR;
  for (int o = threadIdx.x; o < nw; o += blockDim.x) {
    const int pair = o % NPAIR, a = o / NPAIR;
    const int l2 = pair % TB2, l3 = pair / TB2;
    float2 acc = make_float2(0.f, 0.f);
    for (int b = 0; b < r2; ++b) acc = cfma(s.P[(a * r2 + b) * TB3 + l3], s.u2[b * TB2 + l2], acc);
    s.W[a * NPAIR + pair] = acc;
  }
  __syncthreads();
  float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
  for (int a = 0; a < r1; ++a) {
    const float2 u = s.u1[a * TB1 + lane];
    a0 = cfma(u, s.W[a * NPAIR + warp], a0);
    a1 = cfma(u, s.W[a * NPAIR + warp + 8], a1);
  }
  z0 = a0;
  z1 = a1;
}

__device__ __forceinline__ void load_factors(const float2* __restrict__ base, const TensorDesc& d, int n1,
                                             int n2, int n3, int b1, int b2, int b3, const SimtSmem& s) {
  const float2* U1 = base + (int64_t)d.r1 * d.r2 * d.r3;
  const float2* U2 = U1 + (int64_t)n1 * d.r1;
  const float2* U3 = U2 + (int64_t)n2 * d.r2;
  for (int e = threadIdx.x; e < d.r1 * TB1; e += blockDim.x) {
    const int l = e % TB1, a = e / TB1;
    s.u1[a * TB1 + l] = (b1 + l < n1) ? __ldg(U1 + (b1 + l) + (int64_t)n1 * a) : make_float2(0.f, 0.f);
  }
  for (int e = threadIdx.x; e < d.r2 * TB2; e += blockDim.x) {
    const int l = e % TB2, b = e / TB2;
    s.u2[b * TB2 + l] = (b2 + l < n2) ? __ldg(U2 + (b2 + l) + (int64_t)n2 * b) : make_float2(0.f, 0.f);
  }
  for (int e = threadIdx.x; e < d.r3 * TB3; e += blockDim.x) {
    const int l = e % TB3, c = e / TB3;
    s.u3[c * TB3 + l] = (b3 + l < n3) ? __ldg(U3 + (b3 + l) + (int64_t)n3 * c) : make_float2(0.f, 0.f);
  }
}

// ---------------------------------------------------------------------------------------------
// Algorithm 1
// ---------------------------------------------------------------------------------------------
template <int PS>
__global__ void __launch_bounds__(256, 2)
    matvec_simt_kernel(const float2* __restrict__ pool, const TensorDesc* __restrict__ desc, TileGeom tg, int q,
                       int M, int R, const float2* __restrict__ X, int64_t ldx, int p, float2* __restrict__ Y,
                       int64_t ldy) {
  extern __shared__ __align__(16) unsigned char smem[];
  SimtSmem s;
  s.carve(smem, R);
  const int k = blockIdx.y;
  const int s0 = blockIdx.z * PS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int b1, b2, b3;
  tg.tile(blockIdx.x, b1, b2, b3);
  float2 acc0[PS], acc1[PS];
#pragma unroll
  for (int i = 0; i < PS; ++i) acc0[i] = acc1[i] = make_float2(0.f, 0.f);
  for (int j = 0; j < M; ++j) {
    const TensorDesc d = desc[(int64_t)j * q + k];
    const float2* base = pool + d.off;
    load_factors(base, d, tg.n1, tg.n2, tg.n3, b1, b2, b3, s);
    if (threadIdx.x < PS) s.xs[threadIdx.x] = (s0 + threadIdx.x < p) ? X[j + ldx * (s0 + threadIdx.x)] : make_float2(0.f, 0.f);
    __syncthreads();
    float2 z0, z1;
    decompress_tile(base, d, s, lane, warp, z0, z1);
#pragma unroll
    for (int i = 0; i < PS; ++i) {
      const float2 x = s.xs[i];
      acc0[i] = cfma(z0, x, acc0[i]);
      acc1[i] = cfma(z1, x, acc1[i]);
    }
    __syncthreads();
  }
  const int64_t nv = (int64_t)tg.n1 * tg.n2 * tg.n3;
  const int i1 = b1 + lane;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int pair = warp + 8 * h;
    const int i2 = b2 + pair % TB2, i3 = b3 + pair / TB2;
    if (i1 < tg.n1 && i2 < tg.n2 && i3 < tg.n3) {
      const int64_t v = i1 + (int64_t)tg.n1 * (i2 + (int64_t)tg.n2 * i3);
      float2* y = Y + k * nv + v;
#pragma unroll
      for (int i = 0; i < PS; ++i)
        if (s0 + i < p) y[ldy * (s0 + i)] = h == 0 ? acc0[i] : acc1[i];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// warp reduce-scatter of NV floats per lane: afterwards lane l holds the warp sum of value index
// (l >> (5 - log2 NV)); 31 shuffles for NV = 32 instead of 160 for independent butterflies.
// ---------------------------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[NV], int lane) {
  constexpr int LOG = NV == 1 ? 0 : NV == 2 ? 1 : NV == 4 ? 2 : NV == 8 ? 3 : NV == 16 ? 4 : 5;
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
// Algorithm 2: partial sums per (tile group g, component k): partial[(g*q+k)][s][j] (M x p)
// ---------------------------------------------------------------------------------------------
template <int PS>
__global__ void __launch_bounds__(256, 2)
    rmatvec_simt_kernel(const float2* __restrict__ pool, const TensorDesc* __restrict__ desc, TileGeom tg, int q,
                        int M, int R, int MJ, const float2* __restrict__ Phi, int64_t ldphi, int p,
                        float2* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem[];
  SimtSmem s;
  s.carve(smem, R);
  float* red = (float*)(s.xs + 32);          // [8][2*PS]
  float* pacc = red + 8 * 2 * PS;            // [MJ][2*PS]
  const int k = blockIdx.y % q;
  const int j0 = (blockIdx.y / q) * MJ;
  const int j1 = min(M, j0 + MJ);
  const int s0 = blockIdx.z * PS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntiles = tg.t1 * tg.t2 * tg.t3;
  const int64_t nv = (int64_t)tg.n1 * tg.n2 * tg.n3;
  for (int e = threadIdx.x; e < (j1 - j0) * 2 * PS; e += blockDim.x) pacc[e] = 0.f;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int b1, b2, b3;
    tg.tile(tile, b1, b2, b3);
    float2 ph0[PS], ph1[PS];
    {
      const int i1 = b1 + lane;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int pair = warp + 8 * h;
        const int i2 = b2 + pair % TB2, i3 = b3 + pair / TB2;
        const bool ok = i1 < tg.n1 && i2 < tg.n2 && i3 < tg.n3;
        const int64_t v = i1 + (int64_t)tg.n1 * (i2 + (int64_t)tg.n2 * i3);
#pragma unroll
        for (int i = 0; i < PS; ++i) {
          const float2 val = (ok && s0 + i < p) ? Phi[k * nv + v + ldphi * (s0 + i)] : make_float2(0.f, 0.f);
          if (h == 0) ph0[i] = val; else ph1[i] = val;
        }
      }
    }
    for (int j = j0; j < j1; ++j) {
      const TensorDesc d = desc[(int64_t)j * q + k];
      const float2* base = pool + d.off;
      load_factors(base, d, tg.n1, tg.n2, tg.n3, b1, b2, b3, s);
      __syncthreads();
      float2 z0, z1;
      decompress_tile(base, d, s, lane, warp, z0, z1);
      float vals[2 * PS];
#pragma unroll
      for (int i = 0; i < PS; ++i) {
        float2 a = cfma_conj(z0, ph0[i], make_float2(0.f, 0.f));
        a = cfma_conj(z1, ph1[i], a);
        vals[2 * i] = a.x;
        vals[2 * i + 1] = a.y;
      }
      const float r = warp_reduce_scatter<2 * PS>(vals, lane);
      constexpr int SH = 5 - (2 * PS == 1 ? 0 : 2 * PS == 2 ? 1 : 2 * PS == 4 ? 2 : 2 * PS == 8 ? 3 : 2 * PS == 16 ? 4 : 5);
      if ((lane & ((1 << SH) - 1)) == 0) red[warp * 2 * PS + (lane >> SH)] = r;
      __syncthreads();
      if (threadIdx.x < 2 * PS) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += red[w * 2 * PS + threadIdx.x];
        pacc[(j - j0) * 2 * PS + threadIdx.x] += t;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  float2* out = partial + (int64_t)(blockIdx.x * q + k) * M * p;
  for (int e = threadIdx.x; e < (j1 - j0) * PS; e += blockDim.x) {
    const int jl = e % (j1 - j0), i = e / (j1 - j0);
    if (s0 + i < p) out[(j0 + jl) + (int64_t)M * (s0 + i)] = make_float2(pacc[jl * 2 * PS + 2 * i], pacc[jl * 2 * PS + 2 * i + 1]);
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

// out (ncol x p) = op(V) * B:  conj=1 -> V^H B (V is m x M, out M x p); conj=0 -> V B (out m x p)
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

static TileGeom make_geom(const Handle& h) {
  TileGeom tg;
  tg.n1 = h.n1;
  tg.n2 = h.n2;
  tg.n3 = h.n3;
  tg.t1 = ceil_div(h.n1, TB1);
  tg.t2 = ceil_div(h.n2, TB2);
  tg.t3 = ceil_div(h.n3, TB3);
  return tg;
}

template <int PS>
static int launch_matvec(const Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  TileGeom tg = make_geom(h);
  const int R = std::max(h.max_rank, 1);
  const size_t sm = simt_smem_bytes(R);
  static bool attr_set = false;
  if (!attr_set) {
    ZBC_TRY_CUDA(cudaFuncSetAttribute(matvec_simt_kernel<PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  dim3 grid(tg.t1 * tg.t2 * tg.t3, h.q, ceil_div(p, PS));
  matvec_simt_kernel<PS><<<grid, 256, sm, st>>>(h.d_pool, h.d_desc, tg, h.q, h.M, R, X, ldx, p, Y, ldy);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

template <int PS>
static int launch_rmatvec(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo,
                          cudaStream_t st) {
  TileGeom tg = make_geom(h);
  const int R = std::max(h.max_rank, 1);
  const int ntiles = tg.t1 * tg.t2 * tg.t3;
  // j-chunk so that the per-CTA accumulator stays within ~96 KB of shared memory
  const int MJ = std::max(1, std::min(h.M, (96 * 1024) / (int)(2 * PS * sizeof(float))));
  const int jchunks = ceil_div(h.M, MJ);
  const int schunks = ceil_div(p, PS);
  const int target = 4 * sm_count();
  int G = std::max(1, target / std::max(1, h.q * jchunks * schunks));
  G = std::min(G, ntiles);
  const size_t sm = simt_smem_bytes(R) + sizeof(float) * (8 * 2 * PS + (size_t)MJ * 2 * PS);
  static bool attr_set = false;
  if (!attr_set) {
    ZBC_TRY_CUDA(cudaFuncSetAttribute(rmatvec_simt_kernel<PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    attr_set = true;
  }
  ZBC_CHECK_ARG(sm <= 220 * 1024, "rank %d too large for the FP32 SIMT adjoint", R);
  ZBC_TRY(h.work_partial.ensure(sizeof(float2) * (size_t)G * h.q * h.M * p));
  float2* partial = (float2*)h.work_partial.ptr;
  dim3 grid(G, h.q * jchunks, schunks);
  rmatvec_simt_kernel<PS><<<grid, 256, sm, st>>>(h.d_pool, h.d_desc, tg, h.q, h.M, R, MJ, Phi, ldphi, p, partial);
  ZBC_TRY_CUDA(cudaGetLastError());
  reduce_partials_kernel<<<ceil_div((int64_t)h.M * p, 256), 256, 0, st>>>(partial, G * h.q, h.M, p, out, ldo);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch(2);
  return ZBC_OK;
}

int matvec_simt(const Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  if (h.max_rank > 64) {
    set_error("FP32 SIMT path supports ranks up to 64 (max rank %d)", h.max_rank);
    return ZBC_EINVAL;
  }
  if (p == 1) return launch_matvec<1>(h, X, ldx, p, Y, ldy, st);
  if (p == 2) return launch_matvec<2>(h, X, ldx, p, Y, ldy, st);
  if (p <= 4) return launch_matvec<4>(h, X, ldx, p, Y, ldy, st);
  if (p <= 8) return launch_matvec<8>(h, X, ldx, p, Y, ldy, st);
  return launch_matvec<16>(h, X, ldx, p, Y, ldy, st);
}

int rmatvec_simt(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo, cudaStream_t st) {
  if (h.max_rank > 64) {
    set_error("FP32 SIMT path supports ranks up to 64 (max rank %d)", h.max_rank);
    return ZBC_EINVAL;
  }
  if (p == 1) return launch_rmatvec<1>(h, Phi, ldphi, p, out, ldo, st);
  if (p == 2) return launch_rmatvec<2>(h, Phi, ldphi, p, out, ldo, st);
  if (p <= 4) return launch_rmatvec<4>(h, Phi, ldphi, p, out, ldo, st);
  if (p <= 8) return launch_rmatvec<8>(h, Phi, ldphi, p, out, ldo, st);
  return launch_rmatvec<16>(h, Phi, ldphi, p, out, ldo, st);
}

}  // namespace zbc
