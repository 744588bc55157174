// Chunked decompression front end shared by the product kernels (Sec. III.B, Eq. Tucker).
//
// A CTA owns a voxel tile of B1 (i1) x NU (i2) voxels at one i3 and walks the stored
// columns j in chunks of JC.  For every column of a chunk it forms, in shared memory,
//   P_j[a][b] = sum_c G_j[a,b,c] U3_j[i3,c]          (core x3 one factor row)
//   W_j[a][u] = sum_b P_j[a][b] U2_j[i2_0+u, b]       (x2 the tile's U2 rows)
// so that the last mode product Z[i1,u,j] = sum_a U1_j[i1,a] W_j[a][u] costs r1 complex MACs
// per voxel and column; the core contraction is amortised over the whole B1 x NU tile.
// Threads are laid out as lane groups: lane group g covers 32 consecutive i1 at one u.
#pragma once

#include "zbc_internal.cuh"

namespace zbc {

constexpr int kChunk = 8;      // columns per chunk
constexpr int kThreads = 256;  // threads per CTA
constexpr int kMaxLG = 4;      // lane groups per warp (register arrays)

struct Geo {
  int n1, n2, n3;
  int B1, NU;      // tile extent along i1 and i2
  int nb1, nb2;    // tiles along i1 and i2
  int nb32;        // 32-wide i1 groups per tile
  int nlg;         // lane groups per tile = nb32 * NU
  __host__ __device__ int ntiles() const { return nb1 * nb2 * n3; }
  __device__ __forceinline__ void tile(int t, int& i1_0, int& i2_0, int& i3) const {
    i1_0 = (t % nb1) * B1;
    i2_0 = ((t / nb1) % nb2) * NU;
    i3 = t / (nb1 * nb2);
  }
  // voxel of lane group g, lane l; returns false for padding voxels
  __device__ __forceinline__ bool voxel(int i1_0, int i2_0, int g, int l, int& i1, int& u) const {
    i1 = i1_0 + 32 * (g % nb32) + l;
    u = g / nb32;
    return g < nlg && i1 < n1 && (i1 - i1_0) < B1 && (i2_0 + u) < n2;
  }
};

// NU chosen so that every warp holds at most kMaxLG lane groups (and, for the tensor-core
// kernels, the accumulator rows fit the caller's limit max_rows).
inline Geo make_geo(int n1, int n2, int n3, int max_rows = 1 << 30) {
  Geo g;
  g.n1 = n1;
  g.n2 = n2;
  g.n3 = n3;
  g.B1 = n1 < 128 ? n1 : 128;
  g.nb32 = (g.B1 + 31) / 32;
  int lg_cap = 8 * kMaxLG;
  if (lg_cap * 32 > max_rows) lg_cap = max_rows / 32;
  int nu = lg_cap / g.nb32;
  if (nu < 1) nu = 1;
  if (nu > n2) nu = n2;
  g.NU = nu;
  g.nlg = g.nb32 * nu;
  g.nb1 = (n1 + g.B1 - 1) / g.B1;
  g.nb2 = (n2 + nu - 1) / nu;
  return g;
}

struct ChunkSmem {
  float2* P;        // [kChunk][R*R]
  float2* W;        // [kChunk][R][NU]
  TensorDesc* jd;   // [kChunk]
  static size_t bytes(int R, int NU) {
    return sizeof(float2) * ((size_t)kChunk * R * R + (size_t)kChunk * R * NU) + sizeof(TensorDesc) * kChunk;
  }
  __device__ __forceinline__ unsigned char* carve(unsigned char* base, int R, int NU) {
    P = (float2*)base;
    W = P + (size_t)kChunk * R * R;
    jd = (TensorDesc*)(W + (size_t)kChunk * R * NU);
    return (unsigned char*)(jd + kChunk);
  }
};

// Steps P and W for columns j0 .. j0+jc-1 of component k (jc <= kChunk).  Ends with the W
// values visible to all threads (two __syncthreads).
__device__ __forceinline__ void chunk_pw(const float2* __restrict__ pool, const TensorDesc* __restrict__ desc,
                                         const Geo& g, int q, int k, int j0, int jc, int R, int i2_0, int i3,
                                         const ChunkSmem& s) {
  if (threadIdx.x < jc) s.jd[threadIdx.x] = desc[(int64_t)(j0 + threadIdx.x) * q + k];
  __syncthreads();
  const int RR = R * R;
  for (int o = threadIdx.x; o < jc * RR; o += blockDim.x) {
    const int jj = o / RR, ab = o % RR;
    const TensorDesc d = s.jd[jj];
    const int a = ab % R, b = ab / R;
    if (a >= d.r1 || b >= d.r2) continue;
    const float2* G = pool + d.off;
    const float2* U3 = G + (int64_t)d.r1 * d.r2 * d.r3 + (int64_t)g.n1 * d.r1 + (int64_t)g.n2 * d.r2;
    float2 acc = make_float2(0.f, 0.f);
    const int64_t st = (int64_t)d.r1 * d.r2;
    for (int c = 0; c < d.r3; ++c) acc = cfma(__ldg(G + a + d.r1 * b + st * c), __ldg(U3 + i3 + (int64_t)g.n3 * c), acc);
    s.P[jj * RR + a * R + b] = acc;
  }
  __syncthreads();
  const int RN = R * g.NU;
  for (int o = threadIdx.x; o < jc * RN; o += blockDim.x) {
    const int jj = o / RN, rem = o % RN;
    const int u = rem % g.NU, a = rem / g.NU;
    const TensorDesc d = s.jd[jj];
    if (a >= d.r1) continue;
    float2 acc = make_float2(0.f, 0.f);
    if (i2_0 + u < g.n2) {
      const float2* U2 = pool + d.off + (int64_t)d.r1 * d.r2 * d.r3 + (int64_t)g.n1 * d.r1;
      for (int b = 0; b < d.r2; ++b) acc = cfma(s.P[jj * RR + a * R + b], __ldg(U2 + (i2_0 + u) + (int64_t)g.n2 * b), acc);
    }
    s.W[(jj * R + a) * g.NU + u] = acc;
  }
  __syncthreads();
}

// Last mode product for one column: z = sum_a U1[i1, a] W[a][u]
__device__ __forceinline__ float2 last_mode(const float2* __restrict__ U1, int n1, int r1, int i1, const float2* Wj,
                                            int R, int NU, int u) {
  float2 z = make_float2(0.f, 0.f);
  for (int a = 0; a < r1; ++a) z = cfma(__ldg(U1 + i1 + (int64_t)n1 * a), Wj[a * NU + u], z);
  return z;
}

}  // namespace zbc
