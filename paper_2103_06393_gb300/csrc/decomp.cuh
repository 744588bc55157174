// Chunked decompression front end shared by the product kernels (Sec. III.B, Eq. Tucker).
//
// A CTA owns a voxel tile of B1 (i1) x NU (i2) voxels at one i3 and walks the stored
// columns j in chunks of kChunk.  For every column of a chunk it forms, in shared memory,
//   P_j[a][b] = sum_c G_j[a,b,c] U3_j[i3,c]          (core x3 one factor row)
//   W_j[a][u] = sum_b P_j[a][b] U2_j[i2_0+u, b]       (x2 the tile's U2 rows)
// so that the last mode product Z[i1,u,j] = sum_a U1_j[i1,a] W_j[a][u] costs r1 complex MACs
// per voxel and column; the core contraction is amortised over the whole B1 x NU tile.
// Work is split into tasks: a task is 32 consecutive i1 (one per lane) times kUQ consecutive u,
// so each U1 row a thread loads serves kUQ voxels.
#pragma once

#include "zbc_internal.cuh"

namespace zbc {

constexpr int kChunk = 8;      // columns per chunk
constexpr int kThreads = 256;  // threads per CTA
constexpr int kUQ = 4;         // u values per task

struct Geo {
  int n1, n2, n3;
  int B1, NU, NUp;  // tile extent along i1 and i2 (NUp = NU rounded up to kUQ)
  int nb1, nb2;     // tiles along i1 and i2
  int nb32;         // 32-wide i1 groups per tile
  int ntask;        // tasks per tile = nb32 * NUp / kUQ
  __host__ __device__ int ntiles() const { return nb1 * nb2 * n3; }
  __device__ __forceinline__ void tile(int t, int& i1_0, int& i2_0, int& i3) const {
    i1_0 = (t % nb1) * B1;
    i2_0 = ((t / nb1) % nb2) * NU;
    i3 = t / (nb1 * nb2);
  }
  // task tk, lane l -> i1 and first u; ok_i1 false for padding lanes
  __device__ __forceinline__ void task(int i1_0, int tk, int l, int& i1, int& u0, bool& ok_i1) const {
    i1 = i1_0 + 32 * (tk % nb32) + l;
    u0 = (tk / nb32) * kUQ;
    ok_i1 = i1 < n1 && (i1 - i1_0) < B1;
  }
  // accumulator row of (task, lane, q) -- rows are grouped by 32 lanes
  __device__ __forceinline__ static int row(int tk, int q, int l) { return (tk * kUQ + q) * 32 + l; }
};

// NU chosen so that the tile has at most max_tasks tasks (and, for the tensor-core kernels,
// the accumulator rows ntask * kUQ * 32 stay within max_rows).
inline Geo make_geo(int n1, int n2, int n3, int max_tasks, int max_rows = 1 << 30) {
  Geo g;
  g.n1 = n1;
  g.n2 = n2;
  g.n3 = n3;
  g.B1 = n1 < 128 ? n1 : 128;
  g.nb32 = (g.B1 + 31) / 32;
  int tasks = max_tasks;
  if (tasks * kUQ * 32 > max_rows) tasks = max_rows / (kUQ * 32);
  int nq = tasks / g.nb32;
  if (nq < 1) nq = 1;
  int nu = nq * kUQ;
  const int n2r = (n2 + kUQ - 1) / kUQ * kUQ;
  if (nu > n2r) nu = n2r;
  g.NUp = nu;
  g.NU = nu < n2 ? nu : n2;
  g.ntask = g.nb32 * (g.NUp / kUQ);
  g.nb1 = (n1 + g.B1 - 1) / g.B1;
  g.nb2 = (n2 + g.NU - 1) / g.NU;
  return g;
}

struct ChunkSmem {
  float2* P;        // [kChunk][R*R]
  float2* W;        // [kChunk][R][NUp]
  TensorDesc* jd;   // [kChunk]
  static size_t bytes(int R, int NUp) {
    return sizeof(float2) * ((size_t)kChunk * R * R + (size_t)kChunk * R * NUp) + sizeof(TensorDesc) * kChunk;
  }
  __device__ __forceinline__ unsigned char* carve(unsigned char* base, int R, int NUp) {
    P = (float2*)base;
    W = P + (size_t)kChunk * R * R;
    jd = (TensorDesc*)(W + (size_t)kChunk * R * NUp);
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
  const int RN = R * g.NUp;
  for (int o = threadIdx.x; o < jc * RN; o += blockDim.x) {
    const int jj = o / RN, rem = o % RN;
    const int u = rem % g.NUp, a = rem / g.NUp;
    const TensorDesc d = s.jd[jj];
    float2 acc = make_float2(0.f, 0.f);
    if (a < d.r1 && u < g.NU && i2_0 + u < g.n2) {
      const float2* U2 = pool + d.off + (int64_t)d.r1 * d.r2 * d.r3 + (int64_t)g.n1 * d.r1;
      for (int b = 0; b < d.r2; ++b) acc = cfma(s.P[jj * RR + a * R + b], __ldg(U2 + (i2_0 + u) + (int64_t)g.n2 * b), acc);
    }
    s.W[(jj * R + a) * g.NUp + u] = acc;
  }
  __syncthreads();
}

// Last mode product of one column for kUQ voxels sharing i1:
//   z[q] = sum_a U1[i1, a] W[a][u0 + q]
__device__ __forceinline__ void last_mode4(const float2* __restrict__ U1, int n1, int r1, int i1, bool ok,
                                           const float2* Wj, int NUp, int u0, float2 (&z)[kUQ]) {
#pragma unroll
  for (int qq = 0; qq < kUQ; ++qq) z[qq] = make_float2(0.f, 0.f);
  if (!ok) return;
  const float4* w4 = reinterpret_cast<const float4*>(Wj + u0);
  const int stride4 = NUp / 2;
#pragma unroll 4
  for (int a = 0; a < r1; ++a) {
    const float2 x = __ldg(U1 + i1 + (int64_t)n1 * a);
    const float4 wa = w4[a * stride4], wb = w4[a * stride4 + 1];
    z[0] = cfma(x, make_float2(wa.x, wa.y), z[0]);
    z[1] = cfma(x, make_float2(wa.z, wa.w), z[1]);
    z[2] = cfma(x, make_float2(wb.x, wb.y), z[2]);
    z[3] = cfma(x, make_float2(wb.z, wb.w), z[3]);
  }
}

}  // namespace zbc
