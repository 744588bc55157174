// Decompression front end shared by the product kernels (Sec. III.B, Eq. Tucker).
//
// Z^{kj} = G x1 U1 x2 U2 x3 U3.  The partial product W_j = G_j x2 U2_j x3 U3_j (r1 x n2 x n3)
// does not depend on the right-hand sides, so a handle keeps it (and a copy of U1_j blocked by
// i1 tiles) in a device cache built once, on the first product call (decomp_cache.cu).  A
// product CTA then owns a voxel tile of B1 (i1) x NU (i2) voxels at one i3 and walks the stored
// columns, forming the last mode product
//   Z[i1, u, j] = sum_a U1_j[i1, a] W_j[a, i2_0 + u, i3]
// on CUDA cores.  A task is 32 consecutive i1 (one per lane) times kUQ consecutive u, so each
// U1 row a thread loads serves kUQ voxels.
//
// Cache layout per tensor (all offsets even, so every block starts on 16 bytes):
//   W  : [i3][i2][a], a < r1p (r1 rounded up to 2, the pad entry zero)
//   U1 : [t1][a][i1 - t1 B1], a < r1p, i1 row stride B1p (B1 rounded up to 2), zero padded
// so the U1 block of an i1 tile and the W block of an (i2 range, i3) are each one contiguous
// run that a single bulk copy moves to shared memory.
#pragma once

#include <algorithm>

#include "zbc_internal.cuh"

namespace zbc {

constexpr int kChunk = 8;      // columns per chunk
constexpr int kThreads = 256;  // threads per CTA
constexpr int kUQ = 4;         // u values per task
constexpr int kRmax = 32;      // largest rank r1 the product kernels accept
constexpr int kWPre = 8;       // W values each front-end thread prefetches per chunk

// per-tensor view of the decompression cache
struct CacheDesc {
  int64_t woff;   // W: [i3][i2][a] complex64, r1p per (i2, i3)
  int64_t uoff;   // U1: [t1][a][i1 local], r1p rows of B1p per i1 tile
  int r1, r1p;
};

// i1 tile extent: at most 128 rows (the 32-lane groups of four warps), balanced over the tiles
// so that the last tile is not mostly padding
__host__ __device__ inline int tile_b1(int n1) {
  const int nb1 = (n1 + 127) / 128;
  const int per = (n1 + nb1 - 1) / nb1;
  const int b1 = (per + 31) / 32 * 32;
  return n1 < b1 ? n1 : b1;
}
__host__ __device__ inline int tile_b1p(int n1) { return (tile_b1(n1) + 1) / 2 * 2; }

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
  __device__ __forceinline__ void task(int i1_0, int tk, int l, int& i1, int& u0, bool& ok_i1) const {
    i1 = i1_0 + 32 * (tk % nb32) + l;
    u0 = (tk / nb32) * kUQ;
    ok_i1 = i1 < n1 && (i1 - i1_0) < B1;
  }
  __device__ __forceinline__ static int row(int tk, int q, int l) { return (tk * kUQ + q) * 32 + l; }
};

// R = largest r1 of the handle (rounded up to 2): the chunk's W blocks (kChunk x R x NUp) must
// fit the register prefetch (kWPre values per thread).
inline Geo make_geo(int n1, int n2, int n3, int R, int max_tasks, int max_rows = 1 << 30) {
  Geo g;
  g.n1 = n1;
  g.n2 = n2;
  g.n3 = n3;
  g.B1 = tile_b1(n1);
  g.nb32 = (g.B1 + 31) / 32;
  int tasks = max_tasks;
  if (tasks * kUQ * 32 > max_rows) tasks = max_rows / (kUQ * 32);
  int nq = tasks / g.nb32;
  if (nq < 1) nq = 1;
  // the chunk's W blocks (kChunk x R x 4nq) must fit the register prefetch of the CTA's
  // 32 * max(4, ntask) front-end threads (R = 0: no register prefetch)
  while (R > 0 && nq > 1 && kChunk * R * kUQ * nq > kWPre * 32 * std::max(4, g.nb32 * nq)) --nq;
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

// shared memory of the front end: W[jj][a][NUp] (a < R) for one chunk, and the chunk's cache
// entries
struct ChunkSmem {
  float2* W;
  CacheDesc* cd;
  __host__ __device__ static size_t bytes(int R, int NUp) {
    return sizeof(float2) * (size_t)kChunk * R * NUp + sizeof(CacheDesc) * kChunk;
  }
  __device__ __forceinline__ unsigned char* carve(unsigned char* base, int R, int NUp) {
    W = (float2*)base;
    cd = (CacheDesc*)(W + (size_t)kChunk * R * NUp);
    return (unsigned char*)(cd + kChunk);
  }
};

// Two front-end buffers (chunk c uses buffer c & 1) with a per-chunk staging area of xn complex
// values after each, addressed arithmetically (no local-memory arrays of pointers).
struct FrontEnd2 {
  unsigned char* base;
  size_t stride;
  int R, NUp;
  __host__ __device__ static size_t buf_bytes(int R, int NUp, int xn) {
    return (ChunkSmem::bytes(R, NUp) + sizeof(float2) * (size_t)xn + 15) / 16 * 16;
  }
  __device__ __forceinline__ FrontEnd2(unsigned char* b, int R_, int NUp_, int xn)
      : base(b), stride(buf_bytes(R_, NUp_, xn)), R(R_), NUp(NUp_) {}
  __device__ __forceinline__ ChunkSmem cs(int b) const {
    ChunkSmem s;
    s.carve(base + b * stride, R, NUp);
    return s;
  }
  __device__ __forceinline__ float2* xs(int b) const {
    return (float2*)(base + b * stride + ChunkSmem::bytes(R, NUp));
  }
  __device__ __forceinline__ unsigned char* end() const { return base + 2 * stride; }
};

// Register prefetch of one chunk's W blocks: element e = (jj, a, u) of W[jj][a][NUp].
// Loaded one chunk ahead so the global-memory latency overlaps the current chunk's work.
// tid / nthr: this thread's index among the nthr threads that share the prefetch.
struct WPrefetch {
  float2 v[kWPre];
  CacheDesc cd;  // cache entry of column jj = tid (threads tid < kChunk)
  __device__ __forceinline__ void load(const float2* __restrict__ wc, const CacheDesc* __restrict__ cdesc,
                                       const Geo& g, int R, int q, int k, int j0, int jc, int i2_0, int i3, int tid,
                                       int nthr) {
    if (tid < jc) cd = cdesc[(int64_t)(j0 + tid) * q + k];
    const int per = R * g.NUp;
#pragma unroll
    for (int i = 0; i < kWPre; ++i) {
      const int e = tid + i * nthr;
      float2 x = make_float2(0.f, 0.f);
      if (e < kChunk * per) {
        const int jj = e / per, rem = e % per;
        const int a = rem / g.NUp, u = rem % g.NUp;
        if (jj < jc && u < g.NU && i2_0 + u < g.n2) {
          const CacheDesc d = cdesc[(int64_t)(j0 + jj) * q + k];
          if (a < d.r1) x = __ldg(wc + d.woff + ((int64_t)i3 * g.n2 + i2_0 + u) * d.r1p + a);
        }
      }
      v[i] = x;
    }
  }
  __device__ __forceinline__ void store(const ChunkSmem& s, const Geo& g, int R, int jc, int tid, int nthr) const {
    const int per = R * g.NUp;
#pragma unroll
    for (int i = 0; i < kWPre; ++i) {
      const int e = tid + i * nthr;
      if (e < kChunk * per) s.W[e] = v[i];
    }
    if (tid < jc) s.cd[tid] = cd;
  }
};

// Last mode product of one column for kUQ voxels sharing i1:
//   z[l] = sum_a U1_j[i1, a] W_j[a][u0 + l]
// u1 points at (a = 0, this lane's i1) of the cached U1 tile block (row stride B1p); all loads
// are issued before use.
__device__ __forceinline__ void last_mode4(const float2* __restrict__ u1, int B1p, int r1, bool ok, const float2* Wj,
                                           int NUp, int u0, float2 (&z)[kUQ]) {
#pragma unroll
  for (int l = 0; l < kUQ; ++l) z[l] = make_float2(0.f, 0.f);
  if (!ok) return;
  float2 ur[kRmax];
#pragma unroll
  for (int a = 0; a < kRmax; ++a)
    if (a < r1) ur[a] = __ldg(u1 + (int64_t)a * B1p);
  const float4* w4 = reinterpret_cast<const float4*>(Wj + u0);
  const int stride4 = NUp / 2;
#pragma unroll
  for (int i = 0; i < kRmax / 2; ++i) {
    if (2 * i >= r1) break;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int a = 2 * i + h;
      if (a >= r1) break;
      const float2 x = ur[a];
      const float4 wa = w4[a * stride4], wb = w4[a * stride4 + 1];
      z[0] = cfma(x, make_float2(wa.x, wa.y), z[0]);
      z[1] = cfma(x, make_float2(wa.z, wa.w), z[1]);
      z[2] = cfma(x, make_float2(wb.x, wb.y), z[2]);
      z[3] = cfma(x, make_float2(wb.z, wb.w), z[3]);
    }
  }
}

// the decompression cache of a handle (built by build_decomp_cache in decomp_cache.cu)
// U1 as the A operand of the tensor-core mode product (products_tc2.cu): per tensor and i1 tile,
// two fp16 terms (hi, lo = x - hi) of the real embedding A1[i1][2a + e] = (Re, Im) U1[i1, a],
// K padded to Kp1 = 8 kb1 (a multiple of 16), in the K-major core-matrix layout of tc_common.cuh
// (rows grouped by 8, SBO = kb1 * 128); only the first RG = ceil(B1 / 8) row groups are stored.
struct HalfDesc {
  int64_t off;  // bytes into the fp16 block array: [t1][term][RG row groups][kb1 chunks][8 rows][16 B]
  int kb1;      // 16-byte K chunks per row (even)
  int wexp;     // |W| < 2^wexp: W enters the fp16 operand scaled by 2^-wexp
};

struct DecompCache {
  float2* data = nullptr;   // W blocks and tile-blocked U1
  CacheDesc* d_desc = nullptr;
  int64_t elems = 0;
  unsigned char* half = nullptr;  // fp16 U1 operand blocks (built on first use of the chained path)
  HalfDesc* d_half = nullptr;
  int kb1_max = 0;
};
int build_decomp_cache(Handle& h, cudaStream_t st);
int build_half_cache(Handle& h, cudaStream_t st);

}  // namespace zbc
