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

constexpr int kChunk = 8;      // columns per chunk of the tensor-core contraction
constexpr int kUQ = 4;         // u values per task
constexpr int kRmax = 64;      // largest rank r1 the product kernels accept

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

// Tile geometry: B1 i1 rows (tile_b1) times NU i2 values, tasks of 32 i1 x kUQ u, at most
// max_tasks tasks and max_rows rows (R is unused and kept for the callers' signature).
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

// U1 as the A operand of the tensor-core mode product (products_tc2.cu): per tensor and i1 tile,
// two fp16 terms (hi, lo = x - hi) of the real embedding A1[i1][2a + e] = (Re, Im) U1[i1, a],
// K padded to Kp1 = 8 kb1 (a multiple of 16), in the K-major core-matrix layout of tc_common.cuh
// (rows grouped by 8, SBO = kb1 * 128); only the first RG = ceil(B1 / 8) row groups are stored.
// Both fp16 operands are brought to magnitudes below 2^kHalfShift by powers of two (U1 by
// 2^(kHalfShift - uexp), |U1| < 2^uexp; W by 2^(kHalfShift - wexp), |W| < 2^wexp) so that
// their lo terms (~2^-11 of the value) stay normal fp16 numbers; products carry
// 2^(2 kHalfShift - uexp - wexp), removed exactly from the FP32 result.
constexpr int kHalfShift = 10;

struct HalfDesc {
  int64_t off;  // bytes into the fp16 block array: [t1][term][RG row groups][kb1 chunks][8 rows][16 B]
  int kb1;      // 16-byte K chunks per row (even)
  int wexp;     // |W| < 2^wexp
  int uexp;     // |U1| < 2^uexp (set on the device by the cache build)
};

struct Mode1Cache;  // operands of the mode-1 adjoint (products_mode1.cu), built on its first use
void mode1_release(Mode1Cache* c);

struct DcCache;
void dc_release(DcCache* c);
int64_t dc_bytes(const DcCache* c);

struct DecompCache {
  float2* data = nullptr;   // W blocks and tile-blocked U1
  CacheDesc* d_desc = nullptr;
  std::vector<CacheDesc> host_desc;
  int64_t elems = 0;
  unsigned char* half = nullptr;  // fp16 U1 operand blocks (built on first use of the chained path)
  HalfDesc* d_half = nullptr;
  int kb1_max = 0;
  Mode1Cache* mode1 = nullptr;
  DcCache* dc = nullptr;    // operands of the decompress-and-contract tensor-core forward (products_dc.cu)
  int64_t bytes = 0;        // device bytes held (W, U1, descriptors, fp16 copies; not mode1's)
  int64_t half_bytes = 0;   // the part of bytes held by half / d_half
};
int build_decomp_cache(Handle& h, cudaStream_t st);
int build_half_cache(Handle& h, cudaStream_t st);
void half_release(DecompCache* c);         // the fp16 U1 blocks (rebuilt on the next use)
void mode1_fwd_release(Mode1Cache* c);     // the mode-1 forward's operands (rebuilt on the next use)
void dc_release(DcCache* c);

}  // namespace zbc
