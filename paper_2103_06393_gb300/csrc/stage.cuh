// Bulk-copy stage pipeline that feeds the product kernels' decompression front end
// (Sec. III.B, Algorithms 1 and 2).
//
// A work item is one stored column j on one voxel tile (B1 i1 x NU i2 at one i3).  Its inputs
// are three contiguous runs of the decompression cache and of the right-hand sides:
//   the U1_j block of the i1 tile   [a][i1 local]  r1p x B1p complex64
//   the W_j block of the tile       [u][a]         nu  x r1p complex64 (nu = valid i2 rows)
//   (forward) X^T[j][s0 .. s0+P)                    P complex64
// One producer lane moves them to shared memory with cp.async.bulk, completing on the stage's
// "full" mbarrier (transaction bytes); the consumer warps read them from there and each
// arrives on the stage's "empty" mbarrier when done, which hands the stage back to the
// producer.  kMaxStages stages rotate, so the copies of the next items overlap the arithmetic
// of the current one and no CTA-wide barrier is taken per column.
//
// Every wait is bounded; a wait that gives up sets the CTA's abort flag, after which nobody
// waits or copies any more, and the kernel reports the failure through an error word.
#pragma once

#include "decomp.cuh"
#include "tc_common.cuh"

namespace zbc {

constexpr int kMaxStages = 8;

// X^T (M rows of pst >= p complex64, zero padded to a whole number of `chunk`-wide RHS chunks,
// pst even) in the handle's workspace, so that a column's RHS values are one aligned run
int transpose_rhs(Handle& h, const float2* X, int64_t ldx, int p, int chunk, const float2** XT, int* pst,
                  cudaStream_t st);

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(mbar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive1(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(mbar)) : "memory");
}

// global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc::smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(tc::smem_u32(mbar))
      : "memory");
}

// byte layout of one stage: [U1 R x B1p][W NUp x R][X xb][red rb], each a multiple of 16 bytes
struct StageLayout {
  uint32_t u1, w, x, red, stride;
  __host__ __device__ static uint32_t r16(uint32_t b) { return (b + 15u) / 16u * 16u; }
  __host__ __device__ static StageLayout make(int R, int B1p, int NUp, int xbytes, int redbytes) {
    StageLayout s;
    s.u1 = 0;
    s.w = s.u1 + r16(8u * R * B1p);
    s.x = s.w + r16(8u * NUp * R);
    s.red = s.x + r16((uint32_t)xbytes);
    s.stride = (s.red + r16((uint32_t)redbytes) + 127u) / 128u * 128u;
    return s;
  }
};

// Last mode product of one column for kUQ voxels sharing i1, from the staged blocks:
//   z[l] = sum_a U1s[a][il] Ws[u0 + l][a],  a < r1p (the pad entries are zero)
// Even and odd a accumulate in separate chains (twice the independent FMAs in flight) and the
// next a-pair's operands are loaded before the current pair's FMAs.
__device__ __forceinline__ void last_mode_staged(const float2* U1s, int B1p, int il, const float2* Ws, int r1p,
                                                 int u0, float2 (&z)[kUQ]) {
  float2 ze[kUQ], zo[kUQ];
#pragma unroll
  for (int l = 0; l < kUQ; ++l) ze[l] = zo[l] = make_float2(0.f, 0.f);
  const float2* u = U1s + il;
  const float4* w4 = reinterpret_cast<const float4*>(Ws + u0 * r1p);
  const int ws = r1p / 2;  // float4 stride between consecutive u
  float2 x0 = u[0], x1 = u[B1p];
  float4 w[kUQ];
#pragma unroll
  for (int l = 0; l < kUQ; ++l) w[l] = w4[l * ws];
  for (int a = 0; a < r1p; a += 2) {
    const bool more = a + 2 < r1p;
    const int an = more ? a + 2 : a;
    const float2 nx0 = u[an * B1p], nx1 = u[(an + 1) * B1p];
    float4 nw[kUQ];
#pragma unroll
    for (int l = 0; l < kUQ; ++l) nw[l] = w4[l * ws + an / 2];
#pragma unroll
    for (int l = 0; l < kUQ; ++l) {
      ze[l] = cfma(x0, make_float2(w[l].x, w[l].y), ze[l]);
      zo[l] = cfma(x1, make_float2(w[l].z, w[l].w), zo[l]);
    }
    x0 = nx0;
    x1 = nx1;
#pragma unroll
    for (int l = 0; l < kUQ; ++l) w[l] = nw[l];
  }
#pragma unroll
  for (int l = 0; l < kUQ; ++l) z[l] = make_float2(ze[l].x + zo[l].x, ze[l].y + zo[l].y);
}

// Producer side: issue the copies of item (column j, tile origin i1_0, i2_0, i3) into stage st.
// Called by one lane.  x_src may be null (adjoint).  Returns the bytes in flight.
__device__ __forceinline__ void issue_item(unsigned char* stage, const StageLayout& L, uint64_t* full, int* meta,
                                           const float2* __restrict__ cache, const CacheDesc& d, const Geo& g,
                                           int B1p, int i1_0, int i2_0, int i3, const float2* x_src,
                                           uint32_t xbytes) {
  const int nu = min(g.NU, g.n2 - i2_0);
  const uint32_t ub = 8u * d.r1p * B1p, wb = 8u * nu * d.r1p;
  *meta = d.r1p;
  mbar_arrive_expect_tx(full, ub + wb + (x_src ? xbytes : 0u));
  const int t1 = i1_0 / g.B1;
  bulk_g2s(stage + L.u1, cache + d.uoff + (int64_t)t1 * d.r1p * B1p, ub, full);
  bulk_g2s(stage + L.w, cache + d.woff + ((int64_t)i3 * g.n2 + i2_0) * d.r1p, wb, full);
  if (x_src) bulk_g2s(stage + L.x, x_src, xbytes, full);
}

}  // namespace zbc
