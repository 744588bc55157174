// Algorithm 1 (Y = Z X, Sec. III.B) with both of its GEMM-shaped steps on the tensor cores:
//
//   1. the last mode product of the decompression, per stored column j and voxel tile,
//        Z[i1, u] = sum_a U1_j[i1, a] W_j[a, u]           (W = G x2 U2 x3 U3, cached)
//      as a tcgen05 MMA with M = 128 (i1), N = 16 (u = 0..7, Re / Im), K = 2 r1p (a, Re / Im)
//      padded to 16: the real embedding A1[i1][2a + e] = (Re, Im) U1, and
//        B1[2u][2a] = Re W, B1[2u][2a+1] = -Im W, B1[2u+1][2a] = Im W, B1[2u+1][2a+1] = Re W;
//      operands split into two fp16 terms (hi, lo = x - hi; products hh, hl, lh), U1 pre-split in
//      the handle's cache, W split per column and scaled by 2^-wexp (|W| < 2^wexp) so that it
//      fits fp16's range, the result scaled back exactly;
//   2. the contraction Y[(i1, u), s] += sum_j Z[i1, u, j] X[j, s] over chunks of 8 columns, as in
//      products_tc.cu: A2 = the chunk's Z (rows (u, i1), K = 16 reals), B2 = the chunk's X, bf16
//      split in 3 terms (6 products), D2 in TMEM folded every kFlush2 chunks into a second TMEM
//      sum S with round-to-nearest FP32 adds.
//
// Warp roles (192 threads): warps 0-3 ("Z warps", one i1 row per thread = one TMEM lane) build
// B1 from the staged W block, read D1 = Z from TMEM, split it into A2, write the chunk's B2
// slice, fold and drain D2; warp 4 copies each column's U1 fp16 block, W block and X row into a
// ring of stages with cp.async.bulk; warp 5 issues the MMAs.  Buffers and their mbarriers:
//   stage[S]  sfull (copy bytes)          sempty (commit after GEMM1 + the 4 Z warps)
//   B1[4]     b1full (4 Z warps)          b1empty (commit after GEMM1)
//   D1[4]     d1full (commit after GEMM1) d1empty (4 Z warps, D1 read)
//   A2, B2    a2full (4 Z warps)          a2empty (commit after GEMM2)
// Every wait is bounded and sets the CTA's abort flag on timeout (reported through the handle's
// error word).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "stage.cuh"

namespace zbc {

constexpr int kFlush2 = 4;   // chunks accumulated in D2 before it is folded into S
constexpr int kNU2 = 7;      // u values per tile (N1 = 16 covers 8; TMEM: 2 * 7 * 32 + 64 = 512)
constexpr int kTc2Threads = 192;

struct Tc2Layout {
  // shared memory byte offsets (from the 1024-aligned base)
  uint32_t stage0, stage_stride, st_a1, st_w, st_x;  // stage s at stage0 + s * stride; sub-offsets
  uint32_t a1_term;                                  // bytes between the two fp16 terms of A1
  uint32_t b1, b1_buf, b1_term;                      // B1 buffers (4) and their terms
  uint32_t a2, a2_term, a2_tile;                     // A2: term stride, M-tile stride
  uint32_t b2, b2_term;
  uint32_t total;
  int S, NU, RG, kb1max;
  int tmem_cols;
};

__device__ __forceinline__ void st_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ void st_b32(uint32_t addr, uint32_t a) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(a) : "memory");
}

// fp16 hi / lo of two floats, packed
__device__ __forceinline__ void split_h2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const __half2 l = __floats2half2_rn(x0 - __low2float(h), x1 - __high2float(h));
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}
// bf16 hi / mid / lo of two floats, packed
__device__ __forceinline__ void split_b3(float x0, float x1, uint32_t (&t)[3]) {
#pragma unroll
  for (int term = 0; term < 3; ++term) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(x0, x1);
    t[term] = *reinterpret_cast<const uint32_t*>(&b);
    x0 -= __low2float(b);
    x1 -= __high2float(b);
  }
}

// bf16x3 products (A term, B term): (0,0) (0,1) (1,0) (0,2) (2,0) (1,1); fp16x2: (0,0) (0,1) (1,0)
__device__ __forceinline__ int b3a(int i) { return i == 2 ? 1 : i == 4 ? 2 : i == 5 ? 1 : 0; }
__device__ __forceinline__ int b3b(int i) { return i == 1 ? 1 : i == 3 ? 2 : i == 5 ? 1 : 0; }

template <int P2>
__global__ void __launch_bounds__(kTc2Threads, 1)
    matvec_tc2_kernel(const float2* __restrict__ cache, const CacheDesc* __restrict__ cdesc,
                      const unsigned char* __restrict__ half, const HalfDesc* __restrict__ hdesc, Geo g, int q,
                      int M, Tc2Layout L, const float2* __restrict__ XT, int pst, int p, float2* __restrict__ Y,
                      int64_t ldy, int* __restrict__ err) {
  constexpr int P = P2 / 2;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t sfull[kMaxStages], sempty[kMaxStages], b1full[4], b1empty[4], d1full[4], d1empty[4];
  __shared__ uint64_t a2full, a2empty;
  __shared__ int meta_r1p[kMaxStages], meta_kb1[kMaxStages], meta_wexp[kMaxStages];
  __shared__ uint32_t tbase;
  __shared__ volatile int abort_flag;
  const uint32_t sbase = tc::smem_u32(smem);
  const int k = blockIdx.y, s0 = blockIdx.z * P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int S = L.S, NU = L.NU;
  int i1_0, i2_0, i3;
  g.tile(blockIdx.x, i1_0, i2_0, i3);
  const int nu = min(NU, g.n2 - i2_0);  // valid u of this tile
  const int t1 = i1_0 / g.B1;
  const int nchunks = (M + 7) / 8;

  // clear every operand buffer once: the A1 copies fill only RG row groups, and a short last
  // chunk leaves A2 columns unwritten (their X is zero, their Z must be finite)
  for (uint32_t o = threadIdx.x * 16u; o < L.total; o += blockDim.x * 16u)
    *reinterpret_cast<uint4*>(smem + o) = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) tc::tmem_alloc(&tbase, L.tmem_cols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&sfull[s], 1);
      tc::mbar_init(&sempty[s], 1 + 4);  // GEMM1's commit + the four Z warps
    }
    for (int b = 0; b < 4; ++b) {
      tc::mbar_init(&b1full[b], 4);
      tc::mbar_init(&b1empty[b], 1);
      tc::mbar_init(&d1full[b], 1);
      tc::mbar_init(&d1empty[b], 4);
    }
    tc::mbar_init(&a2full, 4);
    tc::mbar_init(&a2empty, 1);
    abort_flag = 0;
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm_d2 = tbase;                                // NU M-tiles x P2 columns
  const uint32_t tm_s = tbase + (uint32_t)(NU * P2);           // the folded sum S
  const uint32_t tm_d1 = tbase + (uint32_t)(2 * NU * P2);      // 4 buffers x 16 columns

  if (warp == 4) {
    // ---------------- copy warp ----------------
    int issued = 0;
    for (int c0 = 0; c0 < M && !__any_sync(0xffffffffu, abort_flag != 0); c0 += 32) {
      CacheDesc mine{};
      HalfDesc mh{};
      if (c0 + lane < M) {
        mine = cdesc[(int64_t)(c0 + lane) * q + k];
        mh = hdesc[(int64_t)(c0 + lane) * q + k];
      }
      const int nb = min(32, M - c0);
      for (int i = 0; i < nb; ++i) {
        const int64_t woff = __shfl_sync(0xffffffffu, mine.woff, i);
        const int r1p = __shfl_sync(0xffffffffu, mine.r1p, i);
        const int64_t hoff = __shfl_sync(0xffffffffu, mh.off, i);
        const int kb1 = __shfl_sync(0xffffffffu, mh.kb1, i);
        const int wexp = __shfl_sync(0xffffffffu, mh.wexp, i);
        const int c = c0 + i, st = c % S;
        bool bad = false;
        if (lane == 0 && c >= S) bad = abort_flag || !tc::mbar_wait(&sempty[st], ((c / S) - 1) & 1);
        if (__shfl_sync(0xffffffffu, bad, 0)) {
          if (lane == 0) abort_flag = 1;
          break;
        }
        if (lane == 0) {
          meta_r1p[st] = r1p;
          meta_kb1[st] = kb1;
          meta_wexp[st] = wexp;
          unsigned char* sb = smem + L.stage0 + (size_t)st * L.stage_stride;
          const uint32_t ab = (uint32_t)L.RG * kb1 * 128u;  // bytes of one fp16 term
          const uint32_t wb = 8u * nu * r1p;
          const uint32_t xb = StageLayout::r16(8u * P);
          mbar_arrive_expect_tx(&sfull[st], 2u * ab + wb + xb);
          const unsigned char* hsrc = half + hoff + (int64_t)t1 * 2 * ab;
          bulk_g2s(sb + L.st_a1, hsrc, ab, &sfull[st]);
          bulk_g2s(sb + L.st_a1 + L.a1_term, hsrc + ab, ab, &sfull[st]);
          bulk_g2s(sb + L.st_w, cache + woff + ((int64_t)i3 * g.n2 + i2_0) * r1p, wb, &sfull[st]);
          bulk_g2s(sb + L.st_x, XT + (int64_t)c * pst + s0, xb, &sfull[st]);
        }
        issued = c + 1;
      }
    }
    if (lane == 0 && abort_flag)  // let the copies in flight land before the CTA exits
      for (int c = std::max(0, issued - S); c < issued; ++c) tc::mbar_wait(&sfull[c % S], (c / S) & 1);
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t id1 = tc::instr_desc(128, 16, 0);  // fp16 operands
      const uint32_t id2 = tc::instr_desc(128, P2, 1);  // bf16 operands
      for (int c = 0; c < M; ++c) {
        const int st = c % S, b = c & 3;
        if (abort_flag || !tc::mbar_wait(&b1full[b], (c >> 2) & 1) || !tc::mbar_wait(&sfull[st], (c / S) & 1) ||
            (c >= 4 && !tc::mbar_wait(&d1empty[b], ((c >> 2) - 1) & 1))) {
          abort_flag = 1;
          break;
        }
        tc::fence_after();
        const int kb1 = meta_kb1[st];
        const uint32_t sbo = (uint32_t)kb1 * 128u;
        const uint32_t a1 = sbase + L.stage0 + (uint32_t)st * L.stage_stride + L.st_a1;
        const uint32_t b1 = sbase + L.b1 + (uint32_t)b * L.b1_buf;
        for (int ks = 0; ks < kb1 / 2; ++ks) {
#pragma unroll
          for (int pr = 0; pr < 3; ++pr) {  // hi*hi, hi*lo, lo*hi
            const uint64_t ad = tc::smem_desc(a1 + (pr == 2 ? L.a1_term : 0u) + ks * 256u, 128, sbo);
            const uint64_t bd = tc::smem_desc(b1 + (pr == 1 ? L.b1_term : 0u) + ks * 256u, 128, sbo);
            tc::mma<0>(tm_d1 + (uint32_t)b * 16u, ad, bd, id1, (ks == 0 && pr == 0) ? 0u : 1u);
          }
        }
        tc::commit(&d1full[b]);
        tc::commit(&sempty[st]);
        tc::commit(&b1empty[b]);
        if ((c & 7) == 7 || c == M - 1) {
          const int ch = c >> 3;
          if (!tc::mbar_wait(&a2full, ch & 1)) {
            abort_flag = 1;
            break;
          }
          tc::fence_after();
          const bool fresh = (ch % kFlush2) == 0;
          for (int m = 0; m < NU; ++m) {
#pragma unroll
            for (int pr = 0; pr < 6; ++pr) {
              const uint64_t ad =
                  tc::smem_desc(sbase + L.a2 + b3a(pr) * L.a2_term + (uint32_t)m * L.a2_tile, 128, 256);
              const uint64_t bd = tc::smem_desc(sbase + L.b2 + b3b(pr) * L.b2_term, 128, 256);
              tc::mma<0>(tm_d2 + (uint32_t)(m * P2), ad, bd, id2, (fresh && pr == 0) ? 0u : 1u);
            }
          }
          tc::commit(&a2empty);
        }
      }
    }
    __syncwarp();
  } else {
    // ---------------- Z warps (warpgroup 0; thread r = TMEM lane = i1 row of the tile) ----------------
    const int r = threadIdx.x;
    const uint32_t lanebase = (uint32_t)(warp * 32) << 16;
    bool s_valid = false;
    // B1 of column c from its staged W block (buffer c & 3); true unless a wait gave up
    auto build_b1 = [&](int c) -> bool {
      const int st = c % S, b = c & 3;
      bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&sfull[st], (c / S) & 1));
      if (ok && c >= 4) ok = __all_sync(0xffffffffu, tc::mbar_wait(&b1empty[b], ((c >> 2) - 1) & 1));
      if (!ok) return false;
      tc::fence_after();
      const int r1p = meta_r1p[st], kb1 = meta_kb1[st];
      const float sc = ldexpf(1.f, -meta_wexp[st]);
      const float2* Ws = (const float2*)(smem + L.stage0 + (size_t)st * L.stage_stride + L.st_w);
      if (r < 16 * kb1) {
        const int n = r / kb1, kc = r % kb1;
        const int u = n >> 1, f = n & 1;
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int a = 4 * kc + i;
          float2 w = make_float2(0.f, 0.f);
          if (u < nu && a < r1p) w = Ws[u * r1p + a];
          w.x *= sc;
          w.y *= sc;
          split_h2(f ? w.y : w.x, f ? w.x : -w.y, hi[i], lo[i]);
        }
        const uint32_t dst = sbase + L.b1 + (uint32_t)b * L.b1_buf + tc::core_off(n, kc, kb1);
        st_v4(dst, hi[0], hi[1], hi[2], hi[3]);
        st_v4(dst + L.b1_term, lo[0], lo[1], lo[2], lo[3]);
      }
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive1(&b1full[b]);
      return true;
    };
    auto fold = [&]() {
      for (int m = 0; m < NU; ++m) {
#pragma unroll 1
        for (int c0 = 0; c0 < P2; c0 += 16) {
          float dv[16];
          tc::tmem_ld16(tm_d2 + lanebase + (uint32_t)(m * P2 + c0), dv);
          if (s_valid) {
            float sv[16];
            tc::tmem_ld16(tm_s + lanebase + (uint32_t)(m * P2 + c0), sv);
#pragma unroll
            for (int i = 0; i < 16; ++i) dv[i] += sv[i];
          }
          tc::tmem_st16(tm_s + lanebase + (uint32_t)(m * P2 + c0), dv);
        }
      }
      tc::tmem_wait_st();
      s_valid = true;
    };
    bool good = true;
    for (int c = 0; c < 2 && c < M && good; ++c) good = build_b1(c);
    for (int c = 0; c < M && good; ++c) {
      const int st = c % S, b = c & 3, jj = c & 7, ch = c >> 3;
      if (__any_sync(0xffffffffu, abort_flag != 0)) {
        good = false;
        break;
      }
      if (c + 2 < M && !(good = build_b1(c + 2))) break;
      const unsigned char* sb = smem + L.stage0 + (size_t)st * L.stage_stride;
      const float zs = ldexpf(1.f, meta_wexp[st]);
      const float2 xv = r < P2 ? ((const float2*)(sb + L.st_x))[r >> 1] : make_float2(0.f, 0.f);
      // the chunk's A2 / B2 buffer is free once the previous chunk's GEMM2 is done; D2 is then
      // complete for a fold
      if (jj == 0 && ch >= 1) {
        if (!(good = __all_sync(0xffffffffu, tc::mbar_wait(&a2empty, (ch - 1) & 1)))) break;
        tc::fence_after();
        if (ch % kFlush2 == 0) fold();
      }
      // B2 slice of column jj: row n = r = 2s + eo (r < P2), reals 2jj, 2jj + 1
      if (r < P2) {
        const int eo = r & 1;
        uint32_t t3[3];
        split_b3(eo == 0 ? xv.x : xv.y, eo == 0 ? -xv.y : xv.x, t3);
        const uint32_t dst = sbase + L.b2 + tc::core_off(r, jj >> 2, 2) + (jj & 3) * 4u;
#pragma unroll
        for (int term = 0; term < 3; ++term) st_b32(dst + term * L.b2_term, t3[term]);
      }
      // D1 = Z (scaled) of this column
      if (!(good = __all_sync(0xffffffffu, tc::mbar_wait(&d1full[b], (c >> 2) & 1)))) break;
      tc::fence_after();
      float z[16];
      tc::tmem_ld16(tm_d1 + lanebase + (uint32_t)b * 16u, z);
      tc::fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive1(&d1empty[b]);
        mbar_arrive1(&sempty[st]);
      }
      // A2 rows (u, r), reals 2jj, 2jj + 1
      const uint32_t a2r = sbase + L.a2 + tc::core_off(r, jj >> 2, 2) + (jj & 3) * 4u;
      for (int u = 0; u < NU; ++u) {
        uint32_t t3[3];
        split_b3(z[2 * u] * zs, z[2 * u + 1] * zs, t3);
#pragma unroll
        for (int term = 0; term < 3; ++term) st_b32(a2r + term * L.a2_term + (uint32_t)u * L.a2_tile, t3[term]);
      }
      if (jj == 7 || c == M - 1) {
        // the last chunk may be short: its missing columns get zero X
        if (c == M - 1 && r < P2)
          for (int j2 = jj + 1; j2 < 8; ++j2)
            for (int term = 0; term < 3; ++term)
              st_b32(sbase + L.b2 + term * L.b2_term + tc::core_off(r, j2 >> 2, 2) + (j2 & 3) * 4u, 0u);
        tc::fence_proxy_async();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive1(&a2full);
      }
    }
    if (!good && lane == 0) abort_flag = 1;
    // drain: the last GEMM2's commit covers every MMA
    if (__all_sync(0xffffffffu, abort_flag == 0)) {
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&a2empty, (nchunks - 1) & 1))) {
        if (lane == 0) abort_flag = 1;
      }
    }
    tc::fence_after();
    if (__all_sync(0xffffffffu, abort_flag == 0)) {
      const int64_t nv = (int64_t)g.n1 * g.n2 * g.n3;
      const int i1 = i1_0 + r;
      const bool okr = r < g.B1 && i1 < g.n1;
      for (int u = 0; u < NU; ++u) {
        const bool ok = okr && u < nu;
        const int64_t v = i1 + (int64_t)g.n1 * ((i2_0 + u) + (int64_t)g.n2 * i3);
#pragma unroll 1
        for (int c0 = 0; c0 < P2; c0 += 16) {
          float vals[16];
          tc::tmem_ld16(tm_d2 + lanebase + (uint32_t)(u * P2 + c0), vals);
          if (s_valid) {
            float sv[16];
            tc::tmem_ld16(tm_s + lanebase + (uint32_t)(u * P2 + c0), sv);
#pragma unroll
            for (int i = 0; i < 16; ++i) vals[i] += sv[i];
          }
          if (ok) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int s = s0 + c0 / 2 + i;
              if (s < p) Y[k * nv + v + ldy * s] = make_float2(vals[2 * i], vals[2 * i + 1]);
            }
          }
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag) atomicExch(err, 1);
  if (warp == 0) tc::tmem_dealloc(tbase, L.tmem_cols);
}

template <int P2>
static int launch_tc2(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  constexpr int P = P2 / 2;
  ZBC_TRY(build_half_cache(h, st));
  const int R = h.cache_r;
  Tc2Layout L{};
  L.NU = std::min(kNU2, 448 / (2 * P2));
  Geo g{};
  g.n1 = h.n1;
  g.n2 = h.n2;
  g.n3 = h.n3;
  g.B1 = tile_b1(h.n1);
  g.NU = std::min(L.NU, h.n2);
  g.NUp = g.NU;
  g.nb1 = (h.n1 + g.B1 - 1) / g.B1;
  g.nb2 = (h.n2 + g.NU - 1) / g.NU;
  g.nb32 = (g.B1 + 31) / 32;
  L.RG = (g.B1 + 7) / 8;
  L.kb1max = h.cache->kb1_max;
  L.a1_term = 16u * L.kb1max * 128u;
  L.st_a1 = 0;
  L.st_w = 2 * L.a1_term;
  L.st_x = L.st_w + StageLayout::r16(8u * L.NU * R);
  L.stage_stride = (L.st_x + StageLayout::r16(8u * P) + 127u) / 128u * 128u;
  L.b1_term = 2u * L.kb1max * 128u;
  L.b1_buf = 2 * L.b1_term;
  L.a2_tile = 16u * 256u;
  L.a2_term = (uint32_t)L.NU * L.a2_tile;
  L.b2_term = (uint32_t)(P2 / 8) * 256u;
  L.b1 = 0;
  L.a2 = 4 * L.b1_buf;
  L.b2 = L.a2 + 3 * L.a2_term;
  L.stage0 = (L.b2 + 3 * L.b2_term + 127u) / 128u * 128u;
  const size_t budget = 220 * 1024 - 1024;  // 1024: alignment of the dynamic base
  if (L.stage0 + 3 * (size_t)L.stage_stride > budget) {
    set_error("chained tensor-core layout does not fit (rank %d)", R);
    return ZBC_EINVAL;
  }
  L.S = (int)std::min<size_t>(kMaxStages, (budget - L.stage0) / L.stage_stride);
  L.total = L.stage0 + (uint32_t)L.S * L.stage_stride;
  int cols = 32;
  while (cols < 2 * L.NU * P2 + 64) cols <<= 1;
  L.tmem_cols = cols;
  const float2* XT;
  int pst;
  ZBC_TRY(transpose_rhs(h, X, ldx, p, P, &XT, &pst, st));
  static bool attr_set = false;
  if (!attr_set) {
    ZBC_TRY_CUDA(cudaFuncSetAttribute(matvec_tc2_kernel<P2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      220 * 1024));
    attr_set = true;
  }
  dim3 grid(g.ntiles(), h.q, ceil_div(p, P));
  matvec_tc2_kernel<P2><<<grid, kTc2Threads, L.total + 1024, st>>>(h.cache->data, h.cache->d_desc, h.cache->half,
                                                                    h.cache->d_half, g, h.q, h.M, L, XT, pst, p, Y,
                                                                    ldy, (int*)h.work_err.ptr);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

int matvec_tc2(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  if (p <= 8) return launch_tc2<16>(h, X, ldx, p, Y, ldy, st);
  if (p <= 16) return launch_tc2<32>(h, X, ldx, p, Y, ldy, st);
  if (p <= 32) return launch_tc2<64>(h, X, ldx, p, Y, ldy, st);
  return launch_tc2<128>(h, X, ldx, p, Y, ldy, st);
}

}  // namespace zbc
