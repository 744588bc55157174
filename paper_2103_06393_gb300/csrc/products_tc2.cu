// Algorithm 1 (Y = Z X, Sec. III.B) with both of its GEMM-shaped steps on the tensor cores:
//
//   1. the last mode product of the decompression, per stored column j and voxel tile,
//        Z[i1, u] = sum_a U1_j[i1, a] W_j[a, u]           (W = G x2 U2 x3 U3, cached)
//      as a tcgen05 MMA with M = 128 (i1), N = 16 (u = 0..7, Re / Im), K = 2 r1p (a, Re / Im)
//      padded to 16: the real embedding A1[i1][2a + e] = (Re, Im) U1, and
//        B1[2u][2a] = Re W, B1[2u][2a+1] = -Im W, B1[2u+1][2a] = Im W, B1[2u+1][2a+1] = Re W;
//      operands split into two fp16 terms (hi, lo = x - hi; products hh, hl, lh), U1 pre-split in
//      the handle's cache, W split per column after scaling by 2^-wexp (|W| < 2^wexp), both
//      operands scaled by 2^kHalfShift so their lo terms stay normal fp16 numbers, the result
//      scaled back exactly;
//   2. the contraction Y[(i1, u), s] += sum_j Z[i1, u, j] X[j, s] over chunks of 8 columns, as in
//      products_tc.cu: A2 = the chunk's Z (rows (u, i1), K = 16 reals), B2 = the chunk's X, bf16
//      split in 3 terms (6 products), D2 in TMEM folded every kFlush2 chunks into a second TMEM
//      sum S with round-to-nearest FP32 adds.
//
// Warp roles (352 threads): two warpgroups of "Z warps" (warps 0-7; thread = TMEM lane = i1 row
// of the tile), each taking every other pair of a chunk's columns: they build B1 from the staged
// W block (a few columns ahead), read D1 = Z from TMEM, split it into A2 words kept in
// registers, and store a chunk's A2 / B2 once the previous chunk's GEMM2 is done; warpgroup 0
// also folds and drains D2.  Warp 8 copies each column's U1 fp16 block into the A1 ring, warp 9
// its W block and X row into the W / X ring (cp.async.bulk); warp 10 issues the MMAs, GEMM1 and
// GEMM2 each as soon as their operands are ready.  Buffers and mbarriers:
//   A1[S1]    a1full (copy bytes)         a1empty (commit after GEMM1)
//   WX[16]    wxfull (copy bytes)         wxempty (the column's 4 Z warps)
//   B1[8]     b1full (4 Z warps)          b1empty (commit after GEMM1)
//   D1[8]     d1full (commit after GEMM1) d1empty (4 Z warps, D1 read)
//   A2, B2    a2full (all 8 Z warps)      a2empty (commit after GEMM2)
// Every wait is bounded and sets the CTA's abort flag on timeout (reported through the handle's
// error word).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "stage.cuh"

namespace zbc {

constexpr int kFlush2 = 4;   // chunks accumulated in D2 before it is folded into S
constexpr int kNU2 = 8;      // u values per tile at most (N1 = 16: u = 0..7, Re / Im)
constexpr int kB1 = 8;       // B1 buffers and D1 buffers (TMEM: 2 NU P2 + 8 * 16 <= 512)
constexpr int kAhead = 2;    // B1 is built this many of a warpgroup's columns ahead
constexpr int kS2 = 16;      // W / X ring depth
constexpr int kTc2Threads = 352;
constexpr int kCopyA1 = 8, kCopyWX = 9, kMmaWarp = 10;

// non-blocking test of phase `parity`
__device__ __forceinline__ bool mbar_test(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(tc::smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait that lets the thread sleep (up to ~1 us per try) instead of spinning
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* mbar, uint32_t parity, uint32_t max_iter = 4000000u) {
  const uint32_t a = tc::smem_u32(mbar);
  for (uint32_t it = 0; it < max_iter; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity), "r"(1000u)
        : "memory");
    if (ok) return true;
  }
  return false;
}

struct Tc2Layout {
  // shared memory byte offsets (from the 1024-aligned base)
  uint32_t a1, a1_slot, a1_term;   // A1 ring: S1 slots, each two fp16 terms of RG row groups
  uint32_t wx, wx_slot, wx_x;      // W / X ring: S2 slots; X at wx_x within a slot
  uint32_t b1, b1_buf, b1_term;    // B1 buffers (kB1) and their terms
  uint32_t a2, a2_term, a2_tile;   // A2: term stride, M-tile stride
  uint32_t b2, b2_term;
  uint32_t total;
  int S1, S2, NU, RG, kb1max;
  int tmem_cols;
};

__device__ __forceinline__ void st_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ void st_shared_v2(uint32_t addr, uint32_t a, uint32_t b) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
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
  __shared__ uint64_t a1full[kMaxStages], a1empty[kMaxStages], wxfull[kS2], wxempty[kS2];
  __shared__ uint64_t b1full[kB1], b1empty[kB1], d1full[kB1], d1empty[kB1], a2full, a2empty;
  __shared__ int a1_kb1[kMaxStages], wx_r1p[kS2], wx_kb1[kS2], wx_wexp[kS2], wx_uexp[kS2];
  __shared__ uint32_t tbase;
  __shared__ volatile int abort_flag;
  const uint32_t sbase = tc::smem_u32(smem);
  const int k = blockIdx.y, s0 = blockIdx.z * P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int S1 = L.S1, NU = L.NU;
  int i1_0, i2_0, i3;
  g.tile(blockIdx.x, i1_0, i2_0, i3);
  const int nu = min(NU, g.n2 - i2_0);  // valid u of this tile
  const int t1 = i1_0 / g.B1;
  const int nchunks = (M + 7) / 8;

  // clear every buffer once (a short last chunk leaves A2 columns unwritten: finite zeros there)
  for (uint32_t o = threadIdx.x * 16u; o < L.total; o += blockDim.x * 16u)
    *reinterpret_cast<uint4*>(smem + o) = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) tc::tmem_alloc(&tbase, L.tmem_cols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S1; ++s) {
      tc::mbar_init(&a1full[s], 1);
      tc::mbar_init(&a1empty[s], 1);  // GEMM1's commit
    }
    for (int s = 0; s < kS2; ++s) {
      tc::mbar_init(&wxfull[s], 1);
      tc::mbar_init(&wxempty[s], 4);  // the column's four Z warps
    }
    for (int b = 0; b < kB1; ++b) {
      tc::mbar_init(&b1full[b], 4);
      tc::mbar_init(&b1empty[b], 1);
      tc::mbar_init(&d1full[b], 1);
      tc::mbar_init(&d1empty[b], 4);
    }
    tc::mbar_init(&a2full, 8);
    tc::mbar_init(&a2empty, 1);
    abort_flag = 0;
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm_d2 = tbase;                            // NU M-tiles x P2 columns
  const uint32_t tm_s = tbase + (uint32_t)(NU * P2);       // the folded sum S
  const uint32_t tm_d1 = tbase + (uint32_t)(2 * NU * P2);  // kB1 buffers x 16 columns

  if (warp == kCopyA1 || warp == kCopyWX) {
    // ---------------- copy warps: U1 fp16 blocks (A1 ring); W blocks and X rows (W / X ring) ----
    const bool a1w = warp == kCopyA1;
    const int SR = a1w ? S1 : kS2;
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
        const int uexp = __shfl_sync(0xffffffffu, mh.uexp, i);
        const int c = c0 + i, st = c % SR;
        bool bad = false;
        if (lane == 0 && c >= SR)
          bad = abort_flag || !mbar_wait_sleep(a1w ? &a1empty[st] : &wxempty[st], ((c / SR) - 1) & 1);
        if (__shfl_sync(0xffffffffu, bad, 0)) {
          if (lane == 0) abort_flag = 1;
          break;
        }
        if (lane == 0) {
          if (a1w) {
            a1_kb1[st] = kb1;
            unsigned char* dst = smem + L.a1 + (size_t)st * L.a1_slot;
            const uint32_t ab = (uint32_t)L.RG * kb1 * 128u;  // bytes of one fp16 term
            mbar_arrive_expect_tx(&a1full[st], 2u * ab);
            const unsigned char* hsrc = half + hoff + (int64_t)t1 * 2 * ab;
            bulk_g2s(dst, hsrc, ab, &a1full[st]);
            bulk_g2s(dst + L.a1_term, hsrc + ab, ab, &a1full[st]);
          } else {
            wx_r1p[st] = r1p;
            wx_kb1[st] = kb1;
            wx_wexp[st] = wexp;
            wx_uexp[st] = uexp;
            unsigned char* dst = smem + L.wx + (size_t)st * L.wx_slot;
            const uint32_t wb = 8u * nu * r1p;
            const uint32_t xb = StageLayout::r16(8u * P);
            mbar_arrive_expect_tx(&wxfull[st], wb + xb);
            bulk_g2s(dst, cache + woff + ((int64_t)i3 * g.n2 + i2_0) * r1p, wb, &wxfull[st]);
            bulk_g2s(dst + L.wx_x, XT + (int64_t)c * pst + s0, xb, &wxfull[st]);
          }
        }
        issued = c + 1;
      }
    }
    if (lane == 0 && abort_flag)  // let the copies in flight land before the CTA exits
      for (int c = std::max(0, issued - SR); c < issued; ++c)
        tc::mbar_wait(a1w ? &a1full[c % SR] : &wxfull[c % SR], (c / SR) & 1);
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issuer ----------------
    // GEMM1 of the next column and GEMM2 of the next chunk are issued as soon as their operands
    // are ready, in either order (non-blocking tests)
    if (lane == 0) {
      const uint32_t id1 = tc::instr_desc(128, 16, 0);  // fp16 operands
      const uint32_t id2 = tc::instr_desc(128, P2, 1);  // bf16 operands
      int c = 0, ch = 0;
      uint32_t idle = 0;
      while ((c < M || ch < nchunks) && !abort_flag) {
        bool progressed = false;
        if (c < M) {
          const int st = c % S1, b = c & (kB1 - 1);
          if (mbar_test(&b1full[b], (c / kB1) & 1) && mbar_test(&a1full[st], (c / S1) & 1) &&
              (c < kB1 || mbar_test(&d1empty[b], ((c / kB1) - 1) & 1))) {
            tc::fence_after();
            const int kb1 = a1_kb1[st];
            const uint32_t sbo = (uint32_t)kb1 * 128u;
            const uint32_t a1 = sbase + L.a1 + (uint32_t)st * L.a1_slot;
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
            tc::commit(&a1empty[st]);
            tc::commit(&b1empty[b]);
            ++c;
            progressed = true;
          }
        }
        if (ch < nchunks && mbar_test(&a2full, ch & 1)) {
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
          ++ch;
          progressed = true;
        }
        if (progressed) {
          idle = 0;
        } else if (++idle > 100000000u) {  // nothing became ready for seconds
          abort_flag = 1;
        } else {
          __nanosleep(32);
        }
      }
    }
    __syncwarp();
  } else if (warp < 8) {
    // ---------------- Z warps (thread = TMEM lane r = i1 row of the tile) ----------------
    const int wg = warp >> 2;
    const int r = threadIdx.x & 127;
    const uint32_t lanebase = (uint32_t)((warp & 3) * 32) << 16;
    bool s_valid = false;
    // warpgroup wg takes the column pairs {4t + 2wg, 4t + 2wg + 1} (t = 0, 1) of every chunk, so
    // both consume the rings in order; own column number n -> global column
    auto col = [&](int n) { return 8 * (n >> 2) + 4 * ((n & 3) >> 1) + 2 * wg + (n & 1); };
    // B1 of column c from its staged W block (buffer c % kB1); true unless a wait gave up
    auto build_b1 = [&](int c) -> bool {
      const int st = c % kS2, b = c & (kB1 - 1);
      bool ok = __all_sync(0xffffffffu, mbar_wait_sleep(&wxfull[st], (c / kS2) & 1));
      if (ok && c >= kB1) ok = __all_sync(0xffffffffu, mbar_wait_sleep(&b1empty[b], ((c / kB1) - 1) & 1));
      if (!ok) return false;
      tc::fence_after();
      const int r1p = wx_r1p[st], kb1 = wx_kb1[st];
      const float sc = ldexpf(1.f, kHalfShift - wx_wexp[st]);
      const float2* Ws = (const float2*)(smem + L.wx + (size_t)st * L.wx_slot);
      for (int it = r; it < 16 * kb1; it += 128) {  // (row, 16-byte chunk) items
        const int n = it / kb1, kc = it % kb1;
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
    for (int n = 0; n < kAhead && good; ++n)
      if (col(n) < M) good = build_b1(col(n));
    for (int ch = 0; ch < nchunks && good; ++ch) {
      uint32_t aw[4][kNU2][3];  // A2 words: column q4, u, term
      uint32_t bw[4][3];        // B2 words of row r (r < P2)
      int nq = 0;               // this warpgroup's columns in the chunk
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const int n = 4 * ch + q4, c = col(n);
#pragma unroll
        for (int u = 0; u < kNU2; ++u) aw[q4][u][0] = aw[q4][u][1] = aw[q4][u][2] = 0u;
        bw[q4][0] = bw[q4][1] = bw[q4][2] = 0u;
        if (c >= M || !good) continue;
        ++nq;
        const int st = c % kS2, b = c & (kB1 - 1);
        if (__any_sync(0xffffffffu, abort_flag != 0)) {
          good = false;
          continue;
        }
        const int cn = col(n + kAhead);
        if (cn < M && !(good = build_b1(cn))) continue;
        const unsigned char* sb = smem + L.wx + (size_t)st * L.wx_slot;
        const float zs = ldexpf(1.f, wx_wexp[st] + wx_uexp[st] - 2 * kHalfShift);
        if (r < P2) {
          const float2 xv = ((const float2*)(sb + L.wx_x))[r >> 1];
          const int eo = r & 1;
          split_b3(eo == 0 ? xv.x : xv.y, eo == 0 ? -xv.y : xv.x, bw[q4]);
        }
        if (!(good = __all_sync(0xffffffffu, mbar_wait_sleep(&d1full[b], (c / kB1) & 1)))) continue;
        tc::fence_after();
        float z[16];
        tc::tmem_ld16(tm_d1 + lanebase + (uint32_t)b * 16u, z);
        tc::fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive1(&d1empty[b]);
          mbar_arrive1(&wxempty[st]);
        }
#pragma unroll
        for (int u = 0; u < kNU2; ++u)
          if (u < NU) split_b3(z[2 * u] * zs, z[2 * u + 1] * zs, aw[q4][u]);
      }
      if (!good) break;
      // the A2 / B2 buffer is free once GEMM2 of chunk ch-1 is done; D2 is then complete for a
      // fold (warpgroup 0, whose warps own the TMEM lanes like warpgroup 1's)
      if (ch >= 1) {
        if (!(good = __all_sync(0xffffffffu, mbar_wait_sleep(&a2empty, (ch - 1) & 1)))) break;
        tc::fence_after();
        if (wg == 0 && ch % kFlush2 == 0) fold();
      }
      // each pair of columns is 8 contiguous bytes of a row (reals 2j .. 2j + 3); columns at or
      // beyond M carry zero words (their X is zero)
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int jj = 4 * t + 2 * wg;
        const uint32_t off = tc::core_off(r, jj >> 2, 2) + (jj & 3) * 4u;
        if (r < P2)
#pragma unroll
          for (int term = 0; term < 3; ++term)
            st_shared_v2(sbase + L.b2 + term * L.b2_term + off, bw[2 * t][term], bw[2 * t + 1][term]);
        if (nq > 2 * t) {
#pragma unroll
          for (int u = 0; u < kNU2; ++u) {
            if (u >= NU) break;
#pragma unroll
            for (int term = 0; term < 3; ++term)
              st_shared_v2(sbase + L.a2 + term * L.a2_term + (uint32_t)u * L.a2_tile + off, aw[2 * t][u][term],
                           aw[2 * t + 1][u][term]);
          }
        }
      }
      tc::fence_proxy_async();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive1(&a2full);
    }
    if (!good && lane == 0) abort_flag = 1;
    // drain (warpgroup 0): the last GEMM2's commit covers every MMA
    if (wg == 0) {
      if (__all_sync(0xffffffffu, abort_flag == 0)) {
        if (!__all_sync(0xffffffffu, mbar_wait_sleep(&a2empty, (nchunks - 1) & 1))) {
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
  }
  tc::fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag) atomicOr(err, kErrTimeout);
  if (warp == 0) tc::tmem_dealloc(tbase, L.tmem_cols);
}

template <int P2>
static int launch_tc2(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  constexpr int P = P2 / 2;
  ZBC_TRY(build_half_cache(h, st));
  const int R = h.cache_r;
  Tc2Layout L{};
  L.NU = std::min(kNU2, (512 - 16 * kB1) / (2 * P2));
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
  // the A1 ring comes first: an M = 128 MMA on a slot reads up to 16 row groups, past the RG
  // stored ones, into the buffers that follow (rows whose results are never used)
  L.a1_term = (uint32_t)L.RG * L.kb1max * 128u;
  L.a1_slot = 2 * L.a1_term;
  L.wx_x = StageLayout::r16(8u * L.NU * R);
  L.wx_slot = (L.wx_x + StageLayout::r16(8u * P) + 127u) / 128u * 128u;
  L.b1_term = 2u * L.kb1max * 128u;
  L.b1_buf = 2 * L.b1_term;
  L.a2_tile = 16u * 256u;
  L.a2_term = (uint32_t)L.NU * L.a2_tile;
  L.b2_term = (uint32_t)(P2 / 8) * 256u;
  const size_t fixed = (size_t)kS2 * L.wx_slot + (size_t)kB1 * L.b1_buf + 3 * (size_t)L.a2_term + 3 * L.b2_term;
  const size_t budget = 220 * 1024 - 1024;  // 1024: alignment of the dynamic base
  const size_t overrun = (size_t)(16 - L.RG) * L.kb1max * 128u + L.a1_term;
  if (fixed + 2 * (size_t)L.a1_slot > budget || fixed < overrun) {
    set_error("chained tensor-core layout does not fit (rank %d)", R);
    return ZBC_EINVAL;
  }
  L.S1 = (int)std::min<size_t>(kMaxStages, (budget - fixed) / L.a1_slot);
  L.a1 = 0;
  L.wx = (uint32_t)L.S1 * L.a1_slot;
  L.b1 = L.wx + (uint32_t)kS2 * L.wx_slot;
  L.a2 = L.b1 + (uint32_t)kB1 * L.b1_buf;
  L.b2 = L.a2 + 3 * L.a2_term;
  L.total = L.b2 + 3 * L.b2_term;
  int cols = 32;
  while (cols < 2 * L.NU * P2 + 16 * kB1) cols <<= 1;
  L.tmem_cols = cols;
  const float2* XT;
  int pst;
  ZBC_TRY(transpose_rhs(h, X, ldx, p, P, &XT, &pst, st));
  ZBC_TRY((set_smem_limit<matvec_tc2_kernel<P2>>(220 * 1024)));
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
