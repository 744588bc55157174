// Tensor-core form of Algorithm 1 (Y = Z X, Sec. III.B) with tcgen05 on sm_103a.
//
// The decompression front end (decomp.cuh) produces, per chunk of 8 stored columns, the
// tile's decompressed block Z[rho, j] (rho = voxel row of the tile) on CUDA cores and writes
// it straight into shared memory as the A operand of a tcgen05 GEMM; the B operand is the
// matching chunk of X.  Both are complex and enter the MMA through the real embedding
//   A'[rho][2j + e] = (Re, Im) Z[rho, j],
//   B'^T[2s][2j] = Re X[j,s],  B'^T[2s][2j+1] = -Im X[j,s],
//   B'^T[2s+1][2j] = Im X[j,s], B'^T[2s+1][2j+1] = Re X[j,s],
// so that D[rho][2s + e] accumulates (Re, Im) Y[rho, s] in TMEM.
//
// Precision: FP32 values are split into tensor-core terms and the cross products above
// 2^-24 are accumulated (Fmt below):
//   TF32X3 : x = hi + lo (tf32), products hi*hi + hi*lo + lo*hi        (kind::tf32)
//   BF16X3 : x = hi + mid + lo (bf16), products hh hm mh hl lh mm       (kind::f16, bf16)
// The tensor core's FP32 accumulation truncates, so its error grows with the number of
// accumulation steps into one accumulator.  The TMEM accumulator D therefore restarts every
// kFlush chunks and is added, with round-to-nearest FP32 on the CUDA cores, into a second TMEM
// region S; Y = S + D at the end.
//
// Warp roles: two copy warps stream each column's U1 / W blocks into the stage rings of stage.cuh
// (cp.async.bulk); the front-end ("producer") warps form the last mode product of one task of
// the tile from the staged blocks and fill the operands of a chunk -- two warps per task, one
// for each half of the chunk's columns (pairs interleaved), so that more warps hide the
// shared-memory latency; one more warp issues the MMAs.  Each half has its own stage ring: a
// ring shared by halves that consume different columns would let a fast half wait on a slot two
// phases behind, where an mbarrier parity test cannot tell the phases apart.  One operand buffer:
// an mbarrier "full" (one arrival per producer warp) hands the chunk's filled operands to the
// issuer, and tcgen05.commit on an mbarrier "empty" hands them back once the tensor cores have
// consumed them.  No CTA-wide barrier is taken between the prologue and the epilogue.
#include <cuda_bf16.h>

#include <algorithm>

#include "stage.cuh"

namespace zbc {

constexpr int kFlush = 4;       // chunks accumulated in D before it is folded into S
constexpr int kTcMaxTasks = 6;  // tasks per tile, at most (two producer warps each)
constexpr int kTcThreads = 32 * (2 * kTcMaxTasks + 3);  // + a copy warp per half and the MMA issuer

template <int FMT>
struct Fmt;
template <>
struct Fmt<ZBC_TF32X3> {
  static constexpr int esz = 4, terms = 2, nprod = 3, kind = 1, idfmt = 2;
  __device__ static constexpr int pa(int i) { return i == 2 ? 1 : 0; }
  __device__ static constexpr int pb(int i) { return i == 1 ? 1 : 0; }
};
template <>
struct Fmt<ZBC_BF16X3> {
  static constexpr int esz = 2, terms = 3, nprod = 6, kind = 0, idfmt = 1;
  // (0,0) (0,1) (1,0) (0,2) (2,0) (1,1)
  __device__ static constexpr int pa(int i) { return i == 2 ? 1 : i == 4 ? 2 : i == 5 ? 1 : 0; }
  __device__ static constexpr int pb(int i) { return i == 1 ? 1 : i == 3 ? 2 : i == 5 ? 1 : 0; }
};

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Split NF floats (one 16-byte chunk of the operand) into the format's terms.
template <int FMT, int NF>
__device__ __forceinline__ void split_words(const float (&x)[NF], uint32_t (&t)[Fmt<FMT>::terms][4]) {
  if constexpr (FMT == ZBC_TF32X3) {
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      const uint32_t h = tf32_bits(x[i]);
      t[0][i] = h;
      t[1][i] = tf32_bits(x[i] - __uint_as_float(h));
    }
  } else {
#pragma unroll
    for (int i = 0; i < NF / 2; ++i) {
      float r0 = x[2 * i], r1 = x[2 * i + 1];
#pragma unroll
      for (int term = 0; term < 3; ++term) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(r0, r1);
        t[term][i] = *reinterpret_cast<const uint32_t*>(&b);
        r0 -= __low2float(b);
        r1 -= __high2float(b);
      }
    }
  }
}

__device__ __forceinline__ void st_shared_v2(uint32_t addr, uint32_t w0, uint32_t w1) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(w0), "r"(w1) : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, const uint32_t (&w)[4]) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
               : "memory");
}

struct TcLayout {
  int NR;        // accumulator rows of the tile (multiple of 128)
  int nmt;       // M tiles
  int KBA;       // 16-byte K chunks per operand row for one column chunk (= esz)
  int a_bytes;   // one term of one A buffer
  int b_bytes;   // one term of one B buffer
  int tmem_cols;
  int nprodw;    // producer warps (>= 4, >= ntask); the issuer is warp nprodw
};

template <int FMT, int P2>
__global__ void __launch_bounds__(kTcThreads, 1)
    matvec_tc_kernel(const float2* __restrict__ cache, const CacheDesc* __restrict__ cdesc, Geo g, int q, int M,
                     StageLayout SL, int S, TcLayout L, const float2* __restrict__ XT, int pst, int p,
                     float2* __restrict__ Y, int64_t ldy, int* __restrict__ err) {
  using F = Fmt<FMT>;
  constexpr int NF = 16 / F::esz;  // floats per 16-byte chunk
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t sfull[kMaxStages], sempty[kMaxStages], ofull[2], oempty[2];
  __shared__ int meta[kMaxStages];
  __shared__ uint32_t tbase;
  __shared__ volatile int abort_flag;
  unsigned char* stages = smem;
  unsigned char* ops = (unsigned char*)(((uintptr_t)(smem + (size_t)S * SL.stride) + 1023) & ~(uintptr_t)1023);
  // two rings of Sh = S / 2 stages, one per producer half: each ring is consumed in order by all
  // of its consumers, so no waiter can run two phases ahead of a slot (parity waits stay exact)
  const int Sh = S / 2;
  // one operand buffer: a chunk's operands are written once the previous chunk's MMAs are done
  // (the wait comes after the first columns' last mode products, so it rarely blocks), which
  // leaves shared memory for a deeper stage ring
  auto a_op = [&](int, int term) { return ops + (size_t)term * L.a_bytes; };
  auto b_op = [&](int, int term) { return ops + (size_t)F::terms * L.a_bytes + (size_t)term * L.b_bytes; };
  const int k = blockIdx.y;
  const int s0 = blockIdx.z * (P2 / 2);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nprod = L.nprodw * 32;
  const int B1p = (g.B1 + 1) / 2 * 2;
  int i1_0, i2_0, i3;
  g.tile(blockIdx.x, i1_0, i2_0, i3);

  if (warp == 0) tc::tmem_alloc(&tbase, L.tmem_cols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&sfull[s], 1);
      tc::mbar_init(&sempty[s], g.ntask);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&ofull[b], L.nprodw);
      tc::mbar_init(&oempty[b], 1);
    }
    abort_flag = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem_d = tbase;                           // D: nmt * P2 columns
  const uint32_t tmem_s = tbase + (uint32_t)(L.nmt * P2);  // S: nmt * P2 columns
  const int nchunks = (M + kChunk - 1) / kChunk;

  if (warp == L.nprodw || warp == L.nprodw + 1) {
    // ---------------- copy warps, one per half: its columns' U1 / W blocks into its ring ----------------
    // lane l holds the cache entry of column c0 + l of the current batch of 32 columns
    const int hw = warp - L.nprodw;  // the half this warp feeds
    int issued = 0;
    for (int c0 = 0; c0 < M && !__any_sync(0xffffffffu, abort_flag != 0); c0 += 32) {
      CacheDesc mine{};
      if (c0 + lane < M) mine = cdesc[(int64_t)(c0 + lane) * q + k];
      const int nb = min(32, M - c0);
      for (int i = 0; i < nb; ++i) {
        CacheDesc d;
        d.woff = __shfl_sync(0xffffffffu, mine.woff, i);
        d.uoff = __shfl_sync(0xffffffffu, mine.uoff, i);
        d.r1 = __shfl_sync(0xffffffffu, mine.r1, i);
        d.r1p = __shfl_sync(0xffffffffu, mine.r1p, i);
        // column c goes to the ring of the half that consumes it (slots h * Sh .. h * Sh + Sh - 1),
        // as that half's n-th column
        const int c = c0 + i, h = (c >> 1) & 1, n = (c >> 2) * 2 + (c & 1), st = h * Sh + n % Sh;
        if (h != hw) continue;
        bool bad = false;
        if (lane == 0 && n >= Sh) bad = abort_flag || !tc::mbar_wait(&sempty[st], ((n / Sh) - 1) & 1);
        if (__shfl_sync(0xffffffffu, bad, 0)) {
          if (lane == 0) abort_flag = 1;
          break;
        }
        if (lane == 0)
          issue_item(stages + (size_t)st * SL.stride, SL, &sfull[st], &meta[st], cache, d, g, B1p, i1_0, i2_0, i3,
                     nullptr, 0u);
        issued = c + 1;
      }
    }
    if (lane == 0 && abort_flag)  // let the copies in flight land before the CTA exits
      for (int c = std::max(0, issued - 2 * Sh - 2); c < issued; ++c) {
        const int h = (c >> 1) & 1, n = (c >> 2) * 2 + (c & 1);
        if (h == hw) tc::mbar_wait(&sfull[h * Sh + n % Sh], (n / Sh) & 1);
      }
  } else if (warp == L.nprodw + 2) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = tc::instr_desc(128, P2, F::idfmt);
      const uint32_t sbo = L.KBA * 128;
      const int ksteps = L.KBA / 2;
      for (int ch = 0; ch < nchunks; ++ch) {
        const int buf = ch & 1;
        if (abort_flag || !tc::mbar_wait(&ofull[buf], (ch >> 1) & 1)) {
          abort_flag = 1;
          break;
        }
        tc::fence_after();
        const bool fresh = (ch % kFlush) == 0;
#pragma unroll 1
        for (int m = 0; m < L.nmt; ++m) {
#pragma unroll
          for (int pr = 0; pr < F::nprod; ++pr) {
            const uint32_t abase = tc::smem_u32(a_op(buf, F::pa(pr))) + m * 16 * sbo;
            const uint32_t bbase = tc::smem_u32(b_op(buf, F::pb(pr)));
            for (int ks = 0; ks < ksteps; ++ks) {
              const uint64_t ad = tc::smem_desc(abase + ks * 256, 128, sbo);
              const uint64_t bd = tc::smem_desc(bbase + ks * 256, 128, sbo);
              tc::mma<F::kind>(tmem_d + m * P2, ad, bd, idesc, (fresh && pr == 0 && ks == 0) ? 0u : 1u);
            }
          }
        }
        tc::commit(&oempty[buf]);
      }
    }
    __syncwarp();
  } else {
    // ---------------- producers: last mode product, operand split, fold, epilogue ----------------
    const int tid = threadIdx.x;
    const int ngroups = L.nprodw / 4;  // warpgroups that fold and drain the accumulators
    const int wq = warp & 3, wg = warp >> 2;
    // warps tk and tk + ntask share task tk, each taking half of the chunk's columns
    const bool task = warp < 2 * g.ntask;
    const int tk = warp % g.ntask, half = warp / g.ntask;
    int i1 = 0, u0 = 0;
    bool ok = false;
    if (task) g.task(i1_0, tk, lane, i1, u0, ok);
    const int il = ok ? i1 - i1_0 : 0;
    bool s_valid = false;
    // D -> S (round-to-nearest FP32) by whole warpgroups; D must be complete
    auto fold = [&]() {
      if (wg >= ngroups) return;
      for (int m = wg; m < L.nmt; m += ngroups) {
        const uint32_t lanebase = (uint32_t)(wq * 32) << 16;
#pragma unroll 1
        for (int c0 = 0; c0 < P2; c0 += 16) {
          float dv[16];
          tc::tmem_ld16(tmem_d + lanebase + m * P2 + c0, dv);
          if (s_valid) {
            float sv[16];
            tc::tmem_ld16(tmem_s + lanebase + m * P2 + c0, sv);
#pragma unroll
            for (int i = 0; i < 16; ++i) dv[i] += sv[i];
          }
          tc::tmem_st16(tmem_s + lanebase + m * P2 + c0, dv);
        }
      }
      tc::tmem_wait_st();
    };
    for (int ch = 0; ch < nchunks; ++ch) {
      const int buf = ch & 1;
      const int j0 = ch * kChunk;
      const int jc = min(kChunk, M - j0);
      const bool do_fold = ch > 0 && (ch % kFlush) == 0;
      // 1. before the first store: the operand buffer is free, and D complete for a fold, once
      //    chunk ch-1's MMAs are done
      bool freed = ch == 0;
      auto ensure_free = [&]() {
        if (freed) return;
        freed = true;
        bool bad = abort_flag != 0;
        if (!bad) bad = !tc::mbar_wait(&oempty[(ch - 1) & 1], ((ch - 1) >> 1) & 1);
        if (__any_sync(0xffffffffu, bad) && lane == 0) abort_flag = 1;
        tc::fence_after();
        if (do_fold && !__any_sync(0xffffffffu, abort_flag != 0)) {
          fold();
          s_valid = true;
        }
      };
      // 2. this thread's share of the chunk's X values (loaded now, used after the last mode)
      constexpr int nk16 = 2 * kChunk / NF;
      constexpr int kBMax = (P2 * nk16 + 127) / 128;  // B elements per thread (>= 128 producers)
      float2 xv[kBMax][NF / 2];
#pragma unroll
      for (int b = 0; b < kBMax; ++b) {
        const int e = tid + b * nprod;
        const int n = e / nk16, kc = e % nk16;
#pragma unroll
        for (int i = 0; i < NF / 2; ++i) {
          const int jj = kc * (NF / 2) + i;
          xv[b][i] = (e < P2 * nk16 && jj < jc) ? XT[(int64_t)(j0 + jj) * pst + s0 + (n >> 1)] : make_float2(0.f, 0.f);
        }
      }
      // 3. A operand: the last mode product of this warp's task for its columns of the chunk,
      //    pairs {4g + 2 half, 4g + 2 half + 1} (so both halves consume the stage ring in order)
      if (task) {
#pragma unroll 1
        for (int g4 = 0; g4 < kChunk / 4; ++g4) {
          const int jj0 = 4 * g4 + 2 * half;
          float x[kUQ][4];
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const int jj = jj0 + t;
            float2 zz[kUQ];
#pragma unroll
            for (int l = 0; l < kUQ; ++l) zz[l] = make_float2(0.f, 0.f);
            if (jj < jc) {
              const int c = j0 + jj, n = (c >> 2) * 2 + (c & 1), st = half * Sh + n % Sh;
              const bool ab = __any_sync(0xffffffffu, abort_flag != 0);
              if (!ab && __all_sync(0xffffffffu, tc::mbar_wait(&sfull[st], (n / Sh) & 1))) {
                const unsigned char* sb = stages + (size_t)st * SL.stride;
                last_mode_staged((const float2*)(sb + SL.u1), B1p, il, (const float2*)(sb + SL.w), meta[st], u0,
                                 zz);
              } else if (!ab && lane == 0) {
                abort_flag = 1;
              }
              __syncwarp();
              if (lane == 0) mbar_arrive1(&sempty[st]);
            }
#pragma unroll
            for (int l = 0; l < kUQ; ++l) {
              x[l][2 * t] = zz[l].x;
              x[l][2 * t + 1] = zz[l].y;
            }
          }
          ensure_free();
          if (!__any_sync(0xffffffffu, abort_flag != 0)) {
            // reals 2 jj0 .. 2 jj0 + 3 of each row: 8 bytes (bf16) or 16 bytes (tf32) at
            const uint32_t kb = 2u * jj0 * F::esz;  // byte offset along K
#pragma unroll
            for (int l = 0; l < kUQ; ++l) {
              uint32_t t[F::terms][4];
              split_words<FMT, 4>(x[l], t);
              const int rho = Geo::row(tk, l, lane);
#pragma unroll
              for (int term = 0; term < F::terms; ++term) {
                const uint32_t addr = tc::smem_u32(a_op(buf, term)) + tc::core_off(rho, kb / 16, L.KBA) + kb % 16;
                if constexpr (F::esz == 2)
                  st_shared_v2(addr, t[term][0], t[term][1]);
                else
                  st_shared_v4(addr, t[term]);
              }
            }
          }
        }
      }
      // 4. B operand: rows n = 2s + e_out (P2 rows), K = 2*kChunk reals of this chunk
      ensure_free();
      if (!__any_sync(0xffffffffu, abort_flag != 0)) {
#pragma unroll
        for (int b = 0; b < kBMax; ++b) {
          const int e = tid + b * nprod;
          if (e < P2 * nk16) {
            const int n = e / nk16, kc = e % nk16;
            const int eo = n & 1;
            float x[NF];
#pragma unroll
            for (int i = 0; i < NF; ++i) {
              const float2 v = xv[b][i >> 1];
              x[i] = eo == (i & 1) ? v.x : (eo == 0 ? -v.y : v.y);
            }
            uint32_t t[F::terms][4];
            split_words<FMT, NF>(x, t);
#pragma unroll
            for (int term = 0; term < F::terms; ++term)
              st_shared_v4(tc::smem_u32(b_op(buf, term)) + tc::core_off(n, kc, L.KBA), t[term]);
          }
        }
      }
      tc::fence_proxy_async();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive1(&ofull[buf]);
    }
    // drain: the last commit covers every MMA
    {
      bool bad = abort_flag != 0;
      if (!bad && nchunks > 0) bad = !tc::mbar_wait(&oempty[(nchunks - 1) & 1], ((nchunks - 1) >> 1) & 1);
      if (__any_sync(0xffffffffu, bad) && lane == 0) abort_flag = 1;
    }
    tc::fence_after();
    if (!__any_sync(0xffffffffu, abort_flag != 0) && wg < ngroups) {
      const int64_t nv = (int64_t)g.n1 * g.n2 * g.n3;
      for (int m = wg; m < L.nmt; m += ngroups) {
        // row rho = 128 m + 32 wq + lane = (tk * kUQ + l) * 32 + lane
        const int rg = m * 4 + wq;
        const int tk = rg / kUQ, l = rg % kUQ;
        int ei1 = 0, eu0 = 0;
        bool eok = false;
        if (tk < g.ntask) g.task(i1_0, tk, lane, ei1, eu0, eok);
        const int u = eu0 + l;
        eok = eok && u < g.NU && (i2_0 + u) < g.n2;
        const int64_t v = ei1 + (int64_t)g.n1 * ((i2_0 + u) + (int64_t)g.n2 * i3);
        const uint32_t lanebase = (uint32_t)(wq * 32) << 16;
#pragma unroll 1
        for (int c0 = 0; c0 < P2; c0 += 16) {
          float vals[16];
          tc::tmem_ld16(tmem_d + lanebase + m * P2 + c0, vals);
          if (s_valid) {
            float sv[16];
            tc::tmem_ld16(tmem_s + lanebase + m * P2 + c0, sv);
#pragma unroll
            for (int i = 0; i < 16; ++i) vals[i] += sv[i];
          }
          if (eok) {
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
  if (threadIdx.x == 0 && abort_flag) atomicOr(err, kErrTimeout);
  if (warp == 0) tc::tmem_dealloc(tbase, L.tmem_cols);
}

template <int FMT, int P2>
static int launch_tc(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  using F = Fmt<FMT>;
  constexpr int P = P2 / 2;
  ZBC_TRY(build_decomp_cache(h, st));
  const int R = h.cache_r;
  const int B1p = tile_b1p(h.n1);
  // rows limited by TMEM (D and S: 2 * nmt * P2 <= 512), by the block (<= 8 producer warps) and
  // by shared memory (two operand buffers plus at least two stages); the largest tile that
  // fits is taken, and the stages get the rest of shared memory
  const int tmem_rows = 128 * std::max(1, 256 / P2);
  const size_t budget = 220 * 1024;
  Geo g;
  TcLayout L;
  StageLayout SL{};
  int S = 0;
  size_t sm = 0;
  for (int tasks = kTcMaxTasks; tasks >= 1 && S == 0; --tasks) {
    g = make_geo(h.n1, h.n2, h.n3, 0, tasks, tmem_rows);
    if (g.ntask > kTcMaxTasks) continue;
    L.NR = g.ntask * kUQ * 32;
    L.nmt = L.NR / 128;
    L.KBA = 2 * kChunk * F::esz / 16;
    L.a_bytes = L.NR * L.KBA * 16;
    L.b_bytes = P2 * L.KBA * 16;
    L.nprodw = std::max(4, 2 * g.ntask);
    SL = StageLayout::make(R, B1p, g.NUp, 0, 0);
    const size_t ops = 1024 + (size_t)F::terms * (L.a_bytes + L.b_bytes);
    if (ops + 2 * (size_t)SL.stride > budget) continue;
    S = (int)std::min<size_t>(kMaxStages, (budget - ops) / SL.stride) / 2 * 2;
    if (S < 4) {  // each producer half needs a ring of two stages at least
      S = 0;
      continue;
    }
    sm = (size_t)S * SL.stride + ops;
  }
  int cols = 32;
  while (cols < 2 * L.nmt * P2) cols <<= 1;
  L.tmem_cols = cols;
  if (S < 4 || cols > 512) {
    set_error("tensor-core layout does not fit (rank %d, tmem %d)", R, cols);
    return ZBC_EINVAL;
  }
  const float2* XT;
  int pst;
  ZBC_TRY(transpose_rhs(h, X, ldx, p, P, &XT, &pst, st));
  ZBC_TRY((set_smem_limit<matvec_tc_kernel<FMT, P2>>((int)budget)));
  dim3 grid(g.ntiles(), h.q, ceil_div(p, P));
  matvec_tc_kernel<FMT, P2><<<grid, 32 * (L.nprodw + 3), sm, st>>>(h.cache->data, h.cache->d_desc, g, h.q, h.M, SL,
                                                                   S, L, XT, pst, p, Y, ldy, (int*)h.work_err.ptr);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

template <int FMT>
static int matvec_tc_fmt(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  if (p <= 8) return launch_tc<FMT, 16>(h, X, ldx, p, Y, ldy, st);
  if (p <= 16) return launch_tc<FMT, 32>(h, X, ldx, p, Y, ldy, st);
  if (p <= 32) return launch_tc<FMT, 64>(h, X, ldx, p, Y, ldy, st);
  // 64 right-hand sides per CTA need D and S of 2 x 128 TMEM columns per 128 voxel rows, which
  // leaves room for two M tiles only: a tile whose i1 range has three 32-row groups does not
  // fit, and then the right-hand sides go 32 per CTA instead
  const int s = launch_tc<FMT, 128>(h, X, ldx, p, Y, ldy, st);
  if (s != ZBC_EINVAL) return s;
  clear_error();
  return launch_tc<FMT, 64>(h, X, ldx, p, Y, ldy, st);
}

int matvec_tc(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, zbc_precision prec,
              cudaStream_t st) {
  if (prec == ZBC_TF32X3) return matvec_tc_fmt<ZBC_TF32X3>(h, X, ldx, p, Y, ldy, st);
  return matvec_tc_fmt<ZBC_BF16X3>(h, X, ldx, p, Y, ldy, st);
}


}  // namespace zbc
