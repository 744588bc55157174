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
// Warp roles: the front-end ("producer") warps each own one task of the tile and fill the
// operands of a chunk; one extra warp issues the MMAs.  Two operand buffers alternate; an
// mbarrier "full" per buffer (one arrival per producer warp) hands a filled buffer to the
// issuer, and tcgen05.commit on an mbarrier "empty" per buffer hands it back once the tensor
// cores have consumed it.  Producers synchronise among themselves with a named barrier only.
#include <cuda_bf16.h>

#include <algorithm>

#include "decomp.cuh"
#include "tc_common.cuh"

namespace zbc {

constexpr int kFlush = 4;  // chunks accumulated in D before it is folded into S

struct TcPack {
  int dummy;
};
void tc_release(TcPack* p) { delete p; }

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

__device__ __forceinline__ void st_shared_v4(uint32_t addr, const uint32_t (&w)[4]) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
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
__global__ void __launch_bounds__(kThreads, 1)
    matvec_tc_kernel(const float2* __restrict__ cache, const CacheDesc* __restrict__ cdesc, Geo g, int q, int M,
                     int R, TcLayout L, const float2* __restrict__ X, int64_t ldx, int p, float2* __restrict__ Y,
                     int64_t ldy, int* __restrict__ err) {
  using F = Fmt<FMT>;
  constexpr int P = P2 / 2;
  constexpr int NF = 16 / F::esz;  // floats per 16-byte chunk
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t full[2], empty[2];
  __shared__ uint32_t tbase;
  __shared__ volatile int abort_flag;
  const FrontEnd2 fe(smem, R, g.NUp, kChunk * P);  // chunk c uses buffer c & 1
  unsigned char* ops = (unsigned char*)(((uintptr_t)fe.end() + 1023) & ~(uintptr_t)1023);
  auto a_op = [&](int buf, int term) { return ops + (size_t)(buf * F::terms + term) * L.a_bytes; };
  auto b_op = [&](int buf, int term) {
    return ops + (size_t)2 * F::terms * L.a_bytes + (size_t)(buf * F::terms + term) * L.b_bytes;
  };
  const int k = blockIdx.y;
  const int s0 = blockIdx.z * P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nprod = L.nprodw * 32;
  const int B1p = (g.B1 + 1) / 2 * 2;
  int i1_0, i2_0, i3;
  g.tile(blockIdx.x, i1_0, i2_0, i3);

  if (warp == 0) tc::tmem_alloc(&tbase, L.tmem_cols);
  if (threadIdx.x == 0) {
    tc::mbar_init(&full[0], L.nprodw);
    tc::mbar_init(&full[1], L.nprodw);
    tc::mbar_init(&empty[0], 1);
    tc::mbar_init(&empty[1], 1);
    abort_flag = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem_d = tbase;                           // D: nmt * P2 columns
  const uint32_t tmem_s = tbase + (uint32_t)(L.nmt * P2);  // S: nmt * P2 columns
  const int nchunks = (M + kChunk - 1) / kChunk;

  if (warp == L.nprodw) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = tc::instr_desc(128, P2, F::idfmt);
      const uint32_t sbo = L.KBA * 128;
      const int ksteps = L.KBA / 2;
      for (int c = 0; c < nchunks; ++c) {
        const int buf = c & 1;
        if (abort_flag || !tc::mbar_wait(&full[buf], (c >> 1) & 1)) {
          abort_flag = 1;
          break;
        }
        tc::fence_after();
        const bool fresh = (c % kFlush) == 0;
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
        tc::commit(&empty[buf]);
      }
    }
    __syncwarp();
  } else {
    // ---------------- producers ----------------
    const int tid = threadIdx.x;
    const int ngroups = L.nprodw / 4;  // warpgroups that fold and drain the accumulators
    const int wq = warp & 3, wg = warp >> 2;
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
    WPrefetch pf;
    pf.load(cache, cdesc, g, R, q, k, 0, min(kChunk, M), i2_0, i3, tid, nprod);
    for (int c = 0; c < nchunks; ++c) {
      const int buf = c & 1;
      const int j0 = c * kChunk;
      const int jc = min(kChunk, M - j0);
      const bool do_fold = c > 0 && (c % kFlush) == 0;
      const ChunkSmem cs = fe.cs(buf);
      float2* xs = fe.xs(buf);
      for (int e = tid; e < kChunk * P; e += nprod) {
        const int jj = e / P, i = e % P;
        xs[e] = (jj < jc && s0 + i < p) ? X[(j0 + jj) + ldx * (s0 + i)] : make_float2(0.f, 0.f);
      }
      pf.store(cs, g, R, jc, tid, nprod);
      bar_sync(1, nprod);
      if (j0 + kChunk < M)
        pf.load(cache, cdesc, g, R, q, k, j0 + kChunk, min(kChunk, M - j0 - kChunk), i2_0, i3, tid, nprod);
      if (c >= 2 || do_fold) {
        // operand buffer free once chunk c-2 is consumed; folding D needs chunk c-1 done
        const int wc = do_fold ? c - 1 : c - 2;
        if (!abort_flag && !tc::mbar_wait(&empty[wc & 1], (wc >> 1) & 1)) abort_flag = 1;
        tc::fence_after();
        if (do_fold && !abort_flag) {
          fold();
          s_valid = true;
        }
      }
      if (!abort_flag) {
        // B operand: rows n = 2s + e_out (P2 rows), K = 2*kChunk reals of this chunk
        const int nk16 = 2 * kChunk / NF;
        for (int e = tid; e < P2 * nk16; e += nprod) {
          const int n = e / nk16, kc = e % nk16;
          const int s = n >> 1, eo = n & 1;
          float x[NF];
#pragma unroll
          for (int i = 0; i < NF; ++i) {
            const int kk = kc * NF + i;
            const float2 v = xs[(kk >> 1) * P + s];
            const int ei = kk & 1;
            x[i] = eo == ei ? v.x : (eo == 0 ? -v.y : v.y);
          }
          uint32_t t[F::terms][4];
          split_words<FMT, NF>(x, t);
#pragma unroll
          for (int term = 0; term < F::terms; ++term)
            st_shared_v4(tc::smem_u32(b_op(buf, term)) + tc::core_off(n, kc, L.KBA), t[term]);
        }
        // A operand: rows of this warp's task (u = u0 + l, lane -> i1); K = 2*kChunk reals
        if (warp < g.ntask) {
          int i1, u0;
          bool ok;
          g.task(i1_0, warp, lane, i1, u0, ok);
          float z[kUQ][2 * kChunk];
#pragma unroll
          for (int jj = 0; jj < kChunk; ++jj) {
            float2 zz[kUQ];
            if (jj < jc) {
              const CacheDesc d = cs.cd[jj];
              const int t1 = i1_0 / g.B1, il = ok ? i1 - i1_0 : 0;
              last_mode4(cache + d.uoff + (int64_t)t1 * d.r1p * B1p + il, B1p, d.r1, ok,
                         cs.W + (size_t)jj * R * g.NUp, g.NUp, u0, zz);
            } else {
#pragma unroll
              for (int l = 0; l < kUQ; ++l) zz[l] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int l = 0; l < kUQ; ++l) {
              z[l][2 * jj] = zz[l].x;
              z[l][2 * jj + 1] = zz[l].y;
            }
          }
#pragma unroll
          for (int l = 0; l < kUQ; ++l) {
            const int rho = Geo::row(warp, l, lane);
#pragma unroll
            for (int kc = 0; kc < 2 * kChunk / NF; ++kc) {
              float x[NF];
#pragma unroll
              for (int i = 0; i < NF; ++i) x[i] = z[l][kc * NF + i];
              uint32_t t[F::terms][4];
              split_words<FMT, NF>(x, t);
#pragma unroll
              for (int term = 0; term < F::terms; ++term)
                st_shared_v4(tc::smem_u32(a_op(buf, term)) + tc::core_off(rho, kc, L.KBA), t[term]);
            }
          }
        }
      }
      tc::fence_proxy_async();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[buf]);
    }
    // drain: the last commit covers every MMA
    if (nchunks > 0 && !abort_flag &&
        !tc::mbar_wait(&empty[(nchunks - 1) & 1], ((nchunks - 1) >> 1) & 1))
      abort_flag = 1;
    tc::fence_after();
    if (!abort_flag && wg < ngroups) {
      const int64_t nv = (int64_t)g.n1 * g.n2 * g.n3;
      for (int m = wg; m < L.nmt; m += ngroups) {
        // row rho = 128 m + 32 wq + lane = (tk * kUQ + l) * 32 + lane
        const int rg = m * 4 + wq;
        const int tk = rg / kUQ, l = rg % kUQ;
        int i1 = 0, u0 = 0;
        bool ok = false;
        if (tk < g.ntask) g.task(i1_0, tk, lane, i1, u0, ok);
        const int u = u0 + l;
        ok = ok && u < g.NU && (i2_0 + u) < g.n2;
        const int64_t v = i1 + (int64_t)g.n1 * ((i2_0 + u) + (int64_t)g.n2 * i3);
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

template <int FMT, int P2>
static int launch_tc(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  using F = Fmt<FMT>;
  constexpr int P = P2 / 2;
  ZBC_TRY(build_decomp_cache(h, st));
  const int R = h.cache_r;
  // rows limited by TMEM (D and S: 2 * nmt * P2 <= 512), by two shared-memory A buffers and by
  // the block size (producer warps + the issuer <= 8); the largest tile that fits is taken.
  const int tmem_rows = 128 * std::max(1, 256 / P2);
  const size_t budget = 220 * 1024;
  Geo g;
  TcLayout L;
  size_t sm = 0;
  int tasks = 7;
  for (; tasks >= 1; --tasks) {
    g = make_geo(h.n1, h.n2, h.n3, R, tasks, tmem_rows);
    L.NR = g.ntask * kUQ * 32;
    L.nmt = L.NR / 128;
    L.KBA = 2 * kChunk * F::esz / 16;
    L.a_bytes = L.NR * L.KBA * 16;
    L.b_bytes = P2 * L.KBA * 16;
    L.nprodw = std::max(4, g.ntask);
    sm = 2 * FrontEnd2::buf_bytes(R, g.NUp, kChunk * P) + 1024 +
         (size_t)2 * F::terms * (L.a_bytes + L.b_bytes);
    if (sm <= budget && g.ntask <= 7) break;
  }
  int cols = 32;
  while (cols < 2 * L.nmt * P2) cols <<= 1;
  L.tmem_cols = cols;
  if (tasks < 1 || sm > budget || cols > 512) {
    set_error("tensor-core layout does not fit (rank %d, smem %zu, tmem %d)", R, sm, cols);
    return ZBC_EINVAL;
  }
  static bool attr_set = false;
  if (!attr_set) {
    ZBC_TRY_CUDA(cudaFuncSetAttribute(matvec_tc_kernel<FMT, P2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 221 * 1024));
    attr_set = true;
  }
  int* err = (int*)h.work_err.ptr;
  dim3 grid(g.ntiles(), h.q, ceil_div(p, P));
  matvec_tc_kernel<FMT, P2><<<grid, 32 * (L.nprodw + 1), sm, st>>>(h.cache->data, h.cache->d_desc, g, h.q, h.M, R, L,
                                                                   X, ldx, p, Y, ldy, err);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

template <int FMT>
static int matvec_tc_fmt(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  if (p <= 8) return launch_tc<FMT, 16>(h, X, ldx, p, Y, ldy, st);
  if (p <= 16) return launch_tc<FMT, 32>(h, X, ldx, p, Y, ldy, st);
  if (p <= 32) return launch_tc<FMT, 64>(h, X, ldx, p, Y, ldy, st);
  return launch_tc<FMT, 128>(h, X, ldx, p, Y, ldy, st);
}

int matvec_tc(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, zbc_precision prec,
              cudaStream_t st) {
  if (prec == ZBC_TF32X3) return matvec_tc_fmt<ZBC_TF32X3>(h, X, ldx, p, Y, ldy, st);
  return matvec_tc_fmt<ZBC_BF16X3>(h, X, ldx, p, Y, ldy, st);
}

int rmatvec_tc(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo, zbc_precision prec,
               cudaStream_t st) {
  set_error("tensor-core adjoint not built yet");
  return ZBC_EINVAL;
}

}  // namespace zbc
