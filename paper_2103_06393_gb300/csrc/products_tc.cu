// Tensor-core form of Algorithm 1 (Y = Z X, Sec. III.B) with tcgen05 on sm_103a.
//
// The decompression front end (decomp.cuh) produces, per chunk of 8 stored columns, the
// tile's decompressed block Z[rho, j] (rho = voxel row of the tile) on CUDA cores and writes
// it straight into shared memory as the A operand of a tcgen05 GEMM; the B operand is the
// matching chunk of X.  Both are complex and enter the MMA through the real embedding
//   A'[rho][2j + e] = (Re, Im) Z[rho, j],
//   B'^T[2s][2j] = Re X[j,s],  B'^T[2s][2j+1] = -Im X[j,s],
//   B'^T[2s+1][2j] = Im X[j,s], B'^T[2s+1][2j+1] = Re X[j,s],
// so that D[rho][2s + e] accumulates (Re, Im) Y[rho, s] in TMEM (FP32) across all chunks.
//
// Precision: FP32 values are split into tensor-core terms and the cross products above
// 2^-24 are accumulated (Fmt below):
//   TF32X3 : x = hi + lo (tf32), products hi*hi + hi*lo + lo*hi        (kind::tf32)
//   BF16X3 : x = hi + mid + lo (bf16), products hh hm mh hl lh mm       (kind::f16, bf16)
// Two operand buffers alternate: the CUDA cores fill one chunk while the tensor cores consume
// the previous one; an mbarrier per buffer (tcgen05.commit) guards the reuse.
#include <cuda_bf16.h>

#include <algorithm>

#include "decomp.cuh"
#include "tc_common.cuh"

namespace zbc {

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

// Split 2*NC floats (NC complex) into the format's terms, packed as 16-byte words per term.
// Output t[term][w] are 32-bit words: tf32 -> one float per word; bf16 -> two per word.
template <int FMT, int NF>
__device__ __forceinline__ void split_words(const float (&x)[NF], uint32_t (&t)[Fmt<FMT>::terms][NF * Fmt<FMT>::esz / 4]) {
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

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

struct TcLayout {
  int NR;        // accumulator rows of the tile (multiple of 128)
  int nmt;       // M tiles
  int KBA;       // 16-byte K chunks per operand row for one column chunk (= esz)
  int a_bytes;   // one term of one A buffer
  int b_bytes;   // one term of one B buffer
  int tmem_cols;
};

template <int FMT, int P2>
__global__ void __launch_bounds__(kThreads, 1)
    matvec_tc_kernel(const float2* __restrict__ pool, const TensorDesc* __restrict__ desc, Geo g, int q, int M,
                     int R, TcLayout L, const float2* __restrict__ X, int64_t ldx, int p, float2* __restrict__ Y,
                     int64_t ldy, int* __restrict__ err) {
  using F = Fmt<FMT>;
  constexpr int P = P2 / 2;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tbase;
  __shared__ int abort_flag;
  ChunkSmem cs;
  float2* xs = (float2*)cs.carve(smem, R, g.NU);              // [kChunk][P]
  unsigned char* ops = (unsigned char*)(xs + kChunk * P);
  ops = (unsigned char*)(((uintptr_t)ops + 1023) & ~(uintptr_t)1023);
  // A[buf][term] then B[buf][term]
  auto a_op = [&](int buf, int term) { return ops + (size_t)(buf * F::terms + term) * L.a_bytes; };
  auto b_op = [&](int buf, int term) {
    return ops + (size_t)2 * F::terms * L.a_bytes + (size_t)(buf * F::terms + term) * L.b_bytes;
  };
  const int k = blockIdx.y;
  const int s0 = blockIdx.z * P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int i1_0, i2_0, i3;
  g.tile(blockIdx.x, i1_0, i2_0, i3);

  // zero both A buffers once (padding rows stay zero), set up barriers and TMEM
  for (int e = threadIdx.x; e < 2 * F::terms * L.a_bytes / 16; e += blockDim.x)
    reinterpret_cast<uint4*>(ops)[e] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tc::tmem_alloc(&tbase, L.tmem_cols);
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    abort_flag = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tbase;
  const uint32_t idesc = tc::instr_desc(128, P2, F::idfmt);
  const int nchunks = (M + kChunk - 1) / kChunk;
  const uint32_t sbo_a = L.KBA * 128, sbo_b = L.KBA * 128;

  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    const int j0 = c * kChunk;
    const int jc = min(kChunk, M - j0);
    if (c >= 2) {
      if (threadIdx.x == 0) {
        if (!tc::mbar_wait(&mbar[buf], ((c - 2) >> 1) & 1)) abort_flag = 1;
      }
      __syncthreads();
      if (abort_flag) break;
      tc::fence_after();
    }
    for (int e = threadIdx.x; e < kChunk * P; e += blockDim.x) {
      const int jj = e / P, i = e % P;
      xs[e] = (jj < jc && s0 + i < p) ? X[(j0 + jj) + ldx * (s0 + i)] : make_float2(0.f, 0.f);
    }
    chunk_pw(pool, desc, g, q, k, j0, jc, R, i2_0, i3, cs);
    // B operand: rows n = 2s + e_out (P2 rows), K = 2*kChunk reals of this chunk
    {
      constexpr int NF = 16 / F::esz;  // floats per 16-byte chunk
      const int nchunk16 = 2 * kChunk / NF;
      for (int e = threadIdx.x; e < P2 * nchunk16; e += blockDim.x) {
        const int n = e / nchunk16, kc = e % nchunk16;
        const int s = n >> 1, eo = n & 1;
        float x[NF];
#pragma unroll
        for (int i = 0; i < NF; ++i) {
          const int kk = kc * NF + i;
          const int jj = kk >> 1, ei = kk & 1;
          const float2 v = xs[jj * P + s];
          // (eo, ei): (0,0) Re, (0,1) -Im, (1,0) Im, (1,1) Re
          x[i] = eo == ei ? v.x : (eo == 0 ? -v.y : v.y);
        }
        uint32_t t[F::terms][4];
        split_words<FMT, NF>(x, t);
#pragma unroll
        for (int term = 0; term < F::terms; ++term)
          st_shared_v4(tc::smem_u32(b_op(buf, term)) + tc::core_off(n, kc, L.KBA), t[term][0], t[term][1], t[term][2],
                       t[term][3]);
      }
    }
    // A operand: row rho = 32*lane_group + lane, K = 2*kChunk reals
#pragma unroll 1
    for (int l = 0; l < kMaxLG; ++l) {
      const int gi = warp + 8 * l;
      if (gi >= g.nlg) break;
      int i1, u;
      const bool ok = g.voxel(i1_0, i2_0, gi, lane, i1, u);
      float z[2 * kChunk];
#pragma unroll
      for (int jj = 0; jj < kChunk; ++jj) {
        float2 v = make_float2(0.f, 0.f);
        if (ok && jj < jc) {
          const TensorDesc d = cs.jd[jj];
          v = last_mode(pool + d.off + (int64_t)d.r1 * d.r2 * d.r3, g.n1, d.r1, i1, cs.W + (size_t)jj * R * g.NU, R,
                        g.NU, u);
        }
        z[2 * jj] = v.x;
        z[2 * jj + 1] = v.y;
      }
      const int rho = gi * 32 + lane;
      constexpr int NF = 16 / F::esz;
#pragma unroll
      for (int kc = 0; kc < 2 * kChunk / NF; ++kc) {
        float x[NF];
#pragma unroll
        for (int i = 0; i < NF; ++i) x[i] = z[kc * NF + i];
        uint32_t t[F::terms][4];
        split_words<FMT, NF>(x, t);
#pragma unroll
        for (int term = 0; term < F::terms; ++term)
          st_shared_v4(tc::smem_u32(a_op(buf, term)) + tc::core_off(rho, kc, L.KBA), t[term][0], t[term][1],
                       t[term][2], t[term][3]);
      }
    }
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after();
      const int ksteps = L.KBA / 2;
#pragma unroll 1
      for (int m = 0; m < L.nmt; ++m) {
#pragma unroll
        for (int pr = 0; pr < F::nprod; ++pr) {
          const uint32_t abase = tc::smem_u32(a_op(buf, F::pa(pr))) + m * 16 * sbo_a;
          const uint32_t bbase = tc::smem_u32(b_op(buf, F::pb(pr)));
          for (int ks = 0; ks < ksteps; ++ks) {
            const uint64_t ad = tc::smem_desc(abase + ks * 256, 128, sbo_a);
            const uint64_t bd = tc::smem_desc(bbase + ks * 256, 128, sbo_b);
            tc::mma<F::kind>(tmem + m * P2, ad, bd, idesc, (c > 0 || pr > 0 || ks > 0) ? 1u : 0u);
          }
        }
      }
      tc::commit(&mbar[buf]);
    }
  }
  // wait for the last chunk's MMAs (their completion implies all earlier ones)
  if (threadIdx.x == 0 && !abort_flag && nchunks > 0) {
    if (!tc::mbar_wait(&mbar[(nchunks - 1) & 1], ((nchunks - 1) >> 1) & 1)) abort_flag = 1;
  }
  __syncthreads();
  tc::fence_after();
  if (abort_flag) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else {
    const int64_t nv = (int64_t)g.n1 * g.n2 * g.n3;
    const int wq = warp & 3;
    for (int m = warp >> 2; m < L.nmt; m += 2) {
      const int rho = m * 128 + wq * 32 + lane;
      const int gi = rho >> 5;
      int i1, u;
      const bool ok = gi < g.nlg && g.voxel(i1_0, i2_0, gi, lane, i1, u);
      const int64_t v = i1 + (int64_t)g.n1 * ((i2_0 + u) + (int64_t)g.n2 * i3);
#pragma unroll
      for (int c0 = 0; c0 < P2; c0 += 16) {
        float vals[16];
        tc::tmem_ld16(tmem + ((uint32_t)(wq * 32) << 16) + m * P2 + c0, vals);
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
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, L.tmem_cols);
}

template <int FMT, int P2>
static int launch_tc(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  using F = Fmt<FMT>;
  constexpr int P = P2 / 2;
  const int R = std::max(h.max_rank, 1);
  // rows limited by TMEM (nmt * P2 <= 512) and by shared memory for two buffers of A
  const int tmem_rows = 128 * std::max(1, 512 / P2);
  const size_t fixed = ChunkSmem::bytes(R, 32) + sizeof(float2) * kChunk * P + 1024 +
                       (size_t)2 * F::terms * P2 * (2 * kChunk * F::esz);
  const size_t budget = 220 * 1024;
  if (fixed >= budget) {
    set_error("tensor-core path: rank %d too large", R);
    return ZBC_EINVAL;
  }
  const int smem_rows = (int)((budget - fixed) / ((size_t)2 * F::terms * 2 * kChunk * F::esz)) / 128 * 128;
  const int max_rows = std::min(tmem_rows, smem_rows);
  if (max_rows < 128) {
    set_error("tensor-core path: shared memory too small for rank %d", R);
    return ZBC_EINVAL;
  }
  Geo g = make_geo(h.n1, h.n2, h.n3, max_rows);
  TcLayout L;
  L.NR = ceil_div(g.nlg * 32, 128) * 128;
  L.nmt = L.NR / 128;
  L.KBA = 2 * kChunk * F::esz / 16;
  L.a_bytes = L.NR * L.KBA * 16;
  L.b_bytes = P2 * L.KBA * 16;
  int cols = 32;
  while (cols < L.nmt * P2) cols <<= 1;
  L.tmem_cols = cols;
  const size_t sm = ChunkSmem::bytes(R, g.NU) + sizeof(float2) * kChunk * P + 1024 +
                    (size_t)2 * F::terms * (L.a_bytes + L.b_bytes);
  if (sm > budget || cols > 512) {
    set_error("tensor-core layout does not fit (smem %zu, tmem %d)", sm, cols);
    return ZBC_EINVAL;
  }
  static bool attr_set = false;
  if (!attr_set) {
    ZBC_TRY_CUDA(cudaFuncSetAttribute(matvec_tc_kernel<FMT, P2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 221 * 1024));
    attr_set = true;
  }
  ZBC_TRY(h.work_misc.ensure(sizeof(int)));
  int* err = (int*)h.work_misc.ptr;
  ZBC_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  dim3 grid(g.ntiles(), h.q, ceil_div(p, P));
  matvec_tc_kernel<FMT, P2><<<grid, kThreads, sm, st>>>(h.d_pool, h.d_desc, g, h.q, h.M, R, L, X, ldx, p, Y, ldy, err);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

template <int FMT>
static int matvec_tc_fmt(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  if (p <= 8) return launch_tc<FMT, 16>(h, X, ldx, p, Y, ldy, st);
  if (p <= 16) return launch_tc<FMT, 32>(h, X, ldx, p, Y, ldy, st);
  if (p <= 32) return launch_tc<FMT, 64>(h, X, ldx, p, Y, ldy, st);
  if (p <= 64) return launch_tc<FMT, 128>(h, X, ldx, p, Y, ldy, st);
  return launch_tc<FMT, 256>(h, X, ldx, p, Y, ldy, st);
}

int matvec_tc(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, zbc_precision prec,
              cudaStream_t st) {
  if (prec == ZBC_TF32X3) return matvec_tc_fmt<ZBC_TF32X3>(h, X, ldx, p, Y, ldy, st);
  return matvec_tc_fmt<ZBC_BF16X3>(h, X, ldx, p, Y, ldy, st);
}

int rmatvec_simt(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo, cudaStream_t st);

int rmatvec_tc(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo, zbc_precision prec,
               cudaStream_t st) {
  set_error("tensor-core adjoint not built yet");
  return ZBC_EINVAL;
}

}  // namespace zbc
