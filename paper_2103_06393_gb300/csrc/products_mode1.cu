// Adjoint product (Algorithm 2, Sec. III.B) with the mode-1 product on the tensor cores.
//
// With Z^{kj}[i1, i23] = sum_a U1_{kj}[i1, a] W_{kj}[i23, a]  (i23 = i2 + n2 i3, W = G x2 U2 x3 U3,
// the decompression cache of decomp_cache.cu), the adjoint regroups as
//   Psi_j[s] = sum_k sum_a sum_i23 conj(W_{kj}[i23, a]) T_{kja}[i23, s],
//   T_{kja}[i23, s] = sum_i1 conj(U1_{kj}[i1, a]) Phi^k[i1 + n1 i23, s],
// i.e. Phi^k is first projected onto the mode-1 factors.  Stacking the (column j, rank a) pairs
// of component k as rows, 128 to a group, the projection is one dense GEMM per group,
//   T[(j, a)][(i23, s)] = U1^H [128 x n1] . Phi^k [n1 x (n2 n3 p)],
// which runs on tcgen05; the remaining sum over (a, i23) is a short epilogue on CUDA cores that
// reads T from tensor memory.  Per (row, i23, s) it costs one complex multiply-add, against
// r1 + p of the decompress-then-contract form (products_simt.cu), and the GEMM carries the
// rest: the tensor cores do ~r1 times the flops of Table III's count, at ~25 times the FP32 rate.
//
// Real embedding (K = 2 i1 + e', both operands K-major):
//   A[(j, a)][2 i1 + e'] = (Re, Im) U1[i1, a]                     (tensor memory, per group)
//   B[2 (i23l P + s) + 0][2 i1 + e'] = (Re, Im) Phi[i1, i23, s]   -> D = Re T
//   B[2 (i23l P + s) + 1][2 i1 + e'] = (Im, -Re) Phi[i1, i23, s]  -> D = Im T
// Precision: both operands are split into fp16 hi + lo (x = hi + lo to ~2^-22 relative), after
// scaling by powers of two into fp16's normal range -- per row of A (2^(kHalfShift - uexp)) and
// per (N block, right-hand side) of B (2^(kHalfShift - e)) -- and the three products
// hi.hi + hi.lo + lo.hi accumulate in FP32 over K = 2 n1 (at most 2 x 224 per sum); the scales
// are removed exactly in the epilogue.
//
// Kernels, per call:
//   phi_split_kernel      Phi -> the B operand blocks (fp16 hi / lo, one contiguous run per
//                         (component, RHS chunk, N block, K chunk)) and the exponents
//   rmatvec_mode1_kernel  persistent, one CTA per SM; items (RHS chunk, N range, i1 tile, group):
//                         epilogue warps (A into TMEM, T . conj(W) sums), a copy warp
//                         (cp.async.bulk of the B blocks into a stage ring) and an MMA warp
//                         (A from TMEM, B from shared memory, D in TMEM: N = 256 or 192 columns
//                         with one buffer and two epilogue warpgroups, else two buffers)
//   mode1_reduce_kernel   Psi'[j, s] = sum over the partial slots (N ranges, i1 tiles, epilogue
//                         warpgroups), components and ranks, in a fixed order
// plus, once per handle, mode1_build_kernel (the A operand and the row table).
#include <cuda_fp16.h>

#include <algorithm>

#include "mode1.cuh"

namespace zbc {

void mode1_release(Mode1Cache* c) {
  if (!c) return;
  for (void* ptr : {(void*)c->A, (void*)c->rows, (void*)c->kg_k, (void*)c->colrows, (void*)c->rowsrc, (void*)c->Bf,
                    (void*)c->Wc, (void*)c->ew, (void*)c->chunkinfo, (void*)c->jtab, (void*)c->d_chbase})
    if (ptr) cudaFree(ptr);
  delete c;
}

// One thread per row (j, a): exponent of U1[:, a], then the scaled fp16 hi / lo split.
__global__ void __launch_bounds__(128) mode1_build_kernel(const float2* __restrict__ pool,
                                                          const TensorDesc* __restrict__ desc,
                                                          const int4* __restrict__ rowsrc, int n1, int n1p,
                                                          uint32_t* __restrict__ A, Mode1Row* __restrict__ rows) {
  const int kg = blockIdx.x, l = threadIdx.x;
  const int4 src = rowsrc[(int64_t)kg * kM1Rows + l];
  const float2* U1 = nullptr;
  float mx = 0.f;
  if (src.z) {
    const TensorDesc d = desc[src.x];
    U1 = pool + d.off + (int64_t)d.r1 * d.r2 * d.r3 + (int64_t)n1 * src.y;
    for (int i1 = 0; i1 < n1; ++i1) {
      const float2 u = U1[i1];
      mx = fmaxf(mx, fmaxf(fabsf(u.x), fabsf(u.y)));
    }
  }
  int uexp = 0;
  frexpf(mx, &uexp);  // mx < 2^uexp (mx = 0 gives 0)
  if (src.z) rows[(int64_t)kg * kM1Rows + l].uexp = uexp;
  const int sh = kHalfShift - uexp;
  for (int i1 = 0; i1 < n1p; ++i1) {
    const float2 u = (U1 && i1 < n1) ? U1[i1] : make_float2(0.f, 0.f);
    const float xr = ldexpf(u.x, sh), xi = ldexpf(u.y, sh);
    const __half hr = __float2half_rn(xr), hi = __float2half_rn(xi);
    const __half lr = __float2half_rn(xr - __half2float(hr)), li = __float2half_rn(xi - __half2float(hi));
    const __half2 vh = __halves2half2(hr, hi), vl = __halves2half2(lr, li);
    const int64_t base = ((int64_t)kg * 2 * (n1p / 4) + i1 / 4) * (kM1Rows * 4) + l * 4 + (i1 & 3);
    A[base] = *reinterpret_cast<const uint32_t*>(&vh);
    A[base + (int64_t)(n1p / 4) * (kM1Rows * 4)] = *reinterpret_cast<const uint32_t*>(&vl);
  }
}

int64_t cache_bytes(const DecompCache* c) {
  if (!c) return 0;
  return c->bytes + (c->mode1 ? c->mode1->bytes : 0) + dc_bytes(c->dc);
}

int build_mode1_cache(Handle& h, cudaStream_t st) {
  ZBC_TRY(build_decomp_cache(h, st));
  DecompCache& dc = *h.cache;
  if (dc.mode1) return ZBC_OK;
  const int q = h.q, M = h.M;
  std::vector<int> gbase(q + 1, 0);
  for (int k = 0; k < q; ++k) {
    int64_t R = 0;
    for (int j = 0; j < M; ++j) R += h.desc[(size_t)j * q + k].r1;
    gbase[k + 1] = gbase[k] + (int)((R + kM1Rows - 1) / kM1Rows);
  }
  const int KG = gbase[q];
  if (KG == 0) {
    set_error("mode-1 adjoint: the handle has no rows");
    return ZBC_EINVAL;
  }
  std::vector<Mode1Row> rows((size_t)KG * kM1Rows, Mode1Row{-1, 0, 0});
  std::vector<int4> src((size_t)KG * kM1Rows, make_int4(0, 0, 0, 0));
  std::vector<int> kg_k(KG);
  std::vector<int2> colrows((size_t)M * q);
  for (int k = 0; k < q; ++k) {
    for (int g = gbase[k]; g < gbase[k + 1]; ++g) kg_k[g] = k;
    int64_t r = (int64_t)gbase[k] * kM1Rows;
    for (int j = 0; j < M; ++j) {
      const int t = j * q + k;
      const CacheDesc& cd = dc.host_desc[t];
      colrows[t] = make_int2((int)r, cd.r1);
      for (int a = 0; a < cd.r1; ++a, ++r) {
        rows[r] = Mode1Row{cd.woff + a, cd.r1p, 0};
        src[r] = make_int4(t, a, 1, 0);
      }
    }
  }
  auto* c = new Mode1Cache();
  c->KG = KG;
  c->gbase = gbase;
  c->n1p = (h.n1 + 7) / 8 * 8;
  const size_t abytes = sizeof(uint32_t) * (size_t)KG * 2 * c->n1p * kM1Rows;
  cudaError_t e = cudaMalloc(&c->A, abytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->rows, sizeof(Mode1Row) * rows.size());
  if (e == cudaSuccess) e = cudaMalloc(&c->kg_k, sizeof(int) * KG);
  if (e == cudaSuccess) e = cudaMalloc(&c->colrows, sizeof(int2) * colrows.size());
  if (e == cudaSuccess) e = cudaMalloc(&c->rowsrc, sizeof(int4) * src.size());
  if (e == cudaSuccess)
    c->bytes = (int64_t)(abytes + sizeof(Mode1Row) * rows.size() + sizeof(int) * KG + sizeof(int2) * colrows.size() +
                         sizeof(int4) * src.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->rows, rows.data(), sizeof(Mode1Row) * rows.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->kg_k, kg_k.data(), sizeof(int) * KG, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->colrows, colrows.data(), sizeof(int2) * colrows.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->rowsrc, src.data(), sizeof(int4) * src.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    mode1_build_kernel<<<KG, kM1Rows, 0, st>>>(h.d_pool, h.d_desc, c->rowsrc, h.n1, c->n1p, c->A, c->rows);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors go out of scope
  if (e != cudaSuccess) {
    mode1_release(c);
    set_error("mode-1 adjoint cache build failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? ZBC_ENOMEM : ZBC_ECUDA;
  }
  dc.mode1 = c;
  return ZBC_OK;
}

// B operand geometry of one call: N blocks of NB rows (I = NB / (2P) values of i23, each with P
// right-hand sides times (Re, Im) rows), K in nkc chunks of KC = 32 i1 (64 fp16 = one 128-byte
// swizzled row; the last chunk's K steps stop at n1p, its tail is zero).
struct M1Geo {
  int P, NB, I;       // RHS per pass, rows per N block, i23 per N block
  int nsc;            // passes over the right-hand sides (ceil(p / P))
  int n23, NBT;       // n2 n3, N blocks per (component, pass)
  int n1, n1p, KC, nkc;
  int nkt, ntile1;     // K chunks per i1 tile, i1 tiles (A of one tile sits in TMEM at a time)
  uint32_t chunk_u32;  // one term of one K chunk: NB * KC 32-bit words
  __host__ __device__ int64_t block_u32(int k, int sc, int nb, int c) const {
    return ((((int64_t)k * nsc + sc) * NBT + nb) * nkc + c) * 2 * chunk_u32;
  }
  // exponent of (component, pass, N block, right-hand side of the pass)
  __host__ __device__ int64_t exp_index(int k, int sc, int nb, int s) const {
    return (((int64_t)k * nsc + sc) * NBT + nb) * P + s;
  }
};

// One CTA per (N block, pass, component).  The largest |Re|, |Im| of each right-hand side over
// the block fixes that right-hand side's exponent e (max < 2^e), so right-hand sides of very
// different magnitudes keep their accuracy; then each thread writes 16-byte pieces (4 i1 of
// one row, both terms) in the 128-byte swizzled K-major layout (tc::sw128_off; 8 pieces per
// row per chunk).
__global__ void __launch_bounds__(256) phi_split_kernel(const float2* __restrict__ Phi, int64_t ldphi, int p,
                                                        int64_t nv, M1Geo G, uint32_t* __restrict__ Bop,
                                                        int* __restrict__ Eblk, int* __restrict__ err) {
  const int nb = blockIdx.x, sc = blockIdx.y, k = blockIdx.z;
  const int KB4 = G.KC / 4;
  const int npiece = G.NB * G.nkc * KB4;
  __shared__ unsigned int smax[kM1MaxP];  // float bits of non-negative maxima (ordered as integers)
  __shared__ int sexp[kM1MaxP];
  // piece index -> (chunk c, row n, piece kc within the row's chunk), ordered by output address
  auto decode = [&](int pi, int& c, int& n, int& kc) {
    const int r8 = pi & 7;
    const int rest = pi >> 3;
    kc = rest % KB4;
    const int ng = (rest / KB4) % (G.NB / 8);
    c = rest / (KB4 * (G.NB / 8));
    n = ng * 8 + r8;
  };
  auto source = [&](int n, int c, int kc, int& i1, int64_t& off) {  // false: a padding piece
    const int i23 = nb * G.I + n / (2 * G.P);
    const int s = sc * G.P + (n >> 1) % G.P;
    i1 = c * G.KC + kc * 4;
    off = (int64_t)k * nv + (int64_t)G.n1 * i23 + ldphi * s;
    return i23 < G.n23 && s < p;
  };
  if (threadIdx.x < kM1MaxP) smax[threadIdx.x] = 0u;
  __syncthreads();
  for (int pi = threadIdx.x; pi < npiece; pi += blockDim.x) {
    int c, n, kc, i1;
    int64_t off;
    decode(pi, c, n, kc);
    if ((n & 1) || !source(n, c, kc, i1, off)) continue;
    float mx = 0.f;
    bool finite = true;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (i1 + i < G.n1) {
        const float2 v = Phi[off + i1 + i];
        finite = finite && isfinite(v.x) && isfinite(v.y);
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
    if (!finite) atomicOr(err, kErrNonFinite);  // the exponents below then mean nothing
    if (mx > 0.f) atomicMax(&smax[(n >> 1) % G.P], __float_as_uint(mx));
  }
  __syncthreads();
  if (threadIdx.x < G.P) {
    int e = 0;
    frexpf(__uint_as_float(smax[threadIdx.x]), &e);
    sexp[threadIdx.x] = e;
    Eblk[G.exp_index(k, sc, nb, threadIdx.x)] = e;
  }
  __syncthreads();
  uint32_t* out = Bop + G.block_u32(k, sc, nb, 0);
  for (int pi = threadIdx.x; pi < npiece; pi += blockDim.x) {
    int c, n, kc, i1;
    int64_t off;
    decode(pi, c, n, kc);
    uint32_t hw[4], lw[4];
    const bool ok = source(n, c, kc, i1, off);
    const int sh = kHalfShift - sexp[(n >> 1) % G.P];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 v = (ok && i1 + i < G.n1) ? Phi[off + i1 + i] : make_float2(0.f, 0.f);
      if (n & 1) v = make_float2(v.y, -v.x);  // the Im T row
      const float xr = ldexpf(v.x, sh), xi = ldexpf(v.y, sh);
      const __half hr = __float2half_rn(xr), hi = __float2half_rn(xi);
      const __half lr = __float2half_rn(xr - __half2float(hr)), li = __float2half_rn(xi - __half2float(hi));
      const __half2 vh = __halves2half2(hr, hi), vl = __halves2half2(lr, li);
      hw[i] = *reinterpret_cast<const uint32_t*>(&vh);
      lw[i] = *reinterpret_cast<const uint32_t*>(&vl);
    }
    // chunk c, term t: (c * 2 + t) * chunk_u32; piece (n, kc) at sw128_off(n, kc) bytes
    const int64_t o = (int64_t)c * 2 * G.chunk_u32 + tc::sw128_off(n, kc) / 4;
    *reinterpret_cast<uint4*>(out + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(out + o + G.chunk_u32) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint4 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}



struct M1Params {
  const uint32_t* A;
  const Mode1Row* rows;
  const int* kg_k;
  const float2* W;  // decompression cache
  const uint32_t* Bop;
  const int* Eblk;
  float2* partial;  // [NR * ntile1 * EG slots][KG * 128][ppad]
  int* err;
  M1Geo G;
  int KG, NR, S, ppad;
  uint32_t tcols;   // allocated TMEM columns
  int64_t nitems;   // nsc * NR * ntile1 * KG
};

// item -> (pass sc, N range nr, i1 tile t1, group kg); groups vary fastest, so the CTAs running
// at one time share their N range and tile and read the same B blocks (from L2)
__device__ __forceinline__ void m1_item(const M1Params& prm, int64_t it, int& sc, int& nr, int& t1, int& kg, int& nb0,
                                        int& nb1) {
  kg = (int)(it % prm.KG);
  int64_t t = it / prm.KG;
  t1 = (int)(t % prm.G.ntile1);
  t /= prm.G.ntile1;
  nr = (int)(t % prm.NR);
  sc = (int)(t / prm.NR);
  nb0 = (int)((int64_t)prm.G.NBT * nr / prm.NR);
  nb1 = (int)((int64_t)prm.G.NBT * (nr + 1) / prm.NR);
}

// Shape of the main kernel for NB rows per N block: two D buffers while they fit beside A in
// tensor memory (NB <= 160), else one buffer of 192 or 256 columns drained by two epilogue
// warpgroups at once (each takes half of its columns), so that it is handed back after a single
// round of TMEM loads.  Fewer, larger MMAs are what matters: an MMA costs at least ~95 cycles
// to issue whatever its N.
template <int NB>
struct M1Shape {
  static constexpr int DB = NB > 160 ? 1 : 2;       // D buffers
  static constexpr int EG = NB > 160 ? 2 : 1;       // epilogue warpgroups
  static constexpr int threads = 32 * (4 * EG + 2);  // + the copy warp and the MMA warp
};

template <int P, int NB>
__global__ void __launch_bounds__(M1Shape<NB>::threads, 1) rmatvec_mode1_kernel(const M1Params prm) {
  using Sh = M1Shape<NB>;
  constexpr int DB = Sh::DB, EG = Sh::EG;
  constexpr int I = NB / (2 * P);     // i23 per N block
  constexpr int NC = NB / EG;         // D columns per epilogue warpgroup
  constexpr int IW = NC / (2 * P) > 0 ? NC / (2 * P) : 1;  // i23 per warpgroup
  static_assert(NC % (2 * P) == 0, "a warpgroup's columns are whole i23 values");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t sfull[kM1MaxStages], sempty[kM1MaxStages], dfull[2], dempty[2], afull;
  __shared__ uint32_t tbase;
  __shared__ volatile int abort_flag;
  unsigned char* stages = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const M1Geo& G = prm.G;
  const int S = prm.S;
  const uint32_t stage_bytes = 8u * G.chunk_u32;  // both terms of one K chunk
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int copy_warp = 4 * EG, mma_warp = 4 * EG + 1;

  if (warp == 0) tc::tmem_alloc(&tbase, prm.tcols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&sfull[s], 1);
      tc::mbar_init(&sempty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&dfull[b], 1);
      tc::mbar_init(&dempty[b], 4 * EG);
    }
    tc::mbar_init(&afull, 4 * EG);
    abort_flag = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tD = tbase;               // D buffers: columns [b NB, (b + 1) NB)
  const uint32_t tAw = (uint32_t)G.nkt * G.KC;  // TMEM columns of one term of a tile's A
  const uint32_t tA = tbase + DB * NB;          // A: hi in [DB NB, DB NB + tAw), lo after it

  if (warp == copy_warp) {
    // ---------------- copy warp: B blocks into the stage ring ----------------
    if (lane == 0) {
      uint32_t cnt = 0;
      for (int64_t it = blockIdx.x; it < prm.nitems && !abort_flag; it += gridDim.x) {
        int sc, nr, t1, kg, nb0, nb1;
        m1_item(prm, it, sc, nr, t1, kg, nb0, nb1);
        const int c_lo = t1 * G.nkt, c_hi = min(G.nkc, c_lo + G.nkt);
        const int k = prm.kg_k[kg];
        for (int nb = nb0; nb < nb1 && !abort_flag; ++nb)
          for (int c = c_lo; c < c_hi; ++c, ++cnt) {
            const int st = cnt % S;
            if (cnt >= (uint32_t)S && (abort_flag || !tc::mbar_wait(&sempty[st], ((cnt / S) - 1) & 1))) {
              abort_flag = 1;
              break;
            }
            mbar_arrive_expect_tx(&sfull[st], stage_bytes);
            bulk_g2s(stages + (size_t)st * stage_bytes, prm.Bop + G.block_u32(k, sc, nb, c), stage_bytes,
                     &sfull[st]);
          }
      }
      if (abort_flag)  // let the copies in flight land before the CTA exits
        for (uint32_t c = cnt > (uint32_t)S ? cnt - S : 0; c < cnt; ++c) tc::mbar_wait(&sfull[c % S], (c / S) & 1);
    }
    __syncwarp();
  } else if (warp == mma_warp) {
    // ---------------- MMA warp ----------------
    if (lane == 0) {
      const uint32_t idesc = tc::instr_desc(128, NB, 0);  // kind::f16, f16 operands, FP32 D
      uint32_t cnt = 0, dc = 0, ai = 0;
      for (int64_t it = blockIdx.x; it < prm.nitems && !abort_flag; it += gridDim.x, ++ai) {
        int sc, nr, t1, kg, nb0, nb1;
        m1_item(prm, it, sc, nr, t1, kg, nb0, nb1);
        const int c_lo = t1 * G.nkt, c_hi = min(G.nkc, c_lo + G.nkt);
        if (!tc::mbar_wait(&afull, ai & 1)) {
          abort_flag = 1;
          break;
        }
        tc::fence_after();
        for (int nb = nb0; nb < nb1 && !abort_flag; ++nb, ++dc) {
          const int buf = dc % DB;
          const uint32_t use = dc / DB;  // the use-th fill of this D buffer
          if (use >= 1 && !tc::mbar_wait(&dempty[buf], (use - 1) & 1)) {
            abort_flag = 1;
            break;
          }
          tc::fence_after();
          const uint32_t d = tD + buf * NB;
          for (int c = c_lo; c < c_hi; ++c, ++cnt) {
            const int st = cnt % S;
            if (!tc::mbar_wait(&sfull[st], (cnt / S) & 1)) {
              abort_flag = 1;
              break;
            }
            tc::fence_after();
            const int ksn = min(G.KC, G.n1p - c * G.KC) / 8;
            const uint32_t cofs = (uint32_t)(c - c_lo) * G.KC;  // the chunk's first column in A
            const uint32_t sb = tc::smem_u32(stages + (size_t)st * stage_bytes);
            for (int ks = 0; ks < ksn; ++ks) {
              const uint32_t acol = cofs + 8 * ks;
              const uint64_t bh = tc::smem_desc_sw128(sb + ks * 32);
              const uint64_t bl = tc::smem_desc_sw128(sb + 4u * G.chunk_u32 + ks * 32);
              tc::mma_ts(d, tA + acol, bh, idesc, (c != c_lo || ks != 0) ? 1u : 0u);  // hi . hi
              tc::mma_ts(d, tA + acol, bl, idesc, 1u);               // hi . lo
              tc::mma_ts(d, tA + tAw + acol, bh, idesc, 1u);         // lo . hi
            }
            tc::commit(&sempty[st]);
          }
          if (abort_flag) break;
          tc::commit(&dfull[buf]);
        }
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue warps: A into TMEM, then sum_i23 conj(W) T per row ----------------
    const int eg = warp / 4;                  // epilogue warpgroup: D columns [eg NC, (eg + 1) NC)
    const int l = (warp % 4) * 32 + lane;     // row of the group = TMEM lane
    const uint32_t lanebase = (uint32_t)((warp % 4) * 32) << 16;
    uint32_t dc = 0;
    for (int64_t it = blockIdx.x; it < prm.nitems; it += gridDim.x) {
      if (__any_sync(0xffffffffu, abort_flag != 0)) break;
      int sc, nr, t1, kg, nb0, nb1;
      m1_item(prm, it, sc, nr, t1, kg, nb0, nb1);
      const int k = prm.kg_k[kg];
      // A of group kg on the item's i1 tile, the warpgroups splitting its columns; the previous
      // item's MMAs are complete (its last D fill was drained, and that fill's commit came after
      // all of them)
      {
        const int i_lo = t1 * G.nkt * G.KC, i_hi = min(G.n1p, i_lo + G.nkt * G.KC);
        const int nloc = (i_hi - i_lo) / 4;  // 4-column blocks per term
        const uint4* src = reinterpret_cast<const uint4*>(prm.A) + (int64_t)kg * 2 * (G.n1p / 4) * kM1Rows + l;
        const int ncb = 2 * nloc;
        const int cb_lo = ncb * eg / EG, cb_hi = ncb * (eg + 1) / EG;
        for (int cb0 = cb_lo; cb0 < cb_hi; cb0 += 8) {  // 8 loads in flight, then their stores
          uint4 v[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int cb = cb0 + i, term = cb >= nloc, loc = cb - term * nloc;
            if (cb < cb_hi) v[i] = __ldg(src + ((int64_t)term * (G.n1p / 4) + i_lo / 4 + loc) * kM1Rows);
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int cb = cb0 + i, term = cb >= nloc, loc = cb - term * nloc;
            if (cb < cb_hi) tmem_st4(tA + lanebase + term * tAw + 4 * loc, v[i]);
          }
        }
        tc::tmem_wait_st();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive1(&afull);
      }
      const Mode1Row ri = prm.rows[(int64_t)kg * kM1Rows + l];
      float2 acc[P];
#pragma unroll
      for (int s = 0; s < P; ++s) acc[s] = make_float2(0.f, 0.f);
      for (int nb = nb0; nb < nb1; ++nb, ++dc) {
        // this row's W values and the block's scales, loaded before the wait; a scale multiplies
        // each product (not W), so that no intermediate leaves FP32's normal range
        float f[P];
#pragma unroll
        for (int s = 0; s < P; ++s)
          f[s] = ldexpf(1.f, prm.Eblk[G.exp_index(k, sc, nb, s)] + ri.uexp - 2 * kHalfShift);
        float2 w[IW];
#pragma unroll
        for (int i = 0; i < IW; ++i) {
          const int i23 = nb * I + eg * IW + i;
          w[i] = (ri.wbase >= 0 && i23 < G.n23) ? prm.W[ri.wbase + (int64_t)i23 * ri.r1p] : make_float2(0.f, 0.f);
        }
        const int buf = dc % DB;
        const bool ok = !abort_flag && tc::mbar_wait(&dfull[buf], (dc / DB) & 1);
        if (!__all_sync(0xffffffffu, ok)) {
          if (lane == 0) abort_flag = 1;
          break;
        }
        tc::fence_after();
        // this warpgroup's D columns in registers, in rounds of loads that fit the registers; with
        // one D buffer it is handed back as soon as the last round is loaded
        constexpr int kBatch = EG == 2 ? 64 : (NC > 128 ? 96 : NC);
#pragma unroll
        for (int b0 = 0; b0 < NC; b0 += kBatch) {
          float v[kBatch];
#pragma unroll
          for (int c0 = 0; c0 < kBatch; c0 += 16)
            if (b0 + c0 < NC) tmem_ld16_nowait(tD + lanebase + buf * NB + eg * NC + b0 + c0, v + c0);
          tmem_wait_ld();
          if (DB == 1 && b0 + kBatch >= NC) {
            tc::fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive1(&dempty[buf]);
          }
#pragma unroll
          for (int cc = 0; cc < kBatch / 2; ++cc) {
            const int ci = b0 / 2 + cc;  // complex column of the warpgroup: (i23 offset, s)
            if (ci < NC / 2) {
              const float2 t = cfma_conj(w[ci / P], make_float2(v[2 * cc], v[2 * cc + 1]), make_float2(0.f, 0.f));
              acc[ci % P].x = fmaf(t.x, f[ci % P], acc[ci % P].x);
              acc[ci % P].y = fmaf(t.y, f[ci % P], acc[ci % P].y);
            }
          }
        }
        if (DB == 2) {
          tc::fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive1(&dempty[buf]);
        }
      }
      if (__any_sync(0xffffffffu, abort_flag != 0)) break;
      float2* out = prm.partial + ((int64_t)((nr * G.ntile1 + t1) * EG + eg) * prm.KG * kM1Rows +
                                   (int64_t)kg * kM1Rows + l) * prm.ppad + sc * P;
#pragma unroll
      for (int s = 0; s < P; ++s) out[s] = acc[s];
    }
  }
  tc::fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag) atomicOr(prm.err, kErrTimeout);
  if (warp == 0) tc::tmem_dealloc(tbase, prm.tcols);
}

// Psi'[j, s] = sum over partial slots, components and ranks of (j, k).  One CTA per (column, 16
// right-hand sides); its 8 parts take the slots in turn and are added in a fixed order, so the
// result does not depend on scheduling.
__global__ void __launch_bounds__(128) mode1_reduce_kernel(const float2* __restrict__ partial,
                                                           const int2* __restrict__ colrows, int q, int nslots,
                                                           int64_t rows_all, int ppad, int p,
                                                           float2* __restrict__ out, int64_t ldo) {
  const int j = blockIdx.x;
  const int s = blockIdx.y * 16 + (threadIdx.x & 15), part = threadIdx.x >> 4;
  __shared__ float2 red[8][16];
  float2 acc = make_float2(0.f, 0.f);
  if (s < p)
    for (int k = 0; k < q; ++k) {
      const int2 cr = colrows[(int64_t)j * q + k];
      for (int a = 0; a < cr.y; ++a)
        for (int sl = part; sl < nslots; sl += 8) {
          const float2 v = partial[((int64_t)sl * rows_all + cr.x + a) * ppad + s];
          acc.x += v.x;
          acc.y += v.y;
        }
    }
  red[part][threadIdx.x & 15] = acc;
  __syncthreads();
  if (part == 0 && s < p) {
    float2 t = red[0][threadIdx.x];
    for (int i = 1; i < 8; ++i) {
      t.x += red[i][threadIdx.x].x;
      t.y += red[i][threadIdx.x].y;
    }
    out[j + ldo * s] = t;
  }
}

template <int P, int NB>
static int launch_mode1(const M1Params& prm, size_t smem, size_t budget, int grid, cudaStream_t st) {
  // the limit is set once per device: to the budget, which every launch's size stays within
  ZBC_TRY((set_smem_limit<rmatvec_mode1_kernel<P, NB>>((int)budget)));
  rmatvec_mode1_kernel<P, NB><<<grid, M1Shape<NB>::threads, smem, st>>>(prm);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

// rows per N block for P right-hand sides per pass and A of 2 n1p TMEM columns: the widest MMA
// that fits (256 or 192 columns with one D buffer; else 160 or a power of two with two), at most
// 16 values of i23 per block (the epilogue's W registers)
static int mode1_nb(int P, int n1p) {
  if (P >= 8 && 256 + 2 * n1p <= 512) return 256;
  if (P >= 8 && 192 + 2 * n1p <= 512) return 192;  // one buffer beside a wide A (n1 up to 160)
  if (P >= 8 && 2 * 160 + 2 * n1p <= 512) return 160;
  int NB = std::min(128, 32 * P);
  while (NB > 32 && 2 * NB + 2 * n1p > 512) NB /= 2;
  return NB;
}

template <int P>
static int rmatvec_mode1_p(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo,
                           cudaStream_t st) {
  const Mode1Cache& mc = *h.cache->mode1;
  M1Geo G;
  G.P = P;
  G.n1 = h.n1;
  G.n1p = mc.n1p;
  G.n23 = h.n2 * h.n3;
  G.nsc = ceil_div(p, P);
  G.KC = 32;
  G.nkc = ceil_div(G.n1p, 32);
  // i1 tiles: A of the whole n1 while it fits beside a D buffer (n1 <= 224), else tiles of 5 K
  // chunks (160 i1, beside one 192-column D buffer); each tile's partial sums get their own slots
  G.nkt = G.n1p <= kM1MaxN1p ? G.nkc : 5;
  G.ntile1 = ceil_div(G.nkc, G.nkt);
  const int tAw = G.nkt * G.KC;  // TMEM columns per term of a tile's A (whole K chunks)
  const int NB = mode1_nb(P, tAw);
  const int DB = NB > 160 ? 1 : 2, EG = NB > 160 ? 2 : 1;
  if (NB < 2 * P || DB * NB + 2 * tAw > 512) {
    set_error("mode-1 adjoint: %d right-hand sides per pass do not fit tensor memory beside A", P);
    return ZBC_EINVAL;
  }
  G.NB = NB;
  G.I = NB / (2 * P);
  G.NBT = ceil_div(G.n23, G.I);
  G.chunk_u32 = (uint32_t)NB * G.KC;
  const size_t stage_bytes = 8 * (size_t)G.chunk_u32;
  const size_t budget = 225 * 1024;  // 3 stages of 64 KB (N blocks of 256 rows), and the alignment slack
  const int S = (int)std::min<size_t>(kM1MaxStages, (budget - 1024) / stage_bytes);
  if (S < 2) {
    set_error("mode-1 adjoint: stage layout does not fit shared memory");
    return ZBC_EINVAL;
  }
  const size_t smem = 1024 + (size_t)S * stage_bytes;
  // items: N ranges x i1 tiles x groups per pass, balanced over one CTA per SM; an item's cost is
  // its N blocks plus about two for loading A and writing its partial sums
  const int nsm = sm_count();
  int NR = 1;
  double best = 1e300;
  for (int r = 1; r <= std::min(G.NBT, 64); ++r) {
    const int64_t items = (int64_t)G.nsc * r * G.ntile1 * mc.KG;
    const int64_t per = (items + nsm - 1) / nsm;
    const double cost = (double)per * ((double)G.NBT / r + 2.0);
    if (cost < best * 0.999) {
      best = cost;
      NR = r;
    }
  }
  const int64_t nitems = (int64_t)G.nsc * NR * G.ntile1 * mc.KG;
  const int grid = (int)std::min<int64_t>(nsm, nitems);
  // workspaces: B operand blocks + exponents; partial sums (one slot per N range and warpgroup)
  const size_t bop_bytes = 4 * (size_t)h.q * G.nsc * G.NBT * G.nkc * 2 * G.chunk_u32;
  const size_t e_bytes = sizeof(int) * (size_t)h.q * G.nsc * G.NBT * P;
  ZBC_TRY(h.work_phi.ensure(bop_bytes + e_bytes));
  const int ppad = G.nsc * P;
  const int64_t rows_all = (int64_t)mc.KG * kM1Rows;
  const int nslots = NR * G.ntile1 * EG;
  ZBC_TRY(h.work_partial.ensure(sizeof(float2) * (size_t)nslots * rows_all * ppad));
  uint32_t* Bop = (uint32_t*)h.work_phi.ptr;
  int* Eblk = (int*)((unsigned char*)h.work_phi.ptr + bop_bytes);
  phi_split_kernel<<<dim3(G.NBT, G.nsc, h.q), 256, 0, st>>>(Phi, ldphi, p, h.nv(), G, Bop, Eblk,
                                                            (int*)h.work_err.ptr);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  M1Params prm;
  prm.A = mc.A;
  prm.rows = mc.rows;
  prm.kg_k = mc.kg_k;
  prm.W = h.cache->data;
  prm.Bop = Bop;
  prm.Eblk = Eblk;
  prm.partial = (float2*)h.work_partial.ptr;
  prm.err = (int*)h.work_err.ptr;
  prm.G = G;
  prm.KG = mc.KG;
  prm.NR = NR;
  prm.S = S;
  prm.ppad = ppad;
  uint32_t tcols = 32;
  while (tcols < (uint32_t)(DB * NB + 2 * tAw)) tcols <<= 1;
  prm.tcols = tcols;
  prm.nitems = nitems;
  int s;
  if constexpr (P == 1)
    s = launch_mode1<P, 32>(prm, smem, budget, grid, st);
  else if constexpr (P == 2)
    s = NB == 64 ? launch_mode1<P, 64>(prm, smem, budget, grid, st) : launch_mode1<P, 32>(prm, smem, budget, grid, st);
  else if constexpr (P == 4)
    s = NB == 128  ? launch_mode1<P, 128>(prm, smem, budget, grid, st)
        : NB == 64 ? launch_mode1<P, 64>(prm, smem, budget, grid, st)
                   : launch_mode1<P, 32>(prm, smem, budget, grid, st);
  else
    s = NB == 256   ? launch_mode1<P, 256>(prm, smem, budget, grid, st)
        : NB == 192 ? launch_mode1<P, 192>(prm, smem, budget, grid, st)
        : NB == 160 ? launch_mode1<P, 160>(prm, smem, budget, grid, st)
        : NB == 128 ? launch_mode1<P, 128>(prm, smem, budget, grid, st)
        : NB == 64  ? launch_mode1<P, 64>(prm, smem, budget, grid, st)
                    : launch_mode1<P, 32>(prm, smem, budget, grid, st);
  ZBC_TRY(s);
  mode1_reduce_kernel<<<dim3(h.M, ceil_div(p, 16)), 128, 0, st>>>((const float2*)h.work_partial.ptr, mc.colrows, h.q,
                                                                  nslots, rows_all, ppad, p, out, ldo);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

// Psi' = Z^H Phi on the handle's stored columns (M rows of Psi'), mode-1 tensor-core form
int rmatvec_mode1(Handle& h, const float2* Phi, int64_t ldphi, int p, float2* out, int64_t ldo, cudaStream_t st) {
  ZBC_TRY(build_mode1_cache(h, st));
  if (p == 1) return rmatvec_mode1_p<1>(h, Phi, ldphi, p, out, ldo, st);
  if (p == 2) return rmatvec_mode1_p<2>(h, Phi, ldphi, p, out, ldo, st);
  if (p <= 4) return rmatvec_mode1_p<4>(h, Phi, ldphi, p, out, ldo, st);
  if (p <= 8) return rmatvec_mode1_p<8>(h, Phi, ldphi, p, out, ldo, st);
  return rmatvec_mode1_p<kM1MaxP>(h, Phi, ldphi, p, out, ldo, st);
}

}  // namespace zbc
