// Forward product (Algorithm 1, Sec. III.B) with the mode-1 product on the tensor cores.
//
// With Z^{kj}[i1, i23] = sum_a U1_{kj}[i1, a] W_{kj}[i23, a] (i23 = i2 + n2 i3, W = G x2 U2 x3 U3,
// the decompression cache), the forward product regroups as
//   Y^k[i1 + n1 i23, s] = sum_{(j, a)} U1_{kj}[i1, a] C[(j, a), (i23, s)],
//   C[(j, a), (i23, s)] = W_{kj}[i23, a] X[j, s].
// For a block of 128 (i23, s) rows -- I = 128 / P values of i23 times the P right-hand sides of a
// pass -- this is one GEMM over K = (row (j, a) of component k, Re / Im):
//   D[(i23, s)][2 i1 + e] = sum_K A[(i23, s)][K] B[2 i1 + e][K],
//   A = (Re, Im) C, generated on the CUDA cores and stored to tensor memory (fp16 hi / lo),
//   B = U1 from a per-handle fp16 cache, row 2 i1 + 0: (Re U1, -Im U1), row 2 i1 + 1:
//       (Im U1, Re U1), so that D = (Re, Im) Y^k.
// The generated operand costs one complex multiply per (row, i23, s) -- against r1 multiply-adds
// per (voxel, column) for the decompression of the other forms -- and the tensor cores carry
// the mode-1 product.
//
// Scaling (powers of two, removed exactly): U1's row (j, a) by 2^(10 - uexp) (the adjoint's
// operand scaling); W[i23, (j, a)] by 2^(uexp - 10), which undoes it, and by 2^(10 - ew[i23]) with
// max over the rows of |W 2^(uexp - 10)| < 2^ew[i23]; X[:, s] by 2^-ex[s] with max |X[:, s]|
// < 2^ex[s].  Then |Re C|, |Im C| < 2^11 stay in fp16's normal range, and Y = D 2^(ew + ex - 10).
// Precision: fp16 hi + lo for both operands, products hi.hi + hi.lo + lo.hi.  The tensor core's
// FP32 accumulation into one D runs over at most kFwdSeg chunks of 32 rows (72 MMAs); the
// CUDA-core warps then add D into FP32 registers with round-to-nearest ("folds"), two D buffers
// alternating, so K = 2 x (rows of component k) never accumulates in one tensor-core sum (one sum
// over all of K: relative error 6.8e-5 on the 96^3 x 1024-column workload; folds every 3 chunks:
// 8.0e-7, every 6: 1.4e-6).
//
// Per call: m1f_x_kernel (ex and the scaled X^T of each pass), m1f_xe_kernel (X per chunk row),
// then matvec_mode1_kernel, persistent over items (component, pass, block of 128 (i23, s) rows):
//   copy warp  : per chunk of 32 rows, cp.async.bulk of U1's operand block (both terms), the W
//                block of the item's i23 values and the X values of the chunk's rows into a
//                stage ring
//   MMA warp   : per chunk 12 MMAs (4 K steps x 3 products), A from TMEM (two buffers), B from
//                the stage, D in TMEM (two buffers of N = 2 n1t columns for an i1 tile of n1t rows)
//   8 warps    : generate A (each warpgroup half of a chunk's rows), fold D into registers (each
//                warpgroup half of D's columns) and write Y.
#include "mode1.cuh"

namespace zbc {

constexpr int kFwdChunk = 32;   // rows (j, a) per K chunk
constexpr int kFwdSeg = 6;      // chunks per tensor-core accumulation
constexpr int kFwdMaxN1p = 96;  // i1 tile limit: two D buffers of 2 n1t columns + two A buffers of 64 in TMEM

// i1 tiles of the forward: ntile1 = ceil(n1 / 96) tiles of n1t rows (a multiple of 16), each an
// item dimension of its own (the W X operand is generated once per tile, which is cheap)
static void fwd_tiles(int n1, int& ntile1, int& n1t) {
  ntile1 = (n1 + kFwdMaxN1p - 1) / kFwdMaxN1p;
  n1t = ((n1 + ntile1 - 1) / ntile1 + 15) / 16 * 16;
}
constexpr int kFwdThreads = 32 * 10;

// ---------------------------------------------------------------------------------------------
// per-handle operands (built once, on the first forward call)
// ---------------------------------------------------------------------------------------------

// ew[k][i23] = exponent of max over component k's rows of |Re|, |Im| of W[i23, row] 2^(uexp - 10)
__global__ void __launch_bounds__(256) m1f_ew_kernel(const float2* __restrict__ W, const Mode1Row* __restrict__ rows,
                                                     const int* __restrict__ gbase, const int* __restrict__ nrows,
                                                     int n23, int n23p, int* __restrict__ ew) {
  const int k = blockIdx.y;
  const int i23 = blockIdx.x * blockDim.x + threadIdx.x;
  if (i23 >= n23p) return;
  float mx = 0.f;
  if (i23 < n23) {
    const Mode1Row* r = rows + (int64_t)gbase[k] * kM1Rows;
    for (int rho = 0; rho < nrows[k]; ++rho) {
      const Mode1Row ri = r[rho];
      const float2 w = W[ri.wbase + (int64_t)i23 * ri.r1p];
      mx = fmaxf(mx, ldexpf(fmaxf(fabsf(w.x), fabsf(w.y)), ri.uexp - kHalfShift));
    }
  }
  int e = 0;
  frexpf(mx, &e);
  ew[(int64_t)k * n23p + i23] = e;
}

// Wc[c][i23][rho] = W[i23, row] 2^(uexp - ew[k][i23]) for the rows of chunk c (zero for padding
// rows and for i23 >= n23)
__global__ void __launch_bounds__(256) m1f_wc_kernel(const float2* __restrict__ W, const Mode1Row* __restrict__ rows,
                                                     const int* __restrict__ chunk_row0, const int* __restrict__ chunk_k,
                                                     const int* __restrict__ chunk_nr, const int* __restrict__ ew,
                                                     int n23, int n23p, float2* __restrict__ Wc) {
  const int c = blockIdx.y;
  const int k = chunk_k[c];
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n23p * kFwdChunk) return;
  const int i23 = (int)(e / kFwdChunk), rl = (int)(e % kFwdChunk);
  float2 v = make_float2(0.f, 0.f);
  if (i23 < n23 && rl < chunk_nr[c]) {
    const Mode1Row ri = rows[chunk_row0[c] + rl];
    const float2 w = W[ri.wbase + (int64_t)i23 * ri.r1p];
    const int sh = ri.uexp - ew[(int64_t)k * n23p + i23];
    v = make_float2(ldexpf(w.x, sh), ldexpf(w.y, sh));
  }
  Wc[((int64_t)c * n23p + i23) * kFwdChunk + rl] = v;
}

// U1's operand blocks: chunk c, i1 tile t1, term t, row n = 2 (i1 - t1 n1t) + e (N = 2 n1t rows),
// 16-byte piece kc of rows 4 kc .. 4 kc + 3 of the chunk, in the 128-byte swizzled K-major layout
__global__ void __launch_bounds__(256) m1f_b_kernel(const float2* __restrict__ pool, const TensorDesc* __restrict__ desc,
                                                    const int4* __restrict__ rowsrc, const Mode1Row* __restrict__ rows,
                                                    const int* __restrict__ chunk_row0, const int* __restrict__ chunk_nr,
                                                    int n1, int n1t, uint32_t* __restrict__ Bf) {
  const int c = blockIdx.y, t1 = blockIdx.z, ntile1 = gridDim.z;
  const int N = 2 * n1t;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;  // (row n, piece kc)
  if (e >= N * 8) return;
  const int n = e / 8, kc = e % 8;
  const int i1 = t1 * n1t + (n >> 1), eo = n & 1;
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rl = 4 * kc + i;
    float2 u = make_float2(0.f, 0.f);
    int uexp = 0;
    if (rl < chunk_nr[c] && i1 < n1) {
      const int4 src = rowsrc[chunk_row0[c] + rl];
      const TensorDesc d = desc[src.x];
      u = pool[d.off + (int64_t)d.r1 * d.r2 * d.r3 + (int64_t)n1 * src.y + i1];
      uexp = rows[chunk_row0[c] + rl].uexp;
    }
    const float ur = ldexpf(u.x, kHalfShift - uexp), ui = ldexpf(u.y, kHalfShift - uexp);
    const float x0 = eo ? ui : ur, x1 = eo ? ur : -ui;  // (Re, -Im) or (Im, Re)
    const __half h0 = __float2half_rn(x0), h1 = __float2half_rn(x1);
    const __half l0 = __float2half_rn(x0 - __half2float(h0)), l1 = __float2half_rn(x1 - __half2float(h1));
    const __half2 vh = __halves2half2(h0, h1), vl = __halves2half2(l0, l1);
    hw[i] = *reinterpret_cast<const uint32_t*>(&vh);
    lw[i] = *reinterpret_cast<const uint32_t*>(&vl);
  }
  const int64_t term = (int64_t)N * kFwdChunk;  // 32-bit words per term
  uint32_t* blk = Bf + ((int64_t)c * ntile1 + t1) * 2 * term + tc::sw128_off(n, kc) / 4;
  *reinterpret_cast<uint4*>(blk) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  *reinterpret_cast<uint4*>(blk + term) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

void mode1_fwd_release(Mode1Cache* c) {
  if (!c) return;
  for (void** ptr : {(void**)&c->Bf, (void**)&c->Wc, (void**)&c->ew, (void**)&c->chunkinfo, (void**)&c->jtab,
                     (void**)&c->d_chbase}) {
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
  }
  c->bytes -= c->fwd_bytes;
  c->fwd_bytes = 0;
  c->fwd = false;
}

static int build_mode1_fwd(Handle& h, cudaStream_t st) {
  ZBC_TRY(build_mode1_cache(h, st));
  Mode1Cache& mc = *h.cache->mode1;
  if (mc.fwd) return ZBC_OK;
  const int q = h.q, M = h.M;
  const int n23 = h.n2 * h.n3, n23p = (n23 + 31) / 32 * 32;  // whole blocks of up to 32 i23
  // chunks of 32 rows per component; per chunk its first row (global), rows, component, first
  // column and columns, and each row's column relative to the first
  std::vector<int> chbase(q + 1, 0), nrows(q, 0);
  std::vector<int> row0, nr, ck;
  std::vector<int2> info;
  std::vector<int8_t> jtab;
  for (int k = 0; k < q; ++k) {
    std::vector<int> rowj;
    for (int j = 0; j < M; ++j)
      for (int a = 0; a < h.desc[(size_t)j * q + k].r1; ++a) rowj.push_back(j);
    nrows[k] = (int)rowj.size();
    const int nch = ((int)rowj.size() + kFwdChunk - 1) / kFwdChunk;
    chbase[k + 1] = chbase[k] + nch;
    for (int c = 0; c < nch; ++c) {
      const int r0 = c * kFwdChunk, nrc = std::min(kFwdChunk, (int)rowj.size() - r0);
      const int j0 = rowj[r0], nj = rowj[r0 + nrc - 1] - j0 + 1;
      row0.push_back(mc.gbase[k] * kM1Rows + r0);
      nr.push_back(nrc);
      ck.push_back(k);
      info.push_back(make_int2(j0, nj));
      for (int i = 0; i < kFwdChunk; ++i) jtab.push_back((int8_t)(i < nrc ? rowj[r0 + i] - j0 : 0));
    }
  }
  const int NC = chbase[q];
  int ntile1, n1t;
  fwd_tiles(h.n1, ntile1, n1t);
  const int N = 2 * n1t;  // rows 2 i1 + e of one i1 tile
  const size_t bwords = (size_t)NC * ntile1 * 2 * N * kFwdChunk;
  const size_t wc_elems = (size_t)NC * n23p * kFwdChunk;
  int *d_row0 = nullptr, *d_nr = nullptr, *d_ck = nullptr, *d_gbase = nullptr, *d_nrows = nullptr;
  cudaError_t e = cudaMalloc(&mc.Bf, sizeof(uint32_t) * bwords);
  if (e == cudaSuccess) e = cudaMalloc(&mc.Wc, sizeof(float2) * wc_elems);
  if (e == cudaSuccess) e = cudaMalloc(&mc.ew, sizeof(int) * (size_t)q * n23p);
  if (e == cudaSuccess) e = cudaMalloc(&mc.chunkinfo, sizeof(int2) * NC);
  if (e == cudaSuccess) e = cudaMalloc(&mc.jtab, (size_t)NC * kFwdChunk);
  if (e == cudaSuccess) e = cudaMalloc(&mc.d_chbase, sizeof(int) * (q + 1));
  if (e == cudaSuccess) {
    mc.fwd_bytes = (int64_t)(sizeof(uint32_t) * bwords + sizeof(float2) * wc_elems + sizeof(int) * (size_t)q * n23p +
                             sizeof(int2) * NC + (size_t)NC * kFwdChunk + sizeof(int) * (q + 1));
    mc.bytes += mc.fwd_bytes;
  }
  if (e == cudaSuccess) e = cudaMalloc(&d_row0, sizeof(int) * NC);
  if (e == cudaSuccess) e = cudaMalloc(&d_nr, sizeof(int) * NC);
  if (e == cudaSuccess) e = cudaMalloc(&d_ck, sizeof(int) * NC);
  if (e == cudaSuccess) e = cudaMalloc(&d_gbase, sizeof(int) * (q + 1));
  if (e == cudaSuccess) e = cudaMalloc(&d_nrows, sizeof(int) * q);
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  up(mc.chunkinfo, info.data(), sizeof(int2) * NC);
  up(mc.jtab, jtab.data(), jtab.size());
  up(mc.d_chbase, chbase.data(), sizeof(int) * (q + 1));
  up(d_row0, row0.data(), sizeof(int) * NC);
  up(d_nr, nr.data(), sizeof(int) * NC);
  up(d_ck, ck.data(), sizeof(int) * NC);
  up(d_gbase, mc.gbase.data(), sizeof(int) * (q + 1));
  up(d_nrows, nrows.data(), sizeof(int) * q);
  if (e == cudaSuccess) {
    m1f_ew_kernel<<<dim3(ceil_div(n23p, 256), q), 256, 0, st>>>(h.cache->data, mc.rows, d_gbase, d_nrows, n23, n23p,
                                                               mc.ew);
    m1f_wc_kernel<<<dim3(ceil_div((int64_t)n23p * kFwdChunk, 256), NC), 256, 0, st>>>(
        h.cache->data, mc.rows, d_row0, d_ck, d_nr, mc.ew, n23, n23p, mc.Wc);
    m1f_b_kernel<<<dim3(ceil_div(N * 8, 256), NC, ntile1), 256, 0, st>>>(h.d_pool, h.d_desc, mc.rowsrc, mc.rows,
                                                                        d_row0, d_nr, h.n1, n1t, mc.Bf);
    count_launch(3);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (void* ptr : {(void*)d_row0, (void*)d_nr, (void*)d_ck, (void*)d_gbase, (void*)d_nrows})
    if (ptr) cudaFree(ptr);
  if (e != cudaSuccess) {  // leave the cache as it was, so that a later call can build it again
    mode1_fwd_release(&mc);
    set_error("mode-1 forward operand build failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? ZBC_ENOMEM : ZBC_ECUDA;
  }
  mc.n23p = n23p;
  mc.chbase = chbase;
  mc.fwd = true;
  return ZBC_OK;
}

// ex[s] = exponent of max_j |Re|, |Im| of X[j, s]; XT[sc][j][P] = X[j, sc P + s] 2^-ex (zero for
// s >= p).  One CTA per padded right-hand side.
__global__ void __launch_bounds__(256) m1f_x_kernel(const float2* __restrict__ X, int64_t ldx, int M, int p, int P,
                                                    float2* __restrict__ XT, int* __restrict__ ex,
                                                    int* __restrict__ err) {
  const int sg = blockIdx.x, sc = sg / P, sl = sg % P;
  __shared__ float wmax[8];
  float mx = 0.f;
  bool finite = true;
  if (sg < p)
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
      const float2 v = X[j + ldx * sg];
      finite = finite && isfinite(v.x) && isfinite(v.y);
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
  if (!finite) atomicOr(err, kErrNonFinite);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
  __syncthreads();
  float m = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wmax[w]);
  int e = 0;
  frexpf(m, &e);
  if (threadIdx.x == 0) ex[sg] = e;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const float2 v = sg < p ? X[j + ldx * sg] : make_float2(0.f, 0.f);
    XT[((int64_t)sc * M + j) * P + sl] = make_float2(ldexpf(v.x, -e), ldexpf(v.y, -e));
  }
}

// XE[sc][c][r][s] = XT[sc][column of row r of chunk c][s]: each chunk row's X values, so that the
// generator reads them without an index lookup (padding rows repeat a column; their W is zero)
__global__ void __launch_bounds__(256) m1f_xe_kernel(const float2* __restrict__ XT, const int2* __restrict__ chunkinfo,
                                                     const int8_t* __restrict__ jtab, int M, int NC, int P, int nsc,
                                                     float2* __restrict__ XE) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nsc * NC * kFwdChunk * P) return;
  const int s = (int)(e % P);
  const int64_t t = e / P;
  const int r = (int)(t % kFwdChunk);
  const int64_t t2 = t / kFwdChunk;
  const int c = (int)(t2 % NC), sc = (int)(t2 / NC);
  const int j = chunkinfo[c].x + jtab[(int64_t)c * kFwdChunk + r];
  XE[e] = XT[((int64_t)sc * M + j) * P + s];
}

// ---------------------------------------------------------------------------------------------
// the product kernel
// ---------------------------------------------------------------------------------------------

struct FwdParams {
  const uint32_t* Bf;
  const float2* Wc;
  const int* ew;
  const float2* XE;   // [nsc][chunk][32][P]: X (scaled by 2^-ex) of each chunk row
  const int* ex;      // [nsc P]
  const int* chbase;  // [q + 1]
  float2* Y;
  int64_t ldy, nv;
  int* err;
  int NC, p, n1, n1t, ntile1, n23, n23p, nsc, nblk, S;
  uint32_t b_bytes, w_off, x_off, stage_bytes;
  int64_t nitems;  // q ntile1 nsc nblk
};

// item -> (component k, i1 tile t1, pass sc, block of I values of i23); blocks vary fastest, so
// the CTAs running at one time stream the same U1 blocks (from L2)
__device__ __forceinline__ void m1f_item(const FwdParams& prm, int64_t it, int& k, int& t1, int& sc, int& blk) {
  blk = (int)(it % prm.nblk);
  int64_t t = it / prm.nblk;
  sc = (int)(t % prm.nsc);
  t /= prm.nsc;
  t1 = (int)(t % prm.ntile1);
  k = (int)(t / prm.ntile1);
}

// 8 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

template <int P>
__global__ void __launch_bounds__(kFwdThreads, 1) matvec_mode1_kernel(const FwdParams prm) {
  constexpr int I = kM1Rows / P;  // i23 per block of 128 rows
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t sfull[kM1MaxStages], sempty[kM1MaxStages], afull[2], aempty[2], dfull[2], dempty[2];
  __shared__ uint32_t tbase;
  __shared__ volatile int abort_flag;
  unsigned char* stages = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = prm.S;
  const int N = 2 * prm.n1t;  // D columns: (i1 of the tile, Re / Im)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  if (warp == 0) tc::tmem_alloc(&tbase, 512);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&sfull[s], 1);
      tc::mbar_init(&sempty[s], 1 + 8);  // the MMA warp's commit and the 8 generator warps
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&afull[b], 8);
      tc::mbar_init(&aempty[b], 1);
      tc::mbar_init(&dfull[b], 1);
      tc::mbar_init(&dempty[b], 8);
    }
    abort_flag = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tD = tbase;          // D buffers: columns [b N, (b + 1) N)
  const uint32_t tA = tbase + 2 * N;  // A buffers: 64 columns each, hi in the first 32

  if (warp == 8) {
    // ---------------- copy warp ----------------
    if (lane == 0) {
      uint32_t cnt = 0;
      for (int64_t it = blockIdx.x; it < prm.nitems && !abort_flag; it += gridDim.x) {
        int k, t1, sc, blk;
        m1f_item(prm, it, k, t1, sc, blk);
        const int c1 = prm.chbase[k + 1];
        for (int c = prm.chbase[k]; c < c1 && !abort_flag; ++c, ++cnt) {
          const int st = cnt % S;
          if (cnt >= (uint32_t)S && (abort_flag || !tc::mbar_wait(&sempty[st], ((cnt / S) - 1) & 1))) {
            abort_flag = 1;
            break;
          }
          constexpr uint32_t wb = I * kFwdChunk * 8, xb = kFwdChunk * P * 8;
          unsigned char* sb = stages + (size_t)st * prm.stage_bytes;
          mbar_arrive_expect_tx(&sfull[st], prm.b_bytes + wb + xb);
          bulk_g2s(sb, prm.Bf + ((int64_t)c * prm.ntile1 + t1) * (prm.b_bytes / 4), prm.b_bytes, &sfull[st]);
          bulk_g2s(sb + prm.w_off, prm.Wc + ((int64_t)c * prm.n23p + (int64_t)blk * I) * kFwdChunk, wb, &sfull[st]);
          bulk_g2s(sb + prm.x_off, prm.XE + ((int64_t)sc * prm.NC + c) * kFwdChunk * P, xb, &sfull[st]);
        }
      }
      if (abort_flag)  // let the copies in flight land before the CTA exits
        for (uint32_t c = cnt > (uint32_t)S ? cnt - S : 0; c < cnt; ++c) tc::mbar_wait(&sfull[c % S], (c / S) & 1);
    }
    __syncwarp();
  } else if (warp == 9) {
    // ---------------- MMA warp ----------------
    if (lane == 0) {
      const uint32_t idesc = tc::instr_desc(128, N, 0);  // kind::f16, f16 operands, FP32 D
      const uint32_t bterm = prm.b_bytes / 2;
      uint32_t gc = 0, gs = 0;
      for (int64_t it = blockIdx.x; it < prm.nitems && !abort_flag; it += gridDim.x) {
        int k, t1, sc, blk;
        m1f_item(prm, it, k, t1, sc, blk);
        const int nch = prm.chbase[k + 1] - prm.chbase[k];
        for (int cl = 0; cl < nch && !abort_flag; ++cl, ++gc) {
          const bool first = cl % kFwdSeg == 0, last = cl % kFwdSeg == kFwdSeg - 1 || cl == nch - 1;
          const int buf = gs & 1;
          const int st = gc % S, ab = gc & 1;
          bool ok = !(first && gs >= 2) || tc::mbar_wait(&dempty[buf], ((gs >> 1) - 1) & 1);
          ok = ok && tc::mbar_wait(&sfull[st], (gc / S) & 1) && tc::mbar_wait(&afull[ab], (gc >> 1) & 1);
          if (!ok) {
            abort_flag = 1;
            break;
          }
          tc::fence_after();
          const uint32_t sb = tc::smem_u32(stages + (size_t)st * prm.stage_bytes);
          const uint32_t d = tD + buf * N, a = tA + ab * 64;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t bh = tc::smem_desc_sw128(sb + ks * 32);
            const uint64_t bl = tc::smem_desc_sw128(sb + bterm + ks * 32);
            tc::mma_ts(d, a + 8 * ks, bh, idesc, (first && ks == 0) ? 0u : 1u);  // hi . hi
            tc::mma_ts(d, a + 8 * ks, bl, idesc, 1u);                          // hi . lo
            tc::mma_ts(d, a + 32 + 8 * ks, bh, idesc, 1u);                     // lo . hi
          }
          tc::commit(&sempty[st]);
          tc::commit(&aempty[ab]);
          if (last) {
            tc::commit(&dfull[buf]);
            ++gs;
          }
        }
      }
    }
    __syncwarp();
  } else {
    // ---------------- 8 warps: generate A, fold D, write Y ----------------
    const int g = warp >> 2;                       // A rows [16 g, 16 g + 16) of each chunk; D columns [g H, g H + H)
    const int row = (warp & 3) * 32 + lane;        // TMEM lane = (i23l, s)
    const uint32_t lanebase = (uint32_t)((warp & 3) * 32) << 16;
    const int i23l = row / P, s = row % P;
    const int H = prm.n1t;                         // D columns per warpgroup
    float acc[kFwdMaxN1p];
#pragma unroll
    for (int i = 0; i < kFwdMaxN1p; ++i) acc[i] = 0.f;
    uint32_t gc = 0, gs = 0;
    for (int64_t it = blockIdx.x; it < prm.nitems; it += gridDim.x) {
      if (__any_sync(0xffffffffu, abort_flag != 0)) break;
      int k, t1, sc, blk;
      m1f_item(prm, it, k, t1, sc, blk);
      const int nch = prm.chbase[k + 1] - prm.chbase[k];
      const int nseg = (nch + kFwdSeg - 1) / kFwdSeg;
      const uint32_t gs0 = gs;
      int folded = 0;
      bool bad = false;
      // add the tensor core's sum of local segment sl into acc (round-to-nearest FP32)
      auto fold = [&](int sl) {
        const uint32_t seg = gs0 + sl;
        const int buf = seg & 1;
        const bool ok = !abort_flag && tc::mbar_wait(&dfull[buf], (seg >> 1) & 1);
        if (!__all_sync(0xffffffffu, ok)) {
          bad = true;
          return;
        }
        tc::fence_after();
#pragma unroll
        for (int b0 = 0; b0 < kFwdMaxN1p; b0 += 16) {
          if (b0 < H) {
            float v[16];
            tmem_ld16_nowait(tD + lanebase + buf * N + g * H + b0, v);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[b0 + i] += v[i];
          }
        }
        tc::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive1(&dempty[buf]);
      };
      for (int cl = 0; cl < nch && !bad; ++cl, ++gc) {
        // segment sl is folded before chunk 3 sl + 5 is generated: by then its MMAs were issued
        // (the MMA warp runs at most two chunks behind), and the fold is done long before
        // segment sl + 2 needs the buffer
        if (cl >= kFwdSeg + 2 && (cl - kFwdSeg - 2) % kFwdSeg == 0) {
          fold(folded++);
          if (bad) break;
        }
        const int st = gc % S, ab = gc & 1;
        bool ok = !abort_flag && (gc < 2 || tc::mbar_wait(&aempty[ab], ((gc >> 1) - 1) & 1));
        ok = ok && tc::mbar_wait(&sfull[st], (gc / S) & 1);
        if (!__all_sync(0xffffffffu, ok)) {
          bad = true;
          break;
        }
        const unsigned char* sb = stages + (size_t)st * prm.stage_bytes;
        const float4* Ws = (const float4*)(sb + prm.w_off) + i23l * (kFwdChunk / 2);  // this row's i23
        const float2* Xs = (const float2*)(sb + prm.x_off) + s;                      // [chunk row][P]
#pragma unroll
        for (int r0 = 0; r0 < 16; r0 += 8) {
          uint32_t hi[8], lo[8];
          float4 w4[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) w4[r] = Ws[(16 * g + r0) / 2 + r];
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int rl = 16 * g + r0 + r;
            const float2 wv = (r & 1) ? make_float2(w4[r / 2].z, w4[r / 2].w) : make_float2(w4[r / 2].x, w4[r / 2].y);
            const float2 c = cmul(wv, Xs[rl * P]);
            const __half2 h2 = __floats2half2_rn(c.x, c.y);
            const float2 hf = __half22float2(h2);
            const __half2 l2 = __floats2half2_rn(c.x - hf.x, c.y - hf.y);
            hi[r] = *reinterpret_cast<const uint32_t*>(&h2);
            lo[r] = *reinterpret_cast<const uint32_t*>(&l2);
          }
          tmem_st8(tA + lanebase + ab * 64 + 16 * g + r0, hi);
          tmem_st8(tA + lanebase + ab * 64 + 32 + 16 * g + r0, lo);
        }
        tc::tmem_wait_st();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive1(&afull[ab]);
          mbar_arrive1(&sempty[st]);
        }
      }
      while (!bad && folded < nseg) fold(folded++);
      gs = gs0 + nseg;
      if (bad) {
        if (lane == 0) abort_flag = 1;
        break;
      }
      // Y rows i1 in t1 n1t + [g H / 2, g H / 2 + H / 2) of voxel column i23 for right-hand side s
      const int i23 = blk * I + i23l, sg = sc * P + s;
      if (i23 < prm.n23 && sg < prm.p) {
        const float f = ldexpf(1.f, prm.ew[(int64_t)k * prm.n23p + i23] + prm.ex[sg] - kHalfShift);
        float2* y = prm.Y + (int64_t)k * prm.nv + (int64_t)prm.n1 * i23 + prm.ldy * sg;
#pragma unroll
        for (int ii = 0; ii < kFwdMaxN1p / 2; ++ii) {
          const int i1 = t1 * prm.n1t + g * (H / 2) + ii;
          if (ii < H / 2 && i1 < prm.n1) y[i1] = make_float2(acc[2 * ii] * f, acc[2 * ii + 1] * f);
        }
      }
#pragma unroll
      for (int i = 0; i < kFwdMaxN1p; ++i) acc[i] = 0.f;
    }
  }
  tc::fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag) atomicOr(prm.err, kErrTimeout);
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

template <int P>
static int matvec_mode1_p(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  constexpr int I = kM1Rows / P;
  const Mode1Cache& mc = *h.cache->mode1;
  FwdParams prm;
  prm.p = p;
  prm.n1 = h.n1;
  fwd_tiles(h.n1, prm.ntile1, prm.n1t);
  prm.n23 = h.n2 * h.n3;
  prm.n23p = mc.n23p;
  prm.nsc = ceil_div(p, P);
  prm.nblk = mc.n23p / I;
  prm.nitems = (int64_t)h.q * prm.ntile1 * prm.nsc * prm.nblk;
  prm.ldy = ldy;
  prm.nv = h.nv();
  const int N = 2 * prm.n1t;
  prm.b_bytes = (uint32_t)(2 * N * 128);
  prm.w_off = prm.b_bytes;
  prm.x_off = prm.w_off + (uint32_t)(I * kFwdChunk * 8);
  prm.stage_bytes = (prm.x_off + (uint32_t)(kFwdChunk * P * 8) + 1023) / 1024 * 1024;
  const size_t budget = 226 * 1024;
  prm.S = (int)std::min<size_t>(kM1MaxStages, (budget - 1024) / prm.stage_bytes);
  if (prm.S < 2) {
    set_error("mode-1 forward: stage layout does not fit shared memory");
    return ZBC_EINVAL;
  }
  const size_t smem = 1024 + (size_t)prm.S * prm.stage_bytes;
  // scaled X^T per pass, its expansion per chunk row, the exponents (no host copies: a call can
  // be captured in a CUDA graph)
  prm.NC = mc.chbase[h.q];
  const size_t xt_elems = (size_t)prm.nsc * h.M * P, xe_elems = (size_t)prm.nsc * prm.NC * kFwdChunk * P;
  ZBC_TRY(h.work_xt.ensure(sizeof(float2) * (xt_elems + xe_elems) + sizeof(int) * (size_t)prm.nsc * P));
  float2* XT = (float2*)h.work_xt.ptr;
  float2* XE = XT + xt_elems;
  int* ex = (int*)(XE + xe_elems);
  m1f_x_kernel<<<prm.nsc * P, 256, 0, st>>>(X, ldx, h.M, p, P, XT, ex, (int*)h.work_err.ptr);
  m1f_xe_kernel<<<ceil_div((int64_t)xe_elems, 256), 256, 0, st>>>(XT, mc.chunkinfo, mc.jtab, h.M, prm.NC, P, prm.nsc,
                                                                   XE);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch(2);
  prm.Bf = mc.Bf;
  prm.Wc = mc.Wc;
  prm.ew = mc.ew;
  prm.XE = XE;
  prm.ex = ex;
  prm.chbase = mc.d_chbase;
  prm.Y = Y;
  prm.err = (int*)h.work_err.ptr;
  ZBC_TRY((set_smem_limit<matvec_mode1_kernel<P>>((int)budget)));
  const int grid = (int)std::min<int64_t>(sm_count(), prm.nitems);
  matvec_mode1_kernel<P><<<grid, kFwdThreads, smem, st>>>(prm);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

// Y = Z X on the handle's stored columns (X has M rows), mode-1 tensor-core form: passes of 4, 8
// or 16 right-hand sides (a block of 128 rows holds 32, 16 or 8 values of i23), i1 tiles of at
// most 96
int matvec_mode1(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  ZBC_TRY(build_mode1_fwd(h, st));
  if (p <= 4) return matvec_mode1_p<4>(h, X, ldx, p, Y, ldy, st);
  if (p <= 8) return matvec_mode1_p<8>(h, X, ldx, p, Y, ldy, st);
  return matvec_mode1_p<kM1MaxP>(h, X, ldx, p, Y, ldy, st);
}

}  // namespace zbc
