// Forward product (Algorithm 1, Sec. III.B) as decompression then contraction per voxel block,
// the contraction on the tensor cores (ZBC_TC_DC).
//
// Algorithm 1 accumulates Y^k += Z^{kj}(:) X_{j:} column by column.  Here a CTA owns a block of
// voxels of one component k -- 32 consecutive i1 (group g1) times 4T consecutive i23 (i23 = i2 +
// n2 i3) -- and walks the stored columns j in chunks of at most 8 (at most kDcRows rank rows):
//   generator warps : Z^{kj}[i1, i23] = sum_a U1_{kj}[i1, a] W_{kj}[i23, a]  (the last mode product
//                     of the decompression; W = G x2 U2 x3 U3 from the handle's decompression cache)
//                     in FP32 on the CUDA cores, one i1 per thread for T values of i23, so each U1
//                     value a thread loads serves T voxels; written as fp16 hi / lo pieces of the
//                     MMA's A operand (T tiles of 128 voxels x (Re Z, Im Z) of the chunk's 8
//                     columns) in shared memory;
//   MMA warp        : per tile D[voxel][(Re | Im) Y of P right-hand sides] += A B^T, B = the chunk's
//                     rows of X' as [[Re X, Im X], [-Im X, Re X]] (fp16 hi / lo, built per call):
//                     three products (hi.hi, hi.lo, lo.hi), M = 128, N = 2P, K = 16, D in TMEM;
//   every kDcSeg chunks the generator warps add D into an FP32 sum S in TMEM with
//   round-to-nearest adds (the tensor core's own FP32 accumulation does not round to nearest),
//   and after the last chunk they write Y = S scaled back.
// Decompression costs r1 complex multiply-adds per (voxel, column) on the CUDA cores, as in the
// FP32 form; the contraction, q n_v M p complex MACs, runs on the tensor cores with N up to 256
// (128 right-hand sides per pass), so the decompression is done once per pass instead of once per
// 16 or 32 right-hand sides.
//
// Scaling (powers of two, removed exactly): Z by 2^(14 - E_k), |Z| < 2^E_k over component k by
// the bound ||G||_F prod_g max_i ||U_g[i, :]|| of each tensor; X'[:, s] by 2^(14 - ex_s) with
// max |Re|, |Im| of X'[:, s] < 2^ex_s.  Then every fp16 hi term is below 2^14 in magnitude and
// Y = S 2^(E_k + ex_s - 28).
//
// Per-handle operands (built on the first call): U1 in groups of 32 rows, [k][g1][j][a/2][32][2]
// (the pair a, a+1 of one row is one 16-byte load), the column chunks of each component, the
// columns' W offsets and strides, E_k.  Per call: ex_s and the B blocks [pass][chunk][hi | lo]
// [2P rows][16 fp16] in the canonical K-major layout.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "mode1.cuh"

namespace zbc {

constexpr int kDcCols = 8;        // columns per chunk: the MMA's K = 16 = (Re, Im) x 8
constexpr int kDcRows = 128;      // rank rows (sum of r1p) per chunk: the stage's U1 capacity
constexpr int kDcSeg = 16;        // chunks per tensor-core accumulation before a fold into S
constexpr int kDcMaxStages = 6;
constexpr int kDcThreads = 32 * 10;  // 8 generator / fold warps, copy warp, MMA warp
constexpr int kDcShift = 14;      // fp16 hi terms below 2^kDcShift

// Per-chunk metadata the copy warp writes into its stage (the generators read it from shared memory
// instead of chasing the chunk and column tables in global memory): columns, and per column its
// r1p and the float4 offsets of its U1 block and of its W rows in the stage.
struct DcHdr {
  int nc;
  int r1p[kDcCols];
  int uo[kDcCols];
  int wo[kDcCols];
};

struct DcCol {
  int64_t woff;  // W_{kj} in the decompression cache ([i23][a], stride r1p)
  int r1p;       // r1 rounded up to 2 (the cache's stride)
  int pad;
};

// What the copy warp needs of one chunk, in 128 bytes (one coalesced load of 32 words)
struct __align__(16) DcChunk {
  int j0, nc, z, k;     // first column, columns, sum of r1p, component
  int r1p[kDcCols];
  int64_t woff[kDcCols];
  int64_t pre32;        // 32 x (sum of r1p over the component's columns before j0): the chunk's
                        // U1 block within a (component, i1 group) block of u1g
  int pad[2];
};
static_assert(sizeof(DcChunk) == 128, "one word per lane");

struct DcCache {
  int ng1 = 0, NC = 0;
  std::vector<int> chbase;        // host: first chunk of each component (q + 1 entries)
  std::vector<int4> chunks_h;     // host copy of the chunk table
  std::vector<int> Ek_h;
  int max_rows = 0;               // largest sum of r1p over a chunk (sizes the stages)
  float2* u1g = nullptr;          // [k][g1][j][a/2][32][2]
  int64_t* u1off = nullptr;       // [(k ng1 + g1)(M + 1) + j]: start of column j's block (elements)
  int64_t* u1base = nullptr;      // [k ng1 + g1]: start of a (component, i1 group) block
  DcChunk* rec = nullptr;         // [chunk]
  int4* chunks = nullptr;         // [chunk]: (first column, columns, sum of r1p, component)
  int* d_chbase = nullptr;        // chbase on the device
  int* Ek = nullptr;              // [q]
  int64_t bytes = 0;
};

int64_t dc_bytes(const DcCache* c) { return c ? c->bytes : 0; }

void dc_release(DcCache* c) {
  if (!c) return;
  cudaFree(c->u1g);
  cudaFree(c->u1off);
  cudaFree(c->u1base);
  cudaFree(c->rec);
  cudaFree(c->chunks);
  cudaFree(c->d_chbase);
  cudaFree(c->Ek);
  delete c;
}

// ---------------------------------------------------------------------------------------------
// per-handle operands
// ---------------------------------------------------------------------------------------------

// bound[t] = ||G||_F * prod_g max_i ||U_g[i, :]||_2 >= max |Z_t|  (one CTA per tensor)
__global__ void __launch_bounds__(256) dc_bound_kernel(const float2* __restrict__ pool,
                                                       const TensorDesc* __restrict__ desc, int n1, int n2, int n3,
                                                       float* __restrict__ bound) {
  const int t = blockIdx.x;
  const TensorDesc d = desc[t];
  const float2* G = pool + d.off;
  const int64_t ng = (int64_t)d.r1 * d.r2 * d.r3;
  __shared__ float red[256];
  float g2 = 0.f;
  for (int64_t o = threadIdx.x; o < ng; o += blockDim.x) g2 += G[o].x * G[o].x + G[o].y * G[o].y;
  red[threadIdx.x] = g2;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  float b = sqrtf(red[0]);
  __syncthreads();
  const float2* U = G + ng;
  const int n[3] = {n1, n2, n3}, r[3] = {d.r1, d.r2, d.r3};
  for (int g = 0; g < 3; ++g) {
    float m = 0.f;
    for (int i = threadIdx.x; i < n[g]; i += blockDim.x) {
      float s = 0.f;
      for (int a = 0; a < r[g]; ++a) {
        const float2 u = U[i + (int64_t)n[g] * a];
        s += u.x * u.x + u.y * u.y;
      }
      m = fmaxf(m, s);
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
      __syncthreads();
    }
    b *= sqrtf(red[0]);
    __syncthreads();
    U += (int64_t)n[g] * r[g];
  }
  if (threadIdx.x == 0) bound[t] = b;
}

// U1 of tensor (j, k) in groups of 32 rows: u1g[u1off + (a/2 * 32 + l) * 2 + a % 2] = U1[32 g1 + l, a]
// (zero for a >= r1 or rows beyond n1); grid (k ng1 + g1, j)
__global__ void __launch_bounds__(256) dc_u1_kernel(const float2* __restrict__ pool, const TensorDesc* __restrict__ desc,
                                                    const int64_t* __restrict__ u1off, int q, int n1, int ng1, int M,
                                                    float2* __restrict__ u1g) {
  const int kg = blockIdx.x, j = blockIdx.y;
  const int k = kg / ng1, g1 = kg % ng1;
  const TensorDesc d = desc[(int64_t)j * q + k];
  const int64_t o0 = u1off[(int64_t)kg * (M + 1) + j], o1 = u1off[(int64_t)kg * (M + 1) + j + 1];
  const float2* U1 = pool + d.off + (int64_t)d.r1 * d.r2 * d.r3;
  for (int64_t e = threadIdx.x; e < o1 - o0; e += blockDim.x) {
    const int a = (int)(e / 64) * 2 + (int)(e % 2), l = (int)((e / 2) % 32);
    const int i1 = 32 * g1 + l;
    u1g[o0 + e] = (a < d.r1 && i1 < n1) ? U1[i1 + (int64_t)n1 * a] : make_float2(0.f, 0.f);
  }
}

static int build_dc(Handle& h, cudaStream_t st) {
  ZBC_TRY(build_decomp_cache(h, st));
  DecompCache* c = h.cache;
  if (c->dc) return ZBC_OK;
  const int q = h.q, M = h.M, T = M * q;
  const int ng1 = (h.n1 + 31) / 32;
  auto* dc = new DcCache();
  dc->ng1 = ng1;
  std::vector<DcCol> cols(T);
  for (int t = 0; t < T; ++t) cols[t] = DcCol{c->host_desc[t].woff, c->host_desc[t].r1p, 0};
  // chunks: consecutive columns of one component, at most kDcCols of them and kDcRows rank rows
  dc->chbase.assign(q + 1, 0);
  for (int k = 0; k < q; ++k) {
    dc->chbase[k] = (int)dc->chunks_h.size();
    int j0 = 0;
    while (j0 < M) {
      int nc = 0, rs = 0;
      while (j0 + nc < M && nc < kDcCols && rs + cols[(int64_t)(j0 + nc) * q + k].r1p <= kDcRows) {
        rs += cols[(int64_t)(j0 + nc) * q + k].r1p;
        ++nc;
      }
      if (nc == 0) {  // r1p > kDcRows cannot happen for r1 <= kRmax
        dc_release(dc);
        set_error("rank too large for the tensor-core decompress-and-contract form");
        return ZBC_EINVAL;
      }
      dc->chunks_h.push_back(make_int4(j0, nc, rs, k));
      dc->max_rows = std::max(dc->max_rows, rs);
      j0 += nc;
    }
  }
  dc->chbase[q] = (int)dc->chunks_h.size();
  dc->NC = dc->chbase[q];
  std::vector<int64_t> u1off((size_t)q * ng1 * (M + 1));
  int64_t off = 0;
  for (int k = 0; k < q; ++k)
    for (int g1 = 0; g1 < ng1; ++g1) {
      int64_t* o = u1off.data() + ((size_t)k * ng1 + g1) * (M + 1);
      for (int j = 0; j < M; ++j) {
        o[j] = off;
        off += (int64_t)cols[(int64_t)j * q + k].r1p * 32;
      }
      o[M] = off;
    }
  std::vector<int64_t> u1base((size_t)q * ng1);
  for (size_t kg = 0; kg < u1base.size(); ++kg) u1base[kg] = u1off[kg * (M + 1)];
  std::vector<DcChunk> rec(dc->NC);
  for (int c = 0; c < dc->NC; ++c) {
    const int4 ch = dc->chunks_h[c];
    DcChunk& r = rec[c];
    std::memset(&r, 0, sizeof(r));
    r.j0 = ch.x;
    r.nc = ch.y;
    r.z = ch.z;
    r.k = ch.w;
    for (int cc = 0; cc < ch.y; ++cc) {
      const DcCol& col = cols[(int64_t)(ch.x + cc) * q + ch.w];
      r.r1p[cc] = col.r1p;
      r.woff[cc] = col.woff;
    }
    r.pre32 = u1off[(size_t)ch.w * ng1 * (M + 1) + ch.x] - u1off[(size_t)ch.w * ng1 * (M + 1)];
  }
  float* d_bound = nullptr;
  cudaError_t e = cudaMalloc(&dc->u1g, sizeof(float2) * std::max<int64_t>(1, off));
  if (e == cudaSuccess) e = cudaMalloc(&dc->u1off, sizeof(int64_t) * u1off.size());
  if (e == cudaSuccess) e = cudaMalloc(&dc->u1base, sizeof(int64_t) * u1base.size());
  if (e == cudaSuccess) e = cudaMalloc(&dc->rec, sizeof(DcChunk) * dc->NC);
  if (e == cudaSuccess) e = cudaMalloc(&dc->chunks, sizeof(int4) * dc->NC);
  if (e == cudaSuccess) e = cudaMalloc(&dc->Ek, sizeof(int) * q);
  if (e == cudaSuccess) e = cudaMalloc(&dc->d_chbase, sizeof(int) * (q + 1));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dc->d_chbase, dc->chbase.data(), sizeof(int) * (q + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMalloc(&d_bound, sizeof(float) * T);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dc->u1off, u1off.data(), sizeof(int64_t) * u1off.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dc->u1base, u1base.data(), sizeof(int64_t) * u1base.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dc->rec, rec.data(), sizeof(DcChunk) * dc->NC, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dc->chunks, dc->chunks_h.data(), sizeof(int4) * dc->NC, cudaMemcpyHostToDevice, st);
  std::vector<float> bound(T);
  if (e == cudaSuccess) {
    dc_bound_kernel<<<T, 256, 0, st>>>(h.d_pool, h.d_desc, h.n1, h.n2, h.n3, d_bound);
    dc_u1_kernel<<<dim3(q * ng1, M), 256, 0, st>>>(h.d_pool, h.d_desc, dc->u1off, q, h.n1, ng1, M, dc->u1g);
    count_launch(2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(bound.data(), d_bound, sizeof(float) * T, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_bound);
  if (e != cudaSuccess) {
    dc_release(dc);
    set_error("tensor-core decompress-and-contract operands: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? ZBC_ENOMEM : ZBC_ECUDA;
  }
  dc->Ek_h.assign(q, 0);
  for (int k = 0; k < q; ++k) {
    float mb = 0.f;
    for (int j = 0; j < M; ++j) mb = std::max(mb, bound[(size_t)j * q + k]);
    int ex = 0;
    if (mb > 0.f) std::frexp(mb, &ex);  // mb < 2^ex
    // one more for the rounding of the FP32 sums; kept in [-100, 127] so that the generators'
    // factor 2^(kDcShift - E_k) is a normal float (a bound below 2^-100 only scales tiny values up)
    dc->Ek_h[k] = std::min(127, std::max(-100, ex + 1));
  }
  e = cudaMemcpyAsync(dc->Ek, dc->Ek_h.data(), sizeof(int) * q, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    dc_release(dc);
    set_error("tensor-core decompress-and-contract operands: %s", cudaGetErrorString(e));
    return ZBC_ECUDA;
  }
  dc->bytes = (int64_t)(sizeof(float2) * std::max<int64_t>(1, off) + sizeof(int64_t) * u1off.size() +
                        sizeof(int64_t) * u1base.size() + sizeof(DcChunk) * dc->NC + sizeof(int4) * dc->NC +
                        sizeof(int) * (2 * q + 1));
  c->dc = dc;
  return ZBC_OK;
}

// ---------------------------------------------------------------------------------------------
// per-call operands: exponents of X' and the B blocks
// ---------------------------------------------------------------------------------------------

// ex[s] = exponent of max_j |Re|, |Im| X'[j, s] (0 for a zero column or s >= p); non-finite values
// set kErrNonFinite.  One CTA per padded right-hand side.
__global__ void __launch_bounds__(256) dc_x_kernel(const float2* __restrict__ X, int64_t ldx, int M, int p,
                                                   int* __restrict__ ex, int* __restrict__ err) {
  const int s = blockIdx.x;
  __shared__ float wmax[8];
  float mx = 0.f;
  bool finite = true;
  if (s < p)
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
      const float2 v = X[j + ldx * s];
      finite = finite && isfinite(v.x) && isfinite(v.y);
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
  if (!finite) atomicOr(err, kErrNonFinite);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wmax[w]);
    int e = 0;
    if (m > 0.f && isfinite(m)) frexpf(m, &e);
    ex[s] = e;
  }
}

// byte offset of element (row n, K index kk < 16) of a 16-wide fp16 K-major operand in the
// canonical no-swizzle layout (8-row x 16-byte core matrices; LBO 128, SBO 256)
__host__ __device__ __forceinline__ uint32_t dc_off(uint32_t n, uint32_t kk) {
  return (n >> 3) * 256u + (kk >> 3) * 128u + (n & 7u) * 16u + (kk & 7u) * 2u;
}

// K slots of a chunk: kk = 8 h + 4 part + c (h, part in {0, 1}, c < 4) holds column j0 + 4 h + c,
// its real part (part 0) or imaginary part (part 1), so that a generator thread writes the 8 slots
// of its four columns as one 16-byte store.
// B blocks: [pass sc][chunk c][term hi | lo][2P rows][16]: row n < P (Re Y of s = n): Re X'[j, s]
// in the real slots, -Im X'[j, s] in the imaginary slots; row n >= P (Im Y of s = n - P): Im X'
// and Re X' (zero beyond the chunk), X' scaled by 2^(kDcShift - ex_s).
// One thread per (sc, c, n, kk).
__global__ void __launch_bounds__(256) dc_b_kernel(const float2* __restrict__ X, int64_t ldx, int p, int P, int NC,
                                                   int nsc, const int4* __restrict__ chunks,
                                                   const int* __restrict__ ex, __half* __restrict__ B) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)2 * P * 16;
  if (e >= (int64_t)nsc * NC * per) return;
  const int kk = (int)(e % 16);
  const int n = (int)((e / 16) % (2 * P));
  const int64_t blk = e / per;  // sc * NC + c
  const int c = (int)(blk % NC), sc = (int)(blk / NC);
  const int4 ch = chunks[c];
  const int jl = (kk >> 3) * 4 + (kk & 3), s = sc * P + (n % P);
  float v = 0.f;
  if (jl < ch.y && s < p) {
    const float2 x = X[ch.x + jl + ldx * s];
    const bool re_row = n < P, first = ((kk >> 2) & 1) == 0;
    v = re_row ? (first ? x.x : -x.y) : (first ? x.y : x.x);
    v = ldexpf(v, kDcShift - ex[s]);  // on the value: 2^(kDcShift - ex) alone may not be a float
  }
  const __half hi = __float2half_rn(v);
  const __half lo = __float2half_rn(v - __half2float(hi));
  unsigned char* base = reinterpret_cast<unsigned char*>(B) + blk * 2 * per * 2;
  *reinterpret_cast<__half*>(base + dc_off(n, kk)) = hi;
  *reinterpret_cast<__half*>(base + per * 2 + dc_off(n, kk)) = lo;
}

// ---------------------------------------------------------------------------------------------
// the product kernel
// ---------------------------------------------------------------------------------------------

struct DcParams {
  const unsigned char* B;    // per call, [nsc][NC][2][2P][16] fp16
  const float2* u1g;
  const int64_t* u1base;
  const DcChunk* rec;
  const int4* chunks;
  const int* chbase;         // device [q + 1]
  const float2* Wc;          // the decompression cache
  const int* Ek;
  const int* ex;
  float2* Y;
  int64_t ldy, nv;
  int* err;
  int q, M, n1, n23, ng1, nb23, nsc, p, S, NC;
  uint32_t stage_bytes, w_off, b_off, h_off, a_off;
  int64_t nitems;
};

// item -> (component k, pass sc, i23 block b, i1 group g1); g1 varies fastest, so the CTAs running
// at one time read the same W blocks (from L2)
__device__ __forceinline__ void dc_item(const DcParams& prm, int64_t it, int& k, int& sc, int& b, int& g1) {
  g1 = (int)(it % prm.ng1);
  int64_t t = it / prm.ng1;
  b = (int)(t % prm.nb23);
  t /= prm.nb23;
  sc = (int)(t % prm.nsc);
  k = (int)(t / prm.nsc);
}

__device__ __forceinline__ void tmem_st8_f(uint32_t taddr, const float (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
}
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// P right-hand sides per pass (N = 2P), T tiles of 128 voxels (4T values of i23) per item
template <int P, int T>
__global__ void __launch_bounds__(kDcThreads, 1) matvec_dc_kernel(const DcParams prm) {
  constexpr int N = 2 * P;
  constexpr int H = P / 2;                       // right-hand sides per warpgroup in the folds / epilogue
  constexpr uint32_t kTile = 128 * 32;           // bytes of one A term of one tile (128 rows x 16 fp16)
  constexpr uint32_t kABuf = (uint32_t)T * 2 * kTile;
  constexpr uint32_t kTmemCols = 2 * T * N <= 32 ? 32 : 2 * T * N <= 64 ? 64 : 2 * T * N <= 128 ? 128
                                 : 2 * T * N <= 256 ? 256 : 512;
  static_assert(2 * T * N <= 512, "D and S must fit TMEM");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t sfull[kDcMaxStages], sempty[kDcMaxStages], afull[2], aempty[2], dfull, dempty, mdone;
  __shared__ uint32_t tbase;
  __shared__ volatile int abort_flag;
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* abuf = smem + prm.a_off;
  const int S = prm.S;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  if (warp == 0) tc::tmem_alloc(&tbase, kTmemCols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&sfull[s], 1);
      tc::mbar_init(&sempty[s], 1 + 8);  // the MMA warp's commit and the 8 generator warps
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&afull[b], 8);
      tc::mbar_init(&aempty[b], 1);
    }
    tc::mbar_init(&dfull, 1);
    tc::mbar_init(&dempty, 8);
    tc::mbar_init(&mdone, 1);
    abort_flag = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tD = tbase;          // D: tile t at columns [t N, (t + 1) N)
  const uint32_t tS = tbase + T * N;  // S: the same layout

  if (warp == 8) {
    // ---------------- copy warp ----------------
    // The lanes share each chunk: its 128-byte record is one coalesced load (issued a chunk ahead,
    // so that no global-memory latency sits between two chunks), lane cc < nc writes column cc's
    // header entries and issues its W copy, lane 0 waits for the free stage, sets the barrier's
    // transaction count and issues the U1 and B copies.
    constexpr unsigned kAll = 0xffffffffu;
    uint32_t cnt = 0;
    bool stop = false;
    for (int64_t it = blockIdx.x; it < prm.nitems && !stop; it += gridDim.x) {
      int k, sc, b, g1;
      dc_item(prm, it, k, sc, b, g1);
      const int i23_0 = b * 4 * T;
      const int rows = min(4 * T, prm.n23 - i23_0);
      const int64_t ubase = prm.u1base[(int64_t)k * prm.ng1 + g1];
      const int c0 = prm.chbase[k], c1 = prm.chbase[k + 1];
      int word = reinterpret_cast<const int*>(prm.rec + c0)[lane];
      for (int c = c0; c < c1; ++c, ++cnt) {
        const int st = cnt % S;
        const int wnext = c + 1 < c1 ? reinterpret_cast<const int*>(prm.rec + c + 1)[lane] : 0;
        bool ok = true;
        if (lane == 0) ok = !abort_flag && (cnt < (uint32_t)S || tc::mbar_wait_idle(&sempty[st], ((cnt / S) - 1) & 1));
        if (!__shfl_sync(kAll, ok, 0)) {
          if (lane == 0) abort_flag = 1;
          stop = true;
          break;
        }
        // record words: 1 nc, 2 sum of r1p, 4 + cc r1p, 12 + 2 cc / 13 + 2 cc woff, 28 / 29 pre32
        const int nc = __shfl_sync(kAll, word, 1);
        const int z = __shfl_sync(kAll, word, 2);
        const int cl = lane & (kDcCols - 1);
        const int r1p = __shfl_sync(kAll, word, 4 + cl);
        const uint32_t wlo = (uint32_t)__shfl_sync(kAll, word, 12 + 2 * cl);
        const uint32_t whi = (uint32_t)__shfl_sync(kAll, word, 13 + 2 * cl);
        const uint32_t plo = (uint32_t)__shfl_sync(kAll, word, 28);
        const uint32_t phi = (uint32_t)__shfl_sync(kAll, word, 29);
        const bool mine = lane < nc;
        int pre = mine ? r1p : 0;  // inclusive sum of r1p over lanes 0 .. lane, then exclusive
#pragma unroll
        for (int o = 1; o < kDcCols; o <<= 1) {
          const int v = __shfl_up_sync(kAll, pre, o);
          if (lane >= o) pre += v;
        }
        pre -= mine ? r1p : 0;
        unsigned char* sb = smem + (size_t)st * prm.stage_bytes;
        DcHdr* hd = reinterpret_cast<DcHdr*>(sb + prm.h_off);
        if (mine) {
          hd->r1p[lane] = r1p;
          hd->uo[lane] = pre * 16;     // float4 units: 32 rows x r1p complex64 per column
          hd->wo[lane] = pre * 2 * T;  // float4 units: 4T rows x r1p complex64 per column
        }
        if (lane == 0) hd->nc = nc;
        __threadfence_block();
        __syncwarp();  // the header stores come before lane 0's arrive (which releases them)
        const uint32_t ub = (uint32_t)z * 32u * 8u, wb = (uint32_t)rows * (uint32_t)z * 8u;
        const uint32_t bb = (uint32_t)(2 * N * 32);
        if (lane == 0) mbar_arrive_expect_tx(&sfull[st], ub + wb + bb);
        __syncwarp();  // the transaction count is set before any copy is issued
        if (lane == 0) {
          const int64_t pre32 = (int64_t)(((uint64_t)phi << 32) | plo);
          bulk_g2s(sb, prm.u1g + ubase + pre32, ub, &sfull[st]);
          bulk_g2s(sb + prm.b_off, prm.B + ((int64_t)sc * prm.NC + c) * bb, bb, &sfull[st]);
        }
        if (mine) {
          const int64_t woff = (int64_t)(((uint64_t)whi << 32) | wlo);
          bulk_g2s(sb + prm.w_off + (uint32_t)pre * (uint32_t)(4 * T) * 8u, prm.Wc + woff + (int64_t)i23_0 * r1p,
                   (uint32_t)rows * (uint32_t)r1p * 8u, &sfull[st]);
        }
        word = wnext;
      }
    }
    if (lane == 0 && abort_flag)  // let the copies in flight land before the CTA exits
      for (uint32_t c = cnt > (uint32_t)S ? cnt - S : 0; c < cnt; ++c) tc::mbar_wait(&sfull[c % S], (c / S) & 1);
    __syncwarp();
  } else if (warp == 9) {
    // ---------------- MMA warp ----------------
    if (lane == 0) {
      const uint32_t idesc = tc::instr_desc(128, N, 0);  // kind::f16, f16 operands, FP32 D
      uint32_t gc = 0, gs = 0;
      for (int64_t it = blockIdx.x; it < prm.nitems && !abort_flag; it += gridDim.x) {
        int k, sc, b, g1;
        dc_item(prm, it, k, sc, b, g1);
        const int nch = prm.chbase[k + 1] - prm.chbase[k];
        for (int cl = 0; cl < nch && !abort_flag; ++cl, ++gc) {
          const bool first = cl % kDcSeg == 0, last = cl % kDcSeg == kDcSeg - 1 || cl == nch - 1;
          const int st = gc % S, ab = gc & 1;
          bool ok = !(first && gs >= 1) || tc::mbar_wait_idle(&dempty, (gs - 1) & 1);
          ok = ok && tc::mbar_wait_idle(&sfull[st], (gc / S) & 1) && tc::mbar_wait_idle(&afull[ab], (gc >> 1) & 1);
          if (!ok) {
            abort_flag = 1;
            break;
          }
          tc::fence_after();
          const uint32_t sb = tc::smem_u32(smem + (size_t)st * prm.stage_bytes + prm.b_off);
          const uint64_t bh = tc::smem_desc(sb, 128, 256), bl = tc::smem_desc(sb + N * 32, 128, 256);
          const uint32_t a0 = tc::smem_u32(abuf + ab * kABuf);
#pragma unroll
          for (int t = 0; t < T; ++t) {
            const uint64_t ah = tc::smem_desc(a0 + (2 * t) * kTile, 128, 256);
            const uint64_t al = tc::smem_desc(a0 + (2 * t + 1) * kTile, 128, 256);
            const uint32_t d = tD + t * N;
            tc::mma<0>(d, ah, bh, idesc, first ? 0u : 1u);  // hi . hi
            tc::mma<0>(d, ah, bl, idesc, 1u);                // hi . lo
            tc::mma<0>(d, al, bh, idesc, 1u);                // lo . hi
          }
          tc::commit(&sempty[st]);
          tc::commit(&aempty[ab]);
          if (last) {
            tc::commit(&dfull);
            ++gs;
          }
        }
      }
      // every MMA issued has completed before the CTA leaves (TMEM is freed below)
      tc::commit(&mdone);
      tc::mbar_wait(&mdone, 0);
    }
    __syncwarp();
  } else {
    // ---------------- 8 warps: generate A, fold D into S, write Y ----------------
    const int hg = warp >> 2;                      // warpgroup: columns [4 hg, 4 hg + 4) of a chunk
    const int w4 = warp & 3;                       // TMEM lanes [32 w4, 32 w4 + 32)
    // Row 32 b + i1 of a tile is the voxel (32 g1 + i1, i23_0 + 4 t + b).  The folds and the
    // epilogue read lane row = 32 w4 + lane; the generator's thread takes i1 = 8 w4 + (lane & 7) and
    // b = lane >> 3, so that a warp's U1 loads touch 8 rows (one wavefront) and the four warps of a
    // warpgroup load disjoint U1 rows.
    const int gi1 = 8 * w4 + (lane & 7), gb = lane >> 3;
    const int row = 32 * gb + gi1;                 // the generator's A row within a tile
    const uint32_t lanebase = (uint32_t)(w4 * 32) << 16;
    uint32_t gc = 0, gs = 0;
    bool bad = false;
    for (int64_t it = blockIdx.x; it < prm.nitems && !bad; it += gridDim.x) {
      if (__any_sync(0xffffffffu, abort_flag != 0)) {
        bad = true;
        break;
      }
      int k, sc, b, g1;
      dc_item(prm, it, k, sc, b, g1);
      const int i23_0 = b * 4 * T;
      const int nch = prm.chbase[k + 1] - prm.chbase[k];
      const int nseg = (nch + kDcSeg - 1) / kDcSeg;
      const float fz = ldexpf(1.f, kDcShift - prm.Ek[k]);
      const uint32_t gs0 = gs;
      // S (+)= D for the local segment sl (round-to-nearest FP32 adds); S = D for the first
      auto fold = [&](int sl) {
        const bool ok = !abort_flag && tc::mbar_wait(&dfull, (gs0 + sl) & 1);
        if (!__all_sync(0xffffffffu, ok)) {
          bad = true;
          return;
        }
        tc::fence_after();
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
          for (int part = 0; part < 2; ++part)
#pragma unroll
            for (int s0 = 0; s0 < H; s0 += 8) {
              const uint32_t col = (uint32_t)(t * N + part * P + hg * H + s0);
              float dv[8], sv[8];
              tmem_ld8_nowait(tD + lanebase + col, dv);
              if (sl > 0) tmem_ld8_nowait(tS + lanebase + col, sv);
              tmem_wait_ld();
              if (sl > 0) {
#pragma unroll
                for (int i = 0; i < 8; ++i) dv[i] += sv[i];
              }
              tmem_st8_f(tS + lanebase + col, dv);
            }
        tc::tmem_wait_st();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive1(&dempty);
      };
      for (int cl = 0; cl < nch && !bad; ++cl, ++gc) {
        const int st = gc % S, ab = gc & 1;
        bool ok = !abort_flag && (gc < 2 || tc::mbar_wait(&aempty[ab], ((gc >> 1) - 1) & 1));
        ok = ok && tc::mbar_wait(&sfull[st], (gc / S) & 1);
        if (!__all_sync(0xffffffffu, ok)) {
          bad = true;
          break;
        }
        const unsigned char* sb = smem + (size_t)st * prm.stage_bytes;
        const DcHdr* hd = reinterpret_cast<const DcHdr*>(sb + prm.h_off);
        const int nc = hd->nc;
        const float4* __restrict__ Us = reinterpret_cast<const float4*>(sb) + gi1;
        const float4* __restrict__ Ws = reinterpret_cast<const float4*>(sb + prm.w_off);
        // T <= 2: the warpgroup's four columns advance together, one rank pair a2 per step: a step
        // loads the U1 pair and the T W pairs of each column, then does the four columns' FMAs, so
        // four independent load / FMA chains are in flight (a column's own chain is only r1 / 2
        // long).  T = 4: one column after the other, each with its next rank pair's operands loaded
        // during the current pair's FMAs (measured faster there: four columns of T = 4 need more
        // registers than the launch leaves).  Per column, even and odd a accumulate separately,
        // each over a in increasing order, in both forms.
        float zr[T][4], zi[T][4];
        if constexpr (T <= 2) {
          constexpr int G = 4;
#pragma unroll
          for (int g0 = 0; g0 < 4; g0 += G) {
            float2 ae[G][T], ao[G][T];
            int n2c[G];
            const float4* Uc[G];
            const float4* Wcol[G];
            int n2max = 0;
#pragma unroll
            for (int c = 0; c < G; ++c) {
              const int cc = 4 * hg + g0 + c;
              const bool on = cc < nc;
              n2c[c] = on ? hd->r1p[cc] / 2 : 0;
              Uc[c] = Us + (on ? hd->uo[cc] : 0);                      // pair a2 at Uc[32 a2]
              Wcol[c] = Ws + (on ? hd->wo[cc] : 0) + gb * n2c[c];      // tile t at Wcol[4 n2 t + a2]
              n2max = max(n2max, n2c[c]);
#pragma unroll
              for (int t = 0; t < T; ++t) ae[c][t] = ao[c][t] = make_float2(0.f, 0.f);
            }
            for (int a2 = 0; a2 < n2max; ++a2) {
              float4 u[G], wv[G][T];
#pragma unroll
              for (int c = 0; c < G; ++c)
                if (a2 < n2c[c]) {
                  u[c] = Uc[c][32 * a2];
#pragma unroll
                  for (int t = 0; t < T; ++t) wv[c][t] = Wcol[c][4 * n2c[c] * t + a2];
                }
#pragma unroll
              for (int c = 0; c < G; ++c)
                if (a2 < n2c[c]) {
#pragma unroll
                  for (int t = 0; t < T; ++t) {
                    const float4 w = wv[c][t];
                    ae[c][t].x = fmaf(u[c].x, w.x, fmaf(-u[c].y, w.y, ae[c][t].x));
                    ae[c][t].y = fmaf(u[c].x, w.y, fmaf(u[c].y, w.x, ae[c][t].y));
                    ao[c][t].x = fmaf(u[c].z, w.z, fmaf(-u[c].w, w.w, ao[c][t].x));
                    ao[c][t].y = fmaf(u[c].z, w.w, fmaf(u[c].w, w.z, ao[c][t].y));
                  }
                }
            }
#pragma unroll
            for (int c = 0; c < G; ++c)
#pragma unroll
              for (int t = 0; t < T; ++t) {
                zr[t][g0 + c] = (ae[c][t].x + ao[c][t].x) * fz;
                zi[t][g0 + c] = (ae[c][t].y + ao[c][t].y) * fz;
              }
          }
        } else {
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) {
            const int cc = 4 * hg + c4;
            float2 ae[T], ao[T];
#pragma unroll
            for (int t = 0; t < T; ++t) ae[t] = ao[t] = make_float2(0.f, 0.f);
            if (cc < nc) {
              const int n2 = hd->r1p[cc] / 2;
              const float4* U = Us + hd->uo[cc];                       // pair a2 at U[32 a2]
              const float4* W = Ws + hd->wo[cc] + gb * n2;             // tile t at W[4 n2 t + a2]
              // two register sets, loaded alternately one rank pair ahead of their use
              auto macc = [&](const float4& u, const float4 (&wv)[T]) {
#pragma unroll
                for (int t = 0; t < T; ++t) {
                  ae[t].x = fmaf(u.x, wv[t].x, fmaf(-u.y, wv[t].y, ae[t].x));
                  ae[t].y = fmaf(u.x, wv[t].y, fmaf(u.y, wv[t].x, ae[t].y));
                  ao[t].x = fmaf(u.z, wv[t].z, fmaf(-u.w, wv[t].w, ao[t].x));
                  ao[t].y = fmaf(u.z, wv[t].w, fmaf(u.w, wv[t].z, ao[t].y));
                }
              };
              float4 u0 = U[0], u1;
              float4 w0[T], w1[T];
#pragma unroll
              for (int t = 0; t < T; ++t) w0[t] = W[4 * n2 * t];
              int a2 = 0;
              for (; a2 + 1 < n2; a2 += 2) {
                u1 = U[32 * (a2 + 1)];
#pragma unroll
                for (int t = 0; t < T; ++t) w1[t] = W[4 * n2 * t + a2 + 1];
                macc(u0, w0);
                if (a2 + 2 < n2) {
                  u0 = U[32 * (a2 + 2)];
#pragma unroll
                  for (int t = 0; t < T; ++t) w0[t] = W[4 * n2 * t + a2 + 2];
                }
                macc(u1, w1);
              }
              if (a2 < n2) macc(u0, w0);  // an odd number of rank pairs
            }
#pragma unroll
            for (int t = 0; t < T; ++t) {
              zr[t][c4] = (ae[t].x + ao[t].x) * fz;
              zi[t][c4] = (ae[t].y + ao[t].y) * fz;
            }
          }
        }
        // A pieces: Re Z of columns 4 hg .. 4 hg + 3 at K = 8 hg .. 8 hg + 3, Im Z at K = 8 hg + 4 ..,
        // one 16-byte store per term (the 32 rows of a warp then fill every bank once per wavefront)
        unsigned char* ab0 = abuf + ab * kABuf;
#pragma unroll
        for (int t = 0; t < T; ++t) {
          uint32_t hr[2], hi_[2], lr[2], li[2];
#pragma unroll
          for (int pr = 0; pr < 2; ++pr) {
            const __half2 h2r = __floats2half2_rn(zr[t][2 * pr], zr[t][2 * pr + 1]);
            const __half2 h2i = __floats2half2_rn(zi[t][2 * pr], zi[t][2 * pr + 1]);
            const float2 fr = __half22float2(h2r), fi = __half22float2(h2i);
            const __half2 l2r = __floats2half2_rn(zr[t][2 * pr] - fr.x, zr[t][2 * pr + 1] - fr.y);
            const __half2 l2i = __floats2half2_rn(zi[t][2 * pr] - fi.x, zi[t][2 * pr + 1] - fi.y);
            hr[pr] = *reinterpret_cast<const uint32_t*>(&h2r);
            hi_[pr] = *reinterpret_cast<const uint32_t*>(&h2i);
            lr[pr] = *reinterpret_cast<const uint32_t*>(&l2r);
            li[pr] = *reinterpret_cast<const uint32_t*>(&l2i);
          }
          unsigned char* th = ab0 + (2 * t) * kTile;
          unsigned char* tl = ab0 + (2 * t + 1) * kTile;
          *reinterpret_cast<uint4*>(th + dc_off(row, 8 * hg)) = make_uint4(hr[0], hr[1], hi_[0], hi_[1]);
          *reinterpret_cast<uint4*>(tl + dc_off(row, 8 * hg)) = make_uint4(lr[0], lr[1], li[0], li[1]);
        }
        tc::fence_proxy_async();  // the generic-proxy stores above are read by the tensor cores
        __syncwarp();
        if (lane == 0) {
          mbar_arrive1(&afull[ab]);
          mbar_arrive1(&sempty[st]);
        }
        // fold segment sl - 1 once the first chunk of segment sl is generated (its MMAs wait for
        // the fold; the generation of the next chunk does not)
        if (cl % kDcSeg == 0 && cl > 0) fold(cl / kDcSeg - 1);
      }
      if (!bad) fold(nseg - 1);
      gs = gs0 + nseg;
      if (bad) {
        if (lane == 0) abort_flag = 1;
        break;
      }
      // Y = S 2^(E_k + ex_s - 2 kDcShift): voxel (i1 = 32 g1 + lane, i23 = i23_0 + 4 t + w4)
      const int i1 = 32 * g1 + lane;
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const int i23 = i23_0 + 4 * t + w4;
#pragma unroll
        for (int s0 = 0; s0 < H; s0 += 8) {
          float re[8], im[8];
          tmem_ld8_nowait(tS + lanebase + (uint32_t)(t * N + hg * H + s0), re);
          tmem_ld8_nowait(tS + lanebase + (uint32_t)(t * N + P + hg * H + s0), im);
          tmem_wait_ld();
          if (i1 < prm.n1 && i23 < prm.n23) {
            float2* y = prm.Y + (int64_t)k * prm.nv + i1 + (int64_t)prm.n1 * i23;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int s = sc * P + hg * H + s0 + i;
              if (s < prm.p) {
                const int sh = prm.Ek[k] + prm.ex[s] - 2 * kDcShift;
                y[prm.ldy * s] = make_float2(ldexpf(re[i], sh), ldexpf(im[i], sh));
              }
            }
          }
        }
      }
      tc::fence_before();
    }
    if (bad && lane == 0) abort_flag = 1;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (threadIdx.x == 0 && abort_flag) atomicOr(prm.err, kErrTimeout);
  if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

template <int P, int T>
static int matvec_dc_p(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  const DcCache& dc = *h.cache->dc;
  DcParams prm;
  prm.q = h.q;
  prm.M = h.M;
  prm.p = p;
  prm.n1 = h.n1;
  prm.n23 = h.n2 * h.n3;
  prm.ng1 = dc.ng1;
  prm.nb23 = ceil_div(prm.n23, 4 * T);
  prm.nsc = ceil_div(p, P);
  prm.NC = dc.NC;
  prm.nitems = (int64_t)h.q * prm.nsc * prm.nb23 * prm.ng1;
  prm.ldy = ldy;
  prm.nv = h.nv();
  // stage: U1 (rows x 32 complex64), W (4T x rows complex64), B (2 terms x 2P x 32 B), header;
  // rows = the handle's largest chunk
  const uint32_t rows = (uint32_t)dc.max_rows;
  prm.w_off = rows * 32u * 8u;
  prm.b_off = prm.w_off + (uint32_t)(4 * T) * rows * 8u;
  prm.h_off = prm.b_off + (uint32_t)(2 * 2 * P * 32);
  prm.stage_bytes = (prm.h_off + (uint32_t)sizeof(DcHdr) + 1023) / 1024 * 1024;
  const uint32_t abytes = 2u * T * 2 * 128 * 32;
  const size_t budget = 226 * 1024;
  prm.S = (int)std::min<size_t>(kDcMaxStages, (budget - 1024 - abytes) / prm.stage_bytes);
  if (prm.S < 2) {
    set_error("tensor-core decompress-and-contract: stage layout does not fit shared memory");
    return ZBC_EINVAL;
  }
  prm.a_off = (uint32_t)prm.S * prm.stage_bytes;
  const size_t smem = 1024 + (size_t)prm.a_off + abytes;
  // per call: exponents and B blocks
  const size_t bbytes = (size_t)prm.nsc * prm.NC * 2 * 2 * P * 32;
  const int ns = prm.nsc * P;
  ZBC_TRY(h.work_xt.ensure(bbytes + sizeof(int) * (size_t)ns));
  unsigned char* B = (unsigned char*)h.work_xt.ptr;
  int* ex = (int*)(B + bbytes);
  dc_x_kernel<<<ns, 256, 0, st>>>(X, ldx, h.M, p, ex, (int*)h.work_err.ptr);
  const int64_t nb = (int64_t)prm.nsc * prm.NC * 2 * P * 16;
  dc_b_kernel<<<ceil_div(nb, 256), 256, 0, st>>>(X, ldx, p, P, prm.NC, prm.nsc, dc.chunks, ex, (__half*)B);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch(2);
  prm.B = B;
  prm.u1g = dc.u1g;
  prm.u1base = dc.u1base;
  prm.rec = dc.rec;
  prm.chunks = dc.chunks;
  prm.chbase = dc.d_chbase;
  prm.Wc = h.cache->data;
  prm.Ek = dc.Ek;
  prm.ex = ex;
  prm.Y = Y;
  prm.err = (int*)h.work_err.ptr;
  ZBC_TRY((set_smem_limit<matvec_dc_kernel<P, T>>((int)budget)));
  const int grid = (int)std::min<int64_t>(sm_count(), prm.nitems);
  matvec_dc_kernel<P, T><<<grid, kDcThreads, smem, st>>>(prm);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

// Y = Z X on the handle's stored columns (X has M rows): passes of 16, 32, 64 or 128 right-hand
// sides (T = 4, 4, 2, 1 tiles of 128 voxels per item)
int matvec_dc(Handle& h, const float2* X, int64_t ldx, int p, float2* Y, int64_t ldy, cudaStream_t st) {
  ZBC_TRY(build_dc(h, st));
  if (p <= 16) return matvec_dc_p<16, 4>(h, X, ldx, p, Y, ldy, st);
  if (p <= 32) return matvec_dc_p<32, 4>(h, X, ldx, p, Y, ldy, st);
  if (p <= 64) return matvec_dc_p<64, 2>(h, X, ldx, p, Y, ldy, st);
  return matvec_dc_p<128, 1>(h, X, ldx, p, Y, ldy, st);
}

}  // namespace zbc
