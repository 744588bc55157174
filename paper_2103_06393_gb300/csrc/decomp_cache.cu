// Decompression cache of a handle: per tensor (column j, component k)
//   W_j[i3][i2][a] = sum_{b,c} G_j[a,b,c] U2_j[i2,b] U3_j[i3,c]     (= G x2 U2 x3 U3, Eq. Tucker)
//   U1_j blocked by i1 tiles: [t1][a][i1 - t1 B1], row stride B1p
// with a < r1p (r1 rounded up to 2) and zero padding, so that the per-tile blocks are 16-byte
// aligned contiguous runs.  Both depend only on the compressed data, so they are computed once
// (first product call) and reused by every product; the last mode product with U1 stays in the
// product kernels.  Size: sum over tensors of (n2 n3 + nb1 B1p) r1p complex64.
#include <algorithm>

#include <cuda_fp16.h>

#include "decomp.cuh"
#include "tc_common.cuh"

namespace zbc {

void cache_release(DecompCache* c) {
  if (!c) return;
  if (c->data) cudaFree(c->data);
  if (c->d_desc) cudaFree(c->d_desc);
  if (c->half) cudaFree(c->half);
  if (c->d_half) cudaFree(c->d_half);
  mode1_release(c->mode1);
  dc_release(c->dc);
  delete c;
}

void half_release(DecompCache* c) {
  if (!c) return;
  if (c->half) cudaFree(c->half);
  if (c->d_half) cudaFree(c->d_half);
  c->half = nullptr;
  c->d_half = nullptr;
  c->bytes -= c->half_bytes;
  c->half_bytes = 0;
}

// one CTA per (i3, tensor): P[a][b] = sum_c G[a,b,c] U3[i3,c]; W[i3][i2][a] = sum_b P[a][b] U2[i2,b]
__global__ void __launch_bounds__(256) build_w_kernel(const float2* __restrict__ pool, const TensorDesc* __restrict__ desc,
                                                      const CacheDesc* __restrict__ cdesc, int n1, int n2, int n3,
                                                      float2* __restrict__ cache) {
  extern __shared__ float2 Ps[];  // r1 * r2
  const int i3 = blockIdx.x, t = blockIdx.y;
  const TensorDesc d = desc[t];
  const CacheDesc cd = cdesc[t];
  const float2* G = pool + d.off;
  const float2* U2 = G + (int64_t)d.r1 * d.r2 * d.r3 + (int64_t)n1 * d.r1;
  const float2* U3 = U2 + (int64_t)n2 * d.r2;
  const int64_t st = (int64_t)d.r1 * d.r2;
  for (int o = threadIdx.x; o < d.r1 * d.r2; o += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int c = 0; c < d.r3; ++c) acc = cfma(G[o + st * c], U3[i3 + (int64_t)n3 * c], acc);
    Ps[o] = acc;  // o = a + r1 * b
  }
  __syncthreads();
  float2* W = cache + cd.woff + (int64_t)i3 * n2 * cd.r1p;
  for (int o = threadIdx.x; o < n2 * cd.r1p; o += blockDim.x) {
    const int a = o % cd.r1p, i2 = o / cd.r1p;
    float2 acc = make_float2(0.f, 0.f);
    if (a < d.r1)
      for (int b = 0; b < d.r2; ++b) acc = cfma(Ps[a + d.r1 * b], U2[i2 + (int64_t)n2 * b], acc);
    W[o] = acc;
  }
}

__global__ void __launch_bounds__(256) build_u1_kernel(const float2* __restrict__ pool, const TensorDesc* __restrict__ desc,
                                                       const CacheDesc* __restrict__ cdesc, int n1,
                                                       float2* __restrict__ cache) {
  const int t = blockIdx.y;
  const TensorDesc d = desc[t];
  const CacheDesc cd = cdesc[t];
  const float2* U1 = pool + d.off + (int64_t)d.r1 * d.r2 * d.r3;
  const int B1 = tile_b1(n1), B1p = tile_b1p(n1), nb1 = (n1 + B1 - 1) / B1;
  const int per = cd.r1p * B1p;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nb1 * per; o += gridDim.x * blockDim.x) {
    const int t1 = o / per, rem = o % per;
    const int a = rem / B1p, il = rem % B1p;
    const int i1 = t1 * B1 + il;
    cache[cd.uoff + o] = (a < d.r1 && il < B1 && i1 < n1) ? U1[i1 + (int64_t)n1 * a] : make_float2(0.f, 0.f);
  }
}

int build_decomp_cache(Handle& h, cudaStream_t st) {
  if (h.cache) return ZBC_OK;
  const int T = (int)h.desc.size();
  std::vector<CacheDesc> cd(T);
  int64_t off = 0;
  int rmax = 0, r2max = 0;
  const int nb1 = (h.n1 + tile_b1(h.n1) - 1) / tile_b1(h.n1);
  for (int t = 0; t < T; ++t) {
    const TensorDesc& d = h.desc[t];
    cd[t].r1 = d.r1;
    cd[t].r1p = (d.r1 + 1) / 2 * 2;
    cd[t].woff = off;
    off += (int64_t)h.n2 * h.n3 * cd[t].r1p;
    cd[t].uoff = off;
    off += (int64_t)nb1 * tile_b1p(h.n1) * cd[t].r1p;
    rmax = std::max(rmax, cd[t].r1p);
    r2max = std::max(r2max, d.r1 * d.r2);
  }
  if (rmax > kRmax) {
    set_error("product kernels support ranks r1 <= %d (handle has %d)", kRmax, rmax);
    return ZBC_EINVAL;
  }
  // the error word of the product kernels lives as long as the cache (no allocation later)
  ZBC_TRY(h.work_err.ensure(sizeof(int)));
  ZBC_TRY_CUDA(cudaMemsetAsync(h.work_err.ptr, 0, sizeof(int), st));
  auto* c = new DecompCache();
  c->elems = off;
  c->host_desc = cd;
  cudaError_t e = cudaMalloc(&c->data, sizeof(float2) * std::max<int64_t>(1, off));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_desc, sizeof(CacheDesc) * T);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_desc, cd.data(), sizeof(CacheDesc) * T, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    cache_release(c);
    set_error("decompression cache allocation failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? ZBC_ENOMEM : ZBC_ECUDA;
  }
  c->bytes = (int64_t)(sizeof(float2) * std::max<int64_t>(1, off) + sizeof(CacheDesc) * T);
  const size_t sm = sizeof(float2) * r2max;
  for (int t0 = 0; t0 < T; t0 += 65535) {
    const int nt = std::min(65535, T - t0);
    build_w_kernel<<<dim3(h.n3, nt), 256, sm, st>>>(h.d_pool, h.d_desc + t0, c->d_desc + t0, h.n1, h.n2, h.n3, c->data);
    build_u1_kernel<<<dim3(ceil_div((int64_t)nb1 * tile_b1p(h.n1) * rmax, 256), nt), 256, 0, st>>>(h.d_pool, h.d_desc + t0, c->d_desc + t0,
                                                                                h.n1, c->data);
    count_launch(2);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cache_release(c);
    set_error("decompression cache build failed: %s", cudaGetErrorString(e));
    return ZBC_ECUDA;
  }
  h.cache = c;
  h.cache_r = rmax;
  return ZBC_OK;
}

// uexp of each tensor: the smallest e with |Re U1|, |Im U1| < 2^e (0 for a zero factor)
__global__ void __launch_bounds__(256) u1_exp_kernel(const float2* __restrict__ pool,
                                                     const TensorDesc* __restrict__ desc, int n1,
                                                     HalfDesc* __restrict__ hdesc) {
  const int t = blockIdx.x;
  const TensorDesc d = desc[t];
  const float2* U1 = pool + d.off + (int64_t)d.r1 * d.r2 * d.r3;
  float m = 0.f;
  for (int64_t o = threadIdx.x; o < (int64_t)n1 * d.r1; o += blockDim.x)
    m = fmaxf(m, fmaxf(fabsf(U1[o].x), fabsf(U1[o].y)));
  __shared__ float red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int e = 0;
    if (red[0] > 0.f) frexpf(red[0], &e);  // red[0] = f 2^e with f in [0.5, 1): red[0] < 2^e
    hdesc[t].uexp = e;
  }
}

// one thread per (tensor, i1 tile, term, row r < 8 RG, chunk kc < kb1): 8 fp16 values
__global__ void __launch_bounds__(256) build_half_kernel(const float2* __restrict__ cache,
                                                         const CacheDesc* __restrict__ cdesc,
                                                         const HalfDesc* __restrict__ hdesc, int ntens, int n1,
                                                         int kb1max, unsigned char* __restrict__ out) {
  const int B1 = tile_b1(n1), B1p = tile_b1p(n1), nb1 = (n1 + B1 - 1) / B1, RG = (B1 + 7) / 8;
  const int t = blockIdx.y;
  if (t >= ntens) return;
  const CacheDesc cd = cdesc[t];
  const HalfDesc hd = hdesc[t];
  const int per_term = RG * 8 * hd.kb1;  // (row, chunk) items per term
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nb1 * 2 * per_term; o += gridDim.x * blockDim.x) {
    const int t1 = o / (2 * per_term), rem = o % (2 * per_term);
    const int term = rem / per_term, rc = rem % per_term;
    const int r = rc / hd.kb1, kc = rc % hd.kb1;
    const int i1 = t1 * B1 + r;
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float x2[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kk = 8 * kc + 2 * i + h, a = kk >> 1, e = kk & 1;
        float x = 0.f;
        if (a < cd.r1 && r < B1 && i1 < n1) {
          const float2 u = cache[cd.uoff + ((int64_t)t1 * cd.r1p + a) * B1p + r];
          x = ldexpf(e ? u.y : u.x, kHalfShift - hd.uexp);
        }
        const __half hi = __float2half_rn(x);
        x2[h] = term == 0 ? x : x - __half2float(hi);
      }
      const __half2 v = __floats2half2_rn(x2[0], x2[1]);
      w[i] = *reinterpret_cast<const uint32_t*>(&v);
    }
    unsigned char* dst = out + hd.off + (int64_t)t1 * 2 * RG * hd.kb1 * 128 + (int64_t)term * RG * hd.kb1 * 128 +
                         tc::core_off(r, kc, hd.kb1);
    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

int build_half_cache(Handle& h, cudaStream_t st) {
  ZBC_TRY(build_decomp_cache(h, st));
  DecompCache* c = h.cache;
  if (c->half) return ZBC_OK;
  const int T = (int)h.desc.size();
  const int B1 = tile_b1(h.n1), nb1 = (h.n1 + B1 - 1) / B1, RG = (B1 + 7) / 8;
  std::vector<HalfDesc> hd(T);
  int64_t off = 0;
  int kbmax = 2;
  for (int t = 0; t < T; ++t) {
    const int r1p = (h.desc[t].r1 + 1) / 2 * 2;
    hd[t].kb1 = (2 * r1p + 15) / 16 * 2;  // Kp1 = 2 r1p rounded up to 16 reals, 8 reals per chunk
    hd[t].wexp = (int)h.desc[t].scale_log2 + 1;
    hd[t].uexp = 0;
    hd[t].off = off;
    off += (int64_t)nb1 * 2 * RG * hd[t].kb1 * 128;
    kbmax = std::max(kbmax, hd[t].kb1);
  }
  cudaError_t e = cudaMalloc(&c->half, std::max<int64_t>(16, off));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_half, sizeof(HalfDesc) * std::max(1, T));
  if (e == cudaSuccess) {
    c->half_bytes = (int64_t)(std::max<int64_t>(16, off) + sizeof(HalfDesc) * std::max(1, T));
    c->bytes += c->half_bytes;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_half, hd.data(), sizeof(HalfDesc) * T, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    for (int t0 = 0; t0 < T; t0 += 65535) {
      const int nt = std::min(65535, T - t0);
      u1_exp_kernel<<<nt, 256, 0, st>>>(h.d_pool, h.d_desc + t0, h.n1, c->d_half + t0);
      count_launch();
    }
    for (int t0 = 0; t0 < T; t0 += 65535) {
      const int nt = std::min(65535, T - t0);
      build_half_kernel<<<dim3(ceil_div((int64_t)nb1 * 2 * RG * 8 * kbmax, 256), nt), 256, 0, st>>>(
          c->data, c->d_desc + t0, c->d_half + t0, nt, h.n1, kbmax, c->half);
      count_launch();
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    half_release(c);
    set_error("fp16 operand cache build failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? ZBC_ENOMEM : ZBC_ECUDA;
  }
  c->kb1_max = kbmax;
  return ZBC_OK;
}

}  // namespace zbc
