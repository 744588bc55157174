// zbc_tc_selftest: one tcgen05 MMA chain D(128 x N) = A(128 x K) B(N x K)^T through the same
// shared-memory layout, descriptors and TMEM path the product kernels use, so the operand
// encoding can be checked against a host GEMM.  Formats 3 and 4 (f16, bf16) take A from tensor
// memory instead (row i in lane i, two 16-bit K elements per 32-bit column, the lower K index in
// the low half), the form the mode-1 adjoint uses.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tc_common.cuh"
#include "zbc_internal.cuh"

namespace zbc {

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ uint32_t pack16(float lo, float hi, bool bf) {
  if (bf) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
  }
  const __half2 v = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// fmt: 0 f16, 1 bf16, 2 tf32; 3 f16 and 4 bf16 with A in tensor memory
__global__ void __launch_bounds__(128) tc_selftest_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                          float* __restrict__ D, int N, int K, int fmt_in, int* err) {
  const bool a_tmem = fmt_in >= 3;
  const int fmt = a_tmem ? fmt_in - 3 : fmt_in;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tbase;
  const int esz = fmt == 2 ? 4 : 2;
  const int KB = K * esz / 16;                 // 16-byte chunks per row
  unsigned char* sa = sm;                      // 128 rows, padded x2
  unsigned char* sb = sm + 2 * 128 * KB * 16;  // N rows, padded x2
  // fill operands in the canonical layout
  for (int e = threadIdx.x; e < 128 * K; e += blockDim.x) {
    const int r = e / K, k = e % K;
    const uint32_t off = tc::core_off(r, (k * esz) / 16, KB) + (k * esz) % 16;
    const float v = A[r * K + k];
    if (fmt == 2) *(float*)(sa + off) = to_tf32(v);
    else if (fmt == 1) *(__nv_bfloat16*)(sa + off) = __float2bfloat16_rn(v);
    else *(__half*)(sa + off) = __float2half_rn(v);
  }
  for (int e = threadIdx.x; e < N * K; e += blockDim.x) {
    const int r = e / K, k = e % K;
    const uint32_t off = tc::core_off(r, (k * esz) / 16, KB) + (k * esz) % 16;
    const float v = B[r * K + k];
    if (fmt == 2) *(float*)(sb + off) = to_tf32(v);
    else if (fmt == 1) *(__nv_bfloat16*)(sb + off) = __float2bfloat16_rn(v);
    else *(__half*)(sb + off) = __float2half_rn(v);
  }
  // tensor memory: D in columns [0, N), A (formats 3, 4) in columns [64, 64 + K / 2)
  const int ncols = a_tmem ? 128 : (N <= 32 ? 32 : 64);
  if (threadIdx.x < 32) tc::tmem_alloc(&tbase, ncols);
  if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tbase;
  if (a_tmem) {
    // thread = row = lane; warp w reaches lanes 32 w .. 32 w + 31
    const int row = threadIdx.x;
    const uint32_t lanebase = (uint32_t)((threadIdx.x / 32) * 32) << 16;
    for (int c0 = 0; c0 < K / 2; c0 += 16) {
      float v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k = 2 * (c0 + i);
        v[i] = k < K ? __uint_as_float(pack16(A[row * K + k], A[row * K + k + 1], fmt == 1)) : 0.f;
      }
      tc::tmem_st16(tmem + lanebase + 64 + c0, v);
    }
    tc::tmem_wait_st();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }
  if (threadIdx.x == 0) {
    const uint32_t idesc = fmt == 2 ? tc::instr_desc(128, N, 2) : tc::instr_desc(128, N, fmt);
    const int steps = KB / 2;
    for (int s = 0; s < steps; ++s) {
      const uint64_t ad = tc::smem_desc(tc::smem_u32(sa) + s * 256, 128, KB * 128);
      const uint64_t bd = tc::smem_desc(tc::smem_u32(sb) + s * 256, 128, KB * 128);
      if (a_tmem) tc::mma_ts(tmem, tmem + 64 + s * 8, bd, idesc, s > 0);
      else if (fmt == 2) tc::mma<1>(tmem, ad, bd, idesc, s > 0);
      else tc::mma<0>(tmem, ad, bd, idesc, s > 0);
    }
    tc::commit(&mbar);
  }
  const bool ok = tc::mbar_wait(&mbar, 0);
  tc::fence_after();
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else {
    const int w = threadIdx.x / 32;
    const int row = threadIdx.x;
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(w * 32) << 16) + c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (c0 + i < N) D[row * N + c0 + i] = v[i];
    }
  }
  tc::fence_before();
  __syncthreads();
  if (threadIdx.x < 32) tc::tmem_dealloc(tmem, ncols);
}

}  // namespace zbc

using namespace zbc;

extern "C" int zbc_tc_selftest(const float* A_host, const float* B_host, float* D_host, int N, int K, int fmt) {
  clear_error();
  ZBC_CHECK_ARG(A_host && B_host && D_host, "null argument");
  ZBC_CHECK_ARG(fmt >= 0 && fmt <= 4, "fmt must be 0 (f16), 1 (bf16), 2 (tf32), 3 / 4 (f16 / bf16, A in TMEM)");
  ZBC_CHECK_ARG(N >= 16 && N <= 64 && N % 16 == 0, "N must be 16, 32, 48 or 64");
  const int step = fmt == 2 ? 8 : 16;
  ZBC_CHECK_ARG(K >= step && K <= 64 && K % step == 0, "K must be a multiple of the MMA K step (<= 64)");
  float *A, *B, *D;
  int* err;
  ZBC_TRY_CUDA(cudaMalloc(&A, sizeof(float) * 128 * K));
  ZBC_TRY_CUDA(cudaMalloc(&B, sizeof(float) * N * K));
  ZBC_TRY_CUDA(cudaMalloc(&D, sizeof(float) * 128 * N));
  ZBC_TRY_CUDA(cudaMalloc(&err, sizeof(int)));
  ZBC_TRY_CUDA(cudaMemset(err, 0, sizeof(int)));
  ZBC_TRY_CUDA(cudaMemcpy(A, A_host, sizeof(float) * 128 * K, cudaMemcpyHostToDevice));
  ZBC_TRY_CUDA(cudaMemcpy(B, B_host, sizeof(float) * N * K, cudaMemcpyHostToDevice));
  const int esz = fmt == 2 ? 4 : 2;
  (void)esz;
  const size_t smem = 2 * (size_t)(128 + N) * K * esz + 1024;
  ZBC_TRY_CUDA(cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  tc_selftest_kernel<<<1, 128, smem>>>(A, B, D, N, K, fmt, err);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  ZBC_TRY_CUDA(cudaDeviceSynchronize());
  int herr = 0;
  ZBC_TRY_CUDA(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
  ZBC_TRY_CUDA(cudaMemcpy(D_host, D, sizeof(float) * 128 * N, cudaMemcpyDeviceToHost));
  cudaFree(A);
  cudaFree(B);
  cudaFree(D);
  cudaFree(err);
  if (herr) {
    set_error("tcgen05 self-test: MMA completion wait timed out");
    return ZBC_ETIMEOUT;
  }
  return ZBC_OK;
}
