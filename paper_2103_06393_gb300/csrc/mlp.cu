// Rank-predictor MLP: forward, backward and Adam on the GPU (no counterpart in the paper,
// whose ranks come from HOSVD only, Sec. IV.A).
//
// 7 -> 64 -> 64 -> 64 -> 9, ReLU after the hidden layers, linear output; loss = mean over
// batch and outputs of (out - target)^2 (target = log of the 9 Tucker ranks: 3 components x
// 3 modes).  Weights are kept as FP32 master copies; forward and backward use the weights
// rounded to BF16, with FP32 arithmetic and accumulation.  Parameters are packed as
//   W1 (64x7, row-major [out][in]), b1, W2 (64x64), b2, W3 (64x64), b3, W4 (9x64), b4.
// Weight gradients are reduced over the batch in a fixed order (per-CTA partials, then a
// column sum), so a backward pass is deterministic.
#include <cuda_bf16.h>

#include <cmath>

#include "zbc_internal.cuh"

namespace zbc {

constexpr int kIn = 7, kH = 64, kOut = 9;
constexpr int kL1 = kH * kIn + kH, kL2 = kH * kH + kH, kL3 = kH * kH + kH, kL4 = kOut * kH + kOut;
constexpr int kNP = kL1 + kL2 + kL3 + kL4;  // 9417
constexpr int kSB = 32;                     // samples per CTA
constexpr int kMT = 128;                    // threads per CTA

struct Mlp {
  float* master = nullptr;  // kNP FP32
  float* wbf = nullptr;     // kNP, the BF16-rounded weights as FP32 (what forward/backward use)
  float* m = nullptr;       // Adam first moment
  float* v = nullptr;       // Adam second moment
  float* partial = nullptr; // per-CTA gradient partials
  int partial_ctas = 0;
  int t = 0;                // Adam step count
};

struct LayerOff {
  int W, b, in, out;
};
__host__ __device__ constexpr LayerOff layer(int l) {
  return l == 0 ? LayerOff{0, kH * kIn, kIn, kH}
         : l == 1 ? LayerOff{kL1, kL1 + kH * kH, kH, kH}
         : l == 2 ? LayerOff{kL1 + kL2, kL1 + kL2 + kH * kH, kH, kH}
                  : LayerOff{kL1 + kL2 + kL3, kL1 + kL2 + kL3 + kOut * kH, kH, kOut};
}

__global__ void round_bf16_kernel(const float* __restrict__ src, float* __restrict__ dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __bfloat162float(__float2bfloat16_rn(src[i]));
}

// Forward (and optionally backward) for kSB samples per CTA.  acts[l][s][*]: input of layer l
// (acts[0] = x), pre[l][s][*]: pre-activation of layer l.
template <bool BACKWARD>
__global__ void __launch_bounds__(kMT) mlp_kernel(const float* __restrict__ w, const float* __restrict__ X,
                                                  const float* __restrict__ T, int B, float* __restrict__ out,
                                                  float* __restrict__ partial, float* __restrict__ loss_part) {
  extern __shared__ float sm[];
  float* ws = sm;                       // kNP
  float* act = ws + kNP;                // 4 x kSB x 64  (inputs of layers 0..3)
  float* pre = act + 4 * kSB * kH;      // 4 x kSB x 64  (pre-activations of layers 0..3)
  float* gbuf = pre + 4 * kSB * kH;     // 2 x kSB x 64  (back-propagated gradients)
  const int s0 = blockIdx.x * kSB;
  const int ns = min(kSB, B - s0);
  for (int i = threadIdx.x; i < kNP; i += kMT) ws[i] = w[i];
  for (int i = threadIdx.x; i < kSB * kH; i += kMT) {
    const int s = i / kH, c = i % kH;
    act[s * kH + c] = (s < ns && c < kIn) ? X[(int64_t)(s0 + s) * kIn + c] : 0.f;
  }
  __syncthreads();
  for (int l = 0; l < 4; ++l) {
    const LayerOff L = layer(l);
    float* a_in = act + l * kSB * kH;
    float* z = pre + l * kSB * kH;
    for (int i = threadIdx.x; i < kSB * L.out; i += kMT) {
      const int s = i / L.out, o = i % L.out;
      float acc = ws[L.b + o];
      for (int k = 0; k < L.in; ++k) acc = fmaf(ws[L.W + o * L.in + k], a_in[s * kH + k], acc);
      z[s * kH + o] = acc;
      if (l < 3) act[(l + 1) * kSB * kH + s * kH + o] = fmaxf(acc, 0.f);
    }
    __syncthreads();
  }
  float* zo = pre + 3 * kSB * kH;
  if (!BACKWARD) {
    for (int i = threadIdx.x; i < ns * kOut; i += kMT) {
      const int s = i / kOut, o = i % kOut;
      out[(int64_t)(s0 + s) * kOut + o] = zo[s * kH + o];
    }
    return;
  }
  // d loss / d out = 2 (out - t) / (B * kOut); loss partial
  float* g = gbuf;
  float lsum = 0.f;
  for (int i = threadIdx.x; i < kSB * kH; i += kMT) {
    const int s = i / kH, o = i % kH;
    float gv = 0.f;
    if (s < ns && o < kOut) {
      const float d = zo[s * kH + o] - T[(int64_t)(s0 + s) * kOut + o];
      lsum += d * d;
      gv = 2.f * d / ((float)B * kOut);
    }
    g[s * kH + o] = gv;
  }
  // loss: per-CTA sum (fixed order over threads via shared reduction)
  __shared__ float lred[kMT];
  lred[threadIdx.x] = lsum;
  __syncthreads();
  for (int st = kMT / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) lred[threadIdx.x] += lred[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = lred[0];
  float* pout = partial + (int64_t)blockIdx.x * kNP;
  for (int l = 3; l >= 0; --l) {
    const LayerOff L = layer(l);
    const float* a_in = act + l * kSB * kH;
    // weight and bias gradients: sum over this CTA's samples
    for (int i = threadIdx.x; i < L.out * L.in; i += kMT) {
      const int o = i / L.in, k = i % L.in;
      float acc = 0.f;
      for (int s = 0; s < kSB; ++s) acc = fmaf(g[s * kH + o], a_in[s * kH + k], acc);
      pout[L.W + i] = acc;
    }
    for (int o = threadIdx.x; o < L.out; o += kMT) {
      float acc = 0.f;
      for (int s = 0; s < kSB; ++s) acc += g[s * kH + o];
      pout[L.b + o] = acc;
    }
    if (l == 0) break;
    // gradient w.r.t. the layer input, through the ReLU of the previous layer
    float* gn = (g == gbuf) ? gbuf + kSB * kH : gbuf;
    const float* zprev = pre + (l - 1) * kSB * kH;
    for (int i = threadIdx.x; i < kSB * kH; i += kMT) {
      const int s = i / kH, k = i % kH;
      float acc = 0.f;
      for (int o = 0; o < L.out; ++o) acc = fmaf(ws[L.W + o * L.in + k], g[s * kH + o], acc);
      gn[s * kH + k] = zprev[s * kH + k] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    g = gn;
  }
}

// grads[i] = sum_c partial[c][i] in CTA order; loss = sum_c loss_part[c] / (B * kOut)
__global__ void reduce_grads_kernel(const float* __restrict__ partial, int nc, float* __restrict__ grads,
                                    const float* __restrict__ loss_part, float* __restrict__ loss, int B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kNP) {
    float acc = 0.f;
    for (int c = 0; c < nc; ++c) acc += partial[(int64_t)c * kNP + i];
    grads[i] = acc;
  }
  if (i == 0 && loss) {
    float l = 0.f;
    for (int c = 0; c < nc; ++c) l += loss_part[c];
    *loss = l / ((float)B * kOut);
  }
}

__global__ void adam_kernel(float* __restrict__ master, float* __restrict__ wbf, float* __restrict__ m,
                            float* __restrict__ v, const float* __restrict__ g, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNP) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float mi = b1 * m[i] + (1.f - b1) * g[i];
  const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  m[i] = mi;
  v[i] = vi;
  const float w = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  master[i] = w;
  wbf[i] = __bfloat162float(__float2bfloat16_rn(w));
}

static size_t mlp_smem() { return sizeof(float) * ((size_t)kNP + 10 * kSB * kH); }

static int ensure_partial(Mlp* M, int nc) {
  if (M->partial_ctas >= nc) return ZBC_OK;
  if (M->partial) cudaFree(M->partial);
  M->partial = nullptr;
  ZBC_TRY_CUDA(cudaMalloc(&M->partial, sizeof(float) * ((size_t)nc * kNP + nc)));
  M->partial_ctas = nc;
  return ZBC_OK;
}

int mlp_forward_dev(const Mlp* M, const float* X, int B, float* out, cudaStream_t st) {
  const int nc = ceil_div(B, kSB);
  static bool attr = false;
  if (!attr) {
    ZBC_TRY_CUDA(cudaFuncSetAttribute(mlp_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem()));
    ZBC_TRY_CUDA(cudaFuncSetAttribute(mlp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem()));
    attr = true;
  }
  mlp_kernel<false><<<nc, kMT, mlp_smem(), st>>>(M->wbf, X, nullptr, B, out, nullptr, nullptr);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

static int mlp_backward_dev(Mlp* M, const float* X, const float* T, int B, float* grads, float* loss, cudaStream_t st) {
  const int nc = ceil_div(B, kSB);
  ZBC_TRY(ensure_partial(M, nc));
  static bool attr = false;
  if (!attr) {
    ZBC_TRY_CUDA(cudaFuncSetAttribute(mlp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem()));
    attr = true;
  }
  float* loss_part = M->partial + (size_t)nc * kNP;
  mlp_kernel<true><<<nc, kMT, mlp_smem(), st>>>(M->wbf, X, T, B, nullptr, M->partial, loss_part);
  reduce_grads_kernel<<<ceil_div(kNP, 256), 256, 0, st>>>(M->partial, nc, grads, loss_part, loss, B);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch(2);
  return ZBC_OK;
}

}  // namespace zbc

using namespace zbc;

struct zbc_mlp {
  Mlp m;
  float* grads = nullptr;
};

namespace zbc {
const Mlp* mlp_of(const zbc_mlp* z) { return &z->m; }
}  // namespace zbc

extern "C" int zbc_mlp_num_params(void) { return kNP; }

extern "C" int zbc_mlp_create(const float* params_host, int n_params, zbc_mlp** out) {
  clear_error();
  ZBC_CHECK_ARG(params_host && out, "zbc_mlp_create: null argument");
  ZBC_CHECK_ARG(n_params == kNP, "expected %d parameters, got %d", kNP, n_params);
  auto* z = new zbc_mlp();
  Mlp& M = z->m;
  auto fail = [&](cudaError_t e) {
    set_error("zbc_mlp_create: %s", cudaGetErrorString(e));
    if (M.master) cudaFree(M.master);
    if (M.wbf) cudaFree(M.wbf);
    if (M.m) cudaFree(M.m);
    if (M.v) cudaFree(M.v);
    if (z->grads) cudaFree(z->grads);
    delete z;
    return ZBC_ENOMEM;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&M.master, sizeof(float) * kNP)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&M.wbf, sizeof(float) * kNP)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&M.m, sizeof(float) * kNP)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&M.v, sizeof(float) * kNP)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&z->grads, sizeof(float) * kNP)) != cudaSuccess) return fail(e);
  cudaMemcpy(M.master, params_host, sizeof(float) * kNP, cudaMemcpyHostToDevice);
  cudaMemset(M.m, 0, sizeof(float) * kNP);
  cudaMemset(M.v, 0, sizeof(float) * kNP);
  round_bf16_kernel<<<ceil_div(kNP, 256), 256>>>(M.master, M.wbf, kNP);
  count_launch();
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e);
  *out = z;
  return ZBC_OK;
}

extern "C" int zbc_mlp_free(zbc_mlp* z) {
  if (!z) return ZBC_OK;
  cudaFree(z->m.master);
  cudaFree(z->m.wbf);
  cudaFree(z->m.m);
  cudaFree(z->m.v);
  if (z->m.partial) cudaFree(z->m.partial);
  cudaFree(z->grads);
  delete z;
  return ZBC_OK;
}

extern "C" int zbc_mlp_get_params(const zbc_mlp* z, float* master_host, float* bf16_host) {
  clear_error();
  ZBC_CHECK_ARG(z, "null model");
  ZBC_TRY_CUDA(cudaDeviceSynchronize());
  if (master_host) ZBC_TRY_CUDA(cudaMemcpy(master_host, z->m.master, sizeof(float) * kNP, cudaMemcpyDeviceToHost));
  if (bf16_host) ZBC_TRY_CUDA(cudaMemcpy(bf16_host, z->m.wbf, sizeof(float) * kNP, cudaMemcpyDeviceToHost));
  return ZBC_OK;
}

extern "C" int zbc_mlp_forward(const zbc_mlp* z, const float* X, int B, float* out, zbc_stream st) {
  clear_error();
  ZBC_CHECK_ARG(z && X && out && B >= 1, "zbc_mlp_forward: bad argument");
  return mlp_forward_dev(&z->m, X, B, out, st);
}

extern "C" int zbc_mlp_backward(zbc_mlp* z, const float* X, const float* T, int B, float* grads, float* loss,
                                zbc_stream st) {
  clear_error();
  ZBC_CHECK_ARG(z && X && T && grads && B >= 1, "zbc_mlp_backward: bad argument");
  return mlp_backward_dev(&z->m, X, T, B, grads, loss, st);
}

extern "C" int zbc_mlp_adam_step(zbc_mlp* z, const float* grads, float lr, zbc_stream st) {
  clear_error();
  ZBC_CHECK_ARG(z && grads && lr > 0, "zbc_mlp_adam_step: bad argument");
  z->m.t += 1;
  const float c1 = 1.f - powf(0.9f, (float)z->m.t), c2 = 1.f - powf(0.999f, (float)z->m.t);
  adam_kernel<<<ceil_div(kNP, 256), 256, 0, st>>>(z->m.master, z->m.wbf, z->m.m, z->m.v, grads, lr, c1, c2);
  ZBC_TRY_CUDA(cudaGetLastError());
  count_launch();
  return ZBC_OK;
}

extern "C" int zbc_mlp_train(zbc_mlp* z, const float* X, const float* T, int B, int steps, float lr,
                             float* loss_hist, zbc_stream st) {
  clear_error();
  ZBC_CHECK_ARG(z && X && T && B >= 1 && steps >= 1 && lr > 0, "zbc_mlp_train: bad argument");
  for (int i = 0; i < steps; ++i) {
    ZBC_TRY(mlp_backward_dev(&z->m, X, T, B, z->grads, loss_hist ? loss_hist + i : nullptr, st));
    ZBC_TRY(zbc_mlp_adam_step(z, z->grads, lr, st));
  }
  return ZBC_OK;
}
