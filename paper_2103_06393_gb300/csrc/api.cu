// Handle lifetime, host import/export, checkpoints and error reporting of the C ABI.
#include <cstdarg>
#include <cmath>
#include <atomic>
#include <cstring>

#include "zbc_internal.cuh"

namespace zbc {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }

int DevBuf::ensure(size_t need) {
  if (need <= bytes && ptr) return ZBC_OK;
  release();
  size_t b = need < 256 ? 256 : need;
  cudaError_t e = cudaMalloc(&ptr, b);
  if (e != cudaSuccess) {
    ptr = nullptr;
    bytes = 0;
    set_error("cudaMalloc(%zu) failed: %s", b, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? ZBC_ENOMEM : ZBC_ECUDA;
  }
  bytes = b;
  return ZBC_OK;
}
void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

Handle::~Handle() {
  if (d_pool) cudaFree(d_pool);
  if (d_desc) cudaFree(d_desc);
  if (d_v) cudaFree(d_v);
  if (cache) cache_release(cache);
}

int Handle::upload() {
  if (d_desc) cudaFree(d_desc);
  d_desc = nullptr;
  ZBC_TRY_CUDA(cudaMalloc(&d_desc, sizeof(TensorDesc) * desc.size()));
  ZBC_TRY_CUDA(cudaMemcpy(d_desc, desc.data(), sizeof(TensorDesc) * desc.size(), cudaMemcpyHostToDevice));
  return ZBC_OK;
}

static void build_desc(Handle* h) {
  h->desc.resize((size_t)h->M * h->q);
  int64_t off = 0;
  h->max_rank = 0;
  for (size_t t = 0; t < h->desc.size(); ++t) {
    int r1 = h->ranks[3 * t], r2 = h->ranks[3 * t + 1], r3 = h->ranks[3 * t + 2];
    h->desc[t].off = off;
    h->desc[t].r1 = r1;
    h->desc[t].r2 = r2;
    h->desc[t].r3 = r3;
    h->desc[t].scale_log2 = 0.f;
    off += (int64_t)r1 * r2 * r3 + (int64_t)h->n1 * r1 + (int64_t)h->n2 * r2 + (int64_t)h->n3 * r3;
    h->max_rank = std::max(h->max_rank, std::max(r1, std::max(r2, r3)));
  }
  h->pool_elems = off;
}

// ||G||_F per tensor -> floor(log2), computed on the host from the pool (used only for scaling)
__global__ void core_norm_kernel(const float2* pool, TensorDesc* desc, int ntens) {
  int t = blockIdx.x;
  if (t >= ntens) return;
  TensorDesc d = desc[t];
  int n = d.r1 * d.r2 * d.r3;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float2 v = pool[d.off + i];
    s += (double)v.x * v.x + (double)v.y * v.y;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double nrm = sqrt(red[0]);
    desc[t].scale_log2 = nrm > 0 ? (float)floor(log2(nrm)) : 0.f;
  }
}

static int finish_desc(Handle* h) {
  ZBC_TRY(h->upload());
  int nt = (int)h->desc.size();
  if (nt > 0) {
    core_norm_kernel<<<nt, 256>>>(h->d_pool, h->d_desc, nt);
    ZBC_TRY_CUDA(cudaGetLastError());
    ZBC_TRY_CUDA(cudaMemcpy(h->desc.data(), h->d_desc, sizeof(TensorDesc) * nt, cudaMemcpyDeviceToHost));
  }
  return ZBC_OK;
}

int handle_append(Handle* h, const std::vector<int32_t>& ranks, const float2* d_pool_new,
                  int64_t new_elems, int ncols, cudaStream_t st) {
  int64_t old = h->pool_elems;
  float2* np = nullptr;
  ZBC_TRY_CUDA(cudaMalloc(&np, sizeof(float2) * (size_t)std::max<int64_t>(1, old + new_elems)));
  if (old) ZBC_TRY_CUDA(cudaMemcpyAsync(np, h->d_pool, sizeof(float2) * old, cudaMemcpyDeviceToDevice, st));
  ZBC_TRY_CUDA(cudaMemcpyAsync(np + old, d_pool_new, sizeof(float2) * new_elems, cudaMemcpyDeviceToDevice, st));
  ZBC_TRY_CUDA(cudaStreamSynchronize(st));
  if (h->d_pool) cudaFree(h->d_pool);
  h->d_pool = np;
  h->ranks.insert(h->ranks.end(), ranks.begin(), ranks.end());
  h->M += ncols;
  h->m = h->M;
  build_desc(h);
  if (h->pool_elems != old + new_elems) {
    set_error("internal: pool size mismatch");
    return ZBC_EINVAL;
  }
  if (h->cache) {
    cache_release(h->cache);
    h->cache = nullptr;
  }
  return finish_desc(h);
}

static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace zbc

using namespace zbc;

extern "C" const char* zbc_last_error(void) { return g_err.c_str(); }

extern "C" const char* zbc_version(void) { return "zbc 0.1 (sm_103a)"; }

extern "C" int64_t zbc_kernel_launches(void) { return (int64_t)g_launches.load(); }

extern "C" int zbc_free(zbc_handle* h) {
  delete h;
  return ZBC_OK;
}

extern "C" int zbc_get_info(const zbc_handle* hh, zbc_info* info) {
  ZBC_CHECK_ARG(hh && info, "zbc_get_info: null argument");
  const Handle& h = hh->h;
  info->n1 = h.n1;
  info->n2 = h.n2;
  info->n3 = h.n3;
  info->q = h.q;
  info->M = h.M;
  info->m = h.m;
  info->has_v = h.has_v ? 1 : 0;
  info->max_rank = h.max_rank;
  info->pool_bytes = h.pool_elems * 8;
  info->v_bytes = h.has_v ? (int64_t)h.m * h.M * 8 : 0;
  return ZBC_OK;
}

extern "C" int zbc_device_bytes(const zbc_handle* hh, int64_t* pool, int64_t* caches, int64_t* work) {
  clear_error();
  ZBC_CHECK_ARG(hh, "zbc_device_bytes: null handle");
  const Handle& h = hh->h;
  if (pool)
    *pool = (int64_t)(sizeof(float2) * h.pool_elems + sizeof(TensorDesc) * h.desc.size() +
                      (h.has_v ? sizeof(float2) * (size_t)h.m * h.M : 0));
  if (caches) *caches = cache_bytes(h.cache);
  if (work)
    *work = (int64_t)(h.work_partial.bytes + h.work_x.bytes + h.work_misc.bytes + h.work_xt.bytes +
                      h.work_err.bytes + h.work_phi.bytes);
  return ZBC_OK;
}

extern "C" int zbc_memory_bytes(const zbc_handle* hh, int64_t* tucker, int64_t* v, int64_t* full) {
  ZBC_CHECK_ARG(hh && tucker && v && full, "zbc_memory_bytes: null argument");
  const Handle& h = hh->h;
  *tucker = h.pool_elems * 8;
  *v = h.has_v ? (int64_t)h.m * h.M * 8 : 0;
  *full = (int64_t)h.q * h.nv() * h.m * 8;
  return ZBC_OK;
}

static int validate_grid(const zbc_grid* g, int q) {
  ZBC_CHECK_ARG(g, "null grid");
  ZBC_CHECK_ARG(g->n1 >= 2 && g->n2 >= 2 && g->n3 >= 2 && g->n1 <= 4096 && g->n2 <= 4096 && g->n3 <= 4096,
                "grid sizes must be in [2, 4096] (got %d %d %d)", g->n1, g->n2, g->n3);
  ZBC_CHECK_ARG(g->h > 0 && std::isfinite(g->h), "grid spacing must be positive");
  ZBC_CHECK_ARG(q >= 1 && q <= 12, "q must be in [1, 12] (3: piecewise-constant basis, 12: piecewise-linear)");
  return ZBC_OK;
}

extern "C" int zbc_create_from_host(const zbc_grid* g, int q, int M, int m, const int32_t* ranks,
                                    const void* pool_host, int64_t pool_elems, const void* v_host,
                                    zbc_handle** out) {
  clear_error();
  ZBC_TRY(validate_grid(g, q));
  ZBC_CHECK_ARG(out && ranks && pool_host && M > 0 && m > 0, "zbc_create_from_host: bad argument");
  ZBC_CHECK_ARG(v_host || m == M, "without V the number of columns m must equal M");
  auto* hh = new zbc_handle();
  Handle& h = hh->h;
  h.n1 = g->n1;
  h.n2 = g->n2;
  h.n3 = g->n3;
  h.q = q;
  h.M = M;
  h.m = m;
  h.has_v = v_host != nullptr;
  h.ranks.assign(ranks, ranks + 3 * (size_t)M * q);
  int n[3] = {h.n1, h.n2, h.n3};
  for (size_t i = 0; i < h.ranks.size(); ++i) {
    if (h.ranks[i] < 1 || h.ranks[i] > n[i % 3]) {
      delete hh;
      set_error("rank %d of tensor %zu mode %zu out of range", h.ranks[i], i / 3, i % 3);
      return ZBC_EINVAL;
    }
  }
  build_desc(&h);
  if (h.pool_elems != pool_elems) {
    int64_t want = h.pool_elems;
    delete hh;
    set_error("pool has %lld entries, ranks imply %lld", (long long)pool_elems, (long long)want);
    return ZBC_EINVAL;
  }
  int st = ZBC_OK;
  auto fail = [&](int s) { delete hh; return s; };
  if (cudaMalloc(&h.d_pool, sizeof(float2) * pool_elems) != cudaSuccess) {
    set_error("cudaMalloc pool failed");
    return fail(ZBC_ENOMEM);
  }
  if (cudaMemcpy(h.d_pool, pool_host, sizeof(float2) * pool_elems, cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("copy of pool failed");
    return fail(ZBC_ECUDA);
  }
  if (h.has_v) {
    size_t vb = sizeof(float2) * (size_t)m * M;
    if (cudaMalloc(&h.d_v, vb) != cudaSuccess) {
      set_error("cudaMalloc V failed");
      return fail(ZBC_ENOMEM);
    }
    if (cudaMemcpy(h.d_v, v_host, vb, cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("copy of V failed");
      return fail(ZBC_ECUDA);
    }
  }
  st = finish_desc(&h);
  if (st != ZBC_OK) return fail(st);
  *out = hh;
  return ZBC_OK;
}

extern "C" int zbc_export_host(const zbc_handle* hh, int32_t* ranks, void* pool_host, void* v_host) {
  clear_error();
  ZBC_CHECK_ARG(hh, "null handle");
  const Handle& h = hh->h;
  ZBC_TRY_CUDA(cudaDeviceSynchronize());
  if (ranks) memcpy(ranks, h.ranks.data(), sizeof(int32_t) * h.ranks.size());
  if (pool_host) ZBC_TRY_CUDA(cudaMemcpy(pool_host, h.d_pool, sizeof(float2) * h.pool_elems, cudaMemcpyDeviceToHost));
  if (v_host && h.has_v) ZBC_TRY_CUDA(cudaMemcpy(v_host, h.d_v, sizeof(float2) * (size_t)h.m * h.M, cudaMemcpyDeviceToHost));
  return ZBC_OK;
}

namespace {
struct FileHeader {
  char magic[4];
  int32_t version;
  int32_t n1, n2, n3, q, M, m, has_v;
  int64_t pool_elems;
};
}  // namespace

extern "C" int zbc_save(const zbc_handle* hh, const char* path) {
  clear_error();
  ZBC_CHECK_ARG(hh && path, "zbc_save: null argument");
  const Handle& h = hh->h;
  FileHeader fh;
  memcpy(fh.magic, "ZBC1", 4);
  fh.version = 1;
  fh.n1 = h.n1;
  fh.n2 = h.n2;
  fh.n3 = h.n3;
  fh.q = h.q;
  fh.M = h.M;
  fh.m = h.m;
  fh.has_v = h.has_v;
  fh.pool_elems = h.pool_elems;
  std::vector<float2> pool(h.pool_elems), v(h.has_v ? (size_t)h.m * h.M : 0);
  int s = zbc_export_host(hh, nullptr, pool.data(), h.has_v ? v.data() : nullptr);
  if (s != ZBC_OK) return s;
  FILE* f = fopen(path, "wb");
  if (!f) {
    set_error("cannot open %s for writing", path);
    return ZBC_EIO;
  }
  bool ok = fwrite(&fh, sizeof(fh), 1, f) == 1 &&
            fwrite(h.ranks.data(), sizeof(int32_t), h.ranks.size(), f) == h.ranks.size() &&
            fwrite(pool.data(), sizeof(float2), pool.size(), f) == pool.size() &&
            (v.empty() || fwrite(v.data(), sizeof(float2), v.size(), f) == v.size());
  ok = (fclose(f) == 0) && ok;
  if (!ok) {
    set_error("write to %s failed", path);
    return ZBC_EIO;
  }
  return ZBC_OK;
}

extern "C" int zbc_load(const char* path, zbc_handle** out) {
  clear_error();
  ZBC_CHECK_ARG(path && out, "zbc_load: null argument");
  FILE* f = fopen(path, "rb");
  if (!f) {
    set_error("cannot open %s", path);
    return ZBC_EIO;
  }
  FileHeader fh;
  if (fread(&fh, sizeof(fh), 1, f) != 1 || memcmp(fh.magic, "ZBC1", 4) != 0 || fh.version != 1 ||
      fh.M <= 0 || fh.q <= 0 || fh.m <= 0 || fh.pool_elems <= 0) {
    fclose(f);
    set_error("%s is not a zbc handle file", path);
    return ZBC_EIO;
  }
  std::vector<int32_t> ranks(3 * (size_t)fh.M * fh.q);
  std::vector<float2> pool(fh.pool_elems), v(fh.has_v ? (size_t)fh.m * fh.M : 0);
  bool ok = fread(ranks.data(), sizeof(int32_t), ranks.size(), f) == ranks.size() &&
            fread(pool.data(), sizeof(float2), pool.size(), f) == pool.size() &&
            (v.empty() || fread(v.data(), sizeof(float2), v.size(), f) == v.size());
  fclose(f);
  if (!ok) {
    set_error("%s is truncated", path);
    return ZBC_EIO;
  }
  zbc_grid g{fh.n1, fh.n2, fh.n3, 1.0, 0.0, 0.0};
  return zbc_create_from_host(&g, fh.q, fh.M, fh.m, ranks.data(), pool.data(), fh.pool_elems,
                              fh.has_v ? v.data() : nullptr, out);
}
