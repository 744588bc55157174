// Operands of the mode-1 forms of the products (products_mode1.cu: the adjoint,
// products_mode1_fwd.cu: the forward), kept per handle beside the decompression cache.
//
// Rows are the (column j, rank a) pairs of one component k, j-major, a inner; component k's
// rows start at group gbase[k] (128 rows to a group, the last group of a component zero padded).
#pragma once

#include <cuda_fp16.h>

#include <vector>

#include "stage.cuh"

namespace zbc {

constexpr int kM1Rows = 128;       // (column, rank) rows per group = MMA M = TMEM lanes
constexpr int kM1MaxP = 16;        // right-hand sides per pass
constexpr int kM1MaxStages = 8;
constexpr int kM1MaxN1p = 224;     // widest A of the adjoint without i1 tiles (2 x 224 TMEM columns + D)

struct Mode1Row {
  int64_t wbase;  // W_{kj}[i23 = 0, a] in the decompression cache; -1 for a padding row
  int r1p;        // W's stride per i23
  int uexp;       // max |Re|, |Im| of U1_{kj}[:, a] < 2^uexp (set by the build kernel)
};

struct Mode1Cache {
  int KG = 0;                 // groups over all components
  int n1p = 0;                // n1 rounded up to 8 (K = 2 n1p reals)
  std::vector<int> gbase;     // host: first group of each component (q + 1 entries)
  uint32_t* A = nullptr;      // [KG][2 terms][n1p / 4][128 rows][4] fp16x2 (Re low, Im high)
  Mode1Row* rows = nullptr;   // [KG * 128]
  int* kg_k = nullptr;        // [KG] component of each group
  int2* colrows = nullptr;    // [M q], tensor t = j q + k -> (first global row, r1)
  int4* rowsrc = nullptr;     // [KG * 128] (tensor, a, valid) for the build
  // forward operands, built on the first forward call (products_mode1_fwd.cu); rows in chunks
  // of 32 (a component's rows start a new chunk)
  bool fwd = false;
  int n23p = 0;               // n2 n3 rounded up to 16
  std::vector<int> chbase;    // host: first chunk of each component (q + 1 entries)
  int* d_chbase = nullptr;    // the same on the device
  uint32_t* Bf = nullptr;     // [chunk][2 terms][2 n1p rows][32 words]: U1, 128-byte swizzled
  float2* Wc = nullptr;       // [chunk][n23p][32]: W scaled per (i23, row)
  int* ew = nullptr;          // [q][n23p]: exponents of the W scaling
  int2* chunkinfo = nullptr;  // [chunk] (first column, number of columns)
  int8_t* jtab = nullptr;     // [chunk][32] column of each row minus the chunk's first column
  int64_t bytes = 0;          // device bytes held by the operands above
  int64_t fwd_bytes = 0;      // the part of bytes held by the forward operands
};

int build_mode1_cache(Handle& h, cudaStream_t st);

// 16 columns of this thread's TMEM lane, without waiting (tmem_wait_ld completes all of them)
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace zbc
