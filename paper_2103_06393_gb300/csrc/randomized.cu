// Randomized Tucker compression entry (learned / fixed widths).
#include "zbc_internal.cuh"

int randomized_compress_entry(const void* cols, int64_t ld, int ncols, const zbc_grid* g, int q, zbc_dtype in_dt,
                              double tol, zbc_tucker_method method, std::vector<int32_t>& ranks, float2** pool,
                              int64_t* elems, zbc_compress_stats* stats, cudaStream_t st) {
  zbc::set_error("randomized Tucker not built yet");
  return ZBC_EINVAL;
}
