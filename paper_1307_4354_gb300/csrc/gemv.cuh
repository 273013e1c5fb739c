// Dense matrix-vector product x (+)= A b for the explicit inverse of the
// coarsest-level matrix (row-major n x n, FP64 or FP32).  HBM-bound: each
// warp streams kGemvRowsPerWarp rows with coalesced loads (independent loads
// in flight per lane), and b passes through shared memory in chunks shared by
// the block's 64 rows, so the staging needs no more than 16 KB whatever n is.
// Accumulation in the matrix type; fixed summation order.
#pragma once
#include <cstdint>

namespace cpm {

constexpr int kGemvWarps = 16;
constexpr int kGemvRowsPerWarp = 4;
constexpr int kGemvRowsPerBlock = kGemvWarps * kGemvRowsPerWarp;
constexpr int kGemvChunk = 2048;

template <typename M, typename T, bool ADD>
__global__ void __launch_bounds__(kGemvWarps * 32) k_dense_gemv(const M* __restrict__ A,
                                                                const T* __restrict__ b,
                                                                T* __restrict__ x, int32_t n) {
  __shared__ M sb[kGemvChunk];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t row0 = blockIdx.x * kGemvRowsPerBlock + warp * kGemvRowsPerWarp;
  const M* a[kGemvRowsPerWarp];
  bool ok[kGemvRowsPerWarp];
  M acc[kGemvRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kGemvRowsPerWarp; ++r) {
    ok[r] = row0 + r < n;
    a[r] = A + (size_t)(ok[r] ? row0 + r : 0) * n;
    acc[r] = M(0);
  }
  for (int32_t c0 = 0; c0 < n; c0 += kGemvChunk) {
    const int32_t cn = min(kGemvChunk, n - c0);
    __syncthreads();
    for (int32_t j = threadIdx.x; j < cn; j += blockDim.x) sb[j] = (M)b[c0 + j];
    __syncthreads();
#pragma unroll 4
    for (int32_t j = lane; j < cn; j += 32) {
      const M bj = sb[j];
#pragma unroll
      for (int r = 0; r < kGemvRowsPerWarp; ++r)
        if (ok[r]) acc[r] += __ldg(a[r] + c0 + j) * bj;
    }
  }
#pragma unroll
  for (int r = 0; r < kGemvRowsPerWarp; ++r) {
    M s = acc[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && ok[r]) x[row0 + r] = ADD ? x[row0 + r] + (T)s : (T)s;
  }
}

inline unsigned dense_gemv_blocks(int32_t n) {
  return (unsigned)((n + kGemvRowsPerBlock - 1) / kGemvRowsPerBlock);
}

}  // namespace cpm
