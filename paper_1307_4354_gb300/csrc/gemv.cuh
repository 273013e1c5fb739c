// Dense matrix-vector products x (+)= A b for the explicit inverse of the
// coarsest-level matrix (row-major n x n, FP64 or FP32), for one or several
// right-hand sides at once.  HBM-bound on A: each warp streams
// kGemvRowsPerWarp rows with coalesced loads (independent loads in flight per
// lane; 16 rows per block, so that even a 4096-point level fills every SM),
// and the vectors pass through shared memory in chunks shared by the block's
// rows (32 KB at most, whatever n is).  Accumulation in the matrix
// type; fixed summation order.
#pragma once
#include <cstdint>

namespace cpm {

constexpr int kGemvWarps = 8;
constexpr int kGemvRowsPerWarp = 2;
constexpr int kGemvRowsPerBlock = kGemvWarps * kGemvRowsPerWarp;
constexpr int kGemvMaxVectors = 4;

// Up to kGemvMaxVectors right-hand sides that share the matrix: each matrix
// element is read once and multiplied into every vector.
template <typename T>
struct GemvVectors {
  const T* b[kGemvMaxVectors];
  T* x[kGemvMaxVectors];
};

// Each lane accumulates the columns j = lane (mod 32) in increasing order, so
// the result of one vector does not depend on NV or on the chunk size (a
// multiple of 32).
template <typename M, typename T, bool ADD, int NV>
__global__ void __launch_bounds__(kGemvWarps * 32) k_dense_gemv(const M* __restrict__ A,
                                                                GemvVectors<T> v, int32_t n) {
  constexpr int kChunk = (4096 / NV) / 32 * 32;  // a multiple of 32
  __shared__ M sb[NV][kChunk];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t row0 = blockIdx.x * kGemvRowsPerBlock + warp * kGemvRowsPerWarp;
  const M* a[kGemvRowsPerWarp];
  bool ok[kGemvRowsPerWarp];
  M acc[kGemvRowsPerWarp][NV];
#pragma unroll
  for (int r = 0; r < kGemvRowsPerWarp; ++r) {
    ok[r] = row0 + r < n;
    a[r] = A + (size_t)(ok[r] ? row0 + r : 0) * n;
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[r][q] = M(0);
  }
  for (int32_t c0 = 0; c0 < n; c0 += kChunk) {
    const int32_t cn = min(kChunk, n - c0);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q)
      for (int32_t j = threadIdx.x; j < cn; j += blockDim.x) sb[q][j] = (M)v.b[q][c0 + j];
    __syncthreads();
#pragma unroll 2
    for (int32_t j = lane; j < cn; j += 32) {
      M bj[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) bj[q] = sb[q][j];
#pragma unroll
      for (int r = 0; r < kGemvRowsPerWarp; ++r) {
        if (!ok[r]) continue;
        const M av = __ldg(a[r] + c0 + j);
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[r][q] += av * bj[q];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kGemvRowsPerWarp; ++r) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      M s = acc[r][q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0 && ok[r]) v.x[q][row0 + r] = ADD ? v.x[q][row0 + r] + (T)s : (T)s;
    }
  }
}

// The same product for an FP32 matrix whose rows start on 16-byte boundaries
// (leading dimension ld, a multiple of 4; columns n .. ld-1 are zero): each
// lane streams groups of four columns with 16-byte loads, four groups per row
// in flight.  FP32 accumulation.
template <typename T, bool ADD, int NV>
__global__ void __launch_bounds__(kGemvWarps * 32) k_dense_gemv_v4(const float* __restrict__ A, int32_t ld,
                                                                   GemvVectors<T> v, int32_t n) {
  constexpr int kChunk = (4096 / NV) / 128 * 128;  // a multiple of 128 columns
  __shared__ __align__(16) float sb[NV][kChunk];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t row0 = blockIdx.x * kGemvRowsPerBlock + warp * kGemvRowsPerWarp;
  const float* a[kGemvRowsPerWarp];
  bool ok[kGemvRowsPerWarp];
  float acc[kGemvRowsPerWarp][NV];
#pragma unroll
  for (int r = 0; r < kGemvRowsPerWarp; ++r) {
    ok[r] = row0 + r < n;
    a[r] = A + (size_t)(ok[r] ? row0 + r : 0) * ld;
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[r][q] = 0.f;
  }
  for (int32_t c0 = 0; c0 < ld; c0 += kChunk) {
    const int32_t cn = min(kChunk, ld - c0);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q)
      for (int32_t j = threadIdx.x; j < cn; j += blockDim.x)
        sb[q][j] = c0 + j < n ? (float)v.b[q][c0 + j] : 0.f;
    __syncthreads();
#pragma unroll 4
    for (int32_t j = 4 * lane; j < cn; j += 128) {
      float4 bj[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) bj[q] = *reinterpret_cast<const float4*>(&sb[q][j]);
#pragma unroll
      for (int r = 0; r < kGemvRowsPerWarp; ++r) {
        if (!ok[r]) continue;
        const float4 av = __ldg(reinterpret_cast<const float4*>(a[r] + c0 + j));
#pragma unroll
        for (int q = 0; q < NV; ++q)
          acc[r][q] += av.x * bj[q].x + av.y * bj[q].y + av.z * bj[q].z + av.w * bj[q].w;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kGemvRowsPerWarp; ++r) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      float s = acc[r][q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0 && ok[r]) v.x[q][row0 + r] = ADD ? v.x[q][row0 + r] + (T)s : (T)s;
    }
  }
}

inline unsigned dense_gemv_blocks(int32_t n) {
  return (unsigned)((n + kGemvRowsPerBlock - 1) / kGemvRowsPerBlock);
}

// x_g (+)= A b_g for g < G, in launches of up to kGemvMaxVectors vectors.
template <typename M, typename T, bool ADD>
void launch_dense_gemv(const M* A, const T* const* b, T* const* x, int G, int32_t n,
                       cudaStream_t st) {
  for (int g0 = 0; g0 < G; g0 += kGemvMaxVectors) {
    const int nv = G - g0 < kGemvMaxVectors ? G - g0 : kGemvMaxVectors;
    GemvVectors<T> v{};
    for (int q = 0; q < nv; ++q) {
      v.b[q] = b[g0 + q];
      v.x[q] = x[g0 + q];
    }
    const unsigned grid = dense_gemv_blocks(n);
    switch (nv) {
      case 1: k_dense_gemv<M, T, ADD, 1><<<grid, kGemvWarps * 32, 0, st>>>(A, v, n); break;
      case 2: k_dense_gemv<M, T, ADD, 2><<<grid, kGemvWarps * 32, 0, st>>>(A, v, n); break;
      case 3: k_dense_gemv<M, T, ADD, 3><<<grid, kGemvWarps * 32, 0, st>>>(A, v, n); break;
      default: k_dense_gemv<M, T, ADD, 4><<<grid, kGemvWarps * 32, 0, st>>>(A, v, n); break;
    }
  }
}

// x_g = A b_g for g < G with the row-aligned FP32 matrix of k_dense_gemv_v4.
template <typename T>
void launch_dense_gemv_v4(const float* A, int32_t ld, const T* const* b, T* const* x, int G, int32_t n,
                          cudaStream_t st) {
  for (int g0 = 0; g0 < G; g0 += kGemvMaxVectors) {
    const int nv = G - g0 < kGemvMaxVectors ? G - g0 : kGemvMaxVectors;
    GemvVectors<T> v{};
    for (int q = 0; q < nv; ++q) {
      v.b[q] = b[g0 + q];
      v.x[q] = x[g0 + q];
    }
    const unsigned grid = dense_gemv_blocks(n);
    switch (nv) {
      case 1: k_dense_gemv_v4<T, false, 1><<<grid, kGemvWarps * 32, 0, st>>>(A, ld, v, n); break;
      case 2: k_dense_gemv_v4<T, false, 2><<<grid, kGemvWarps * 32, 0, st>>>(A, ld, v, n); break;
      case 3: k_dense_gemv_v4<T, false, 3><<<grid, kGemvWarps * 32, 0, st>>>(A, ld, v, n); break;
      default: k_dense_gemv_v4<T, false, 4><<<grid, kGemvWarps * 32, 0, st>>>(A, ld, v, n); break;
    }
  }
}

}  // namespace cpm
