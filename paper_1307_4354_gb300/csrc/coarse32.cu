// Coarsest-level solve for levels too large for the FP64 Gauss-Jordan inverse
// (tori and thin ellipsoids stop coarsening at a few 10^4 points, Sec. 4.3's
// bands must stay inside the reach).  At setup the dense matrix
// A_c = diag(c) - M_c is assembled in FP32 and inverted once with a library LU
// (cuSOLVER getrf / getrs on the identity; setup only).  Each V-cycle then
// applies the explicit inverse with the GEMV below; FP64 V-cycles add two
// steps of iterative refinement with the FP64 residual (hier.cu).
#include <cusolverDn.h>


#include "ops.cuh"
#include "gemv.cuh"

namespace cpm {

static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

#define CPM_SOLVER_TRY(expr)                                                              \
  do {                                                                                    \
    cusolverStatus_t s_ = (expr);                                                         \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                                    \
      throw ::cpm::Error{CPM_ERR_CUDA, std::string(#expr) + ": cusolver status " +        \
                                           std::to_string((int)s_)};                      \
  } while (0)

__global__ void k_identity(float* X, int64_t n) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n * n) X[q] = (q / n == q % n) ? 1.f : 0.f;
}

__global__ void k_check_info(const int* info, int32_t* err) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && info[0] != 0) atomicOr(err, 1);
}

// A: row-major n x n FP32 (overwritten by its LU); X: receives A^-1 (row-major).
// Row-major A read as column-major is A^T; solving A^T Y = I column-major
// gives Y = A^-T, whose column-major storage is A^-1 row-major.
void invert_dense_f32(float* A, float* X, int32_t n, cudaStream_t st, int32_t* err) {
  cusolverDnHandle_t h = nullptr;
  CPM_SOLVER_TRY(cusolverDnCreate(&h));
  struct Guard {
    cusolverDnHandle_t h;
    ~Guard() { cusolverDnDestroy(h); }
  } guard{h};
  CPM_SOLVER_TRY(cusolverDnSetStream(h, st));
  int lwork = 0;
  CPM_SOLVER_TRY(cusolverDnSgetrf_bufferSize(h, n, n, A, n, &lwork));
  DBuf<float> work(lwork > 0 ? lwork : 1);
  DBuf<int> ipiv(n), info(1);
  CPM_SOLVER_TRY(cusolverDnSgetrf(h, n, n, A, n, work.get(), ipiv.get(), info.get()));
  k_check_info<<<1, 32, 0, st>>>(info.get(), err);
  k_identity<<<nblk((int64_t)n * n, 256), 256, 0, st>>>(X, n);
  CPM_SOLVER_TRY(cusolverDnSgetrs(h, CUBLAS_OP_N, n, n, A, n, ipiv.get(), X, n, info.get()));
  k_check_info<<<1, 32, 0, st>>>(info.get(), err);
  CPM_CUDA_TRY(cudaGetLastError());
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
}

// x_g (+)= Ainv b_g with the FP32 inverse (chunked dense product, FP32 accumulation).
template <typename T>
void launch_coarse_gemv32(const float* Ainv, const T* const* b, T* const* x, int G, int32_t n, bool add,
                          cudaStream_t st) {
  if (add) {
    if constexpr (sizeof(T) == 8) launch_dense_gemv<float, T, true>(Ainv, b, x, G, n, st);
  } else {
    launch_dense_gemv<float, T, false>(Ainv, b, x, G, n, st);
  }
  count_launch((G + kGemvMaxVectors - 1) / kGemvMaxVectors);
}

template void launch_coarse_gemv32<double>(const float*, const double* const*, double* const*, int,
                                           int32_t, bool, cudaStream_t);
template void launch_coarse_gemv32<float>(const float*, const float* const*, float* const*, int, int32_t,
                                          bool, cudaStream_t);

}  // namespace cpm
