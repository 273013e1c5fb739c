// Allocation-free residual norms of the finest level (cpm_residual_norms_noalloc).
//
// Some callers cannot allocate device memory at the moment they need the
// residual: loops with hard latency budgets that forbid allocator calls, and
// host frameworks that hand out every byte of device memory from their own
// pool.  This entry point therefore allocates
// nothing and leaves the hierarchy's own work buffers alone: its scratch (the
// extension E u on B+ and the per-block partial norms) is one file-scope
// device array of fixed size, resident on every GPU that loads the library
// until the process exits.  The paper has no counterpart; it is plumbing
// around the residual r = f - A u of the discrete system.
#include <cuda.h>

#include <mutex>

#include "ops.cuh"

#define CPM_NOALLOC_MAX_POINTS_VALUE (1 << 20)
#define CPM_NOALLOC_MAX_BLOCKS ((CPM_NOALLOC_MAX_POINTS_VALUE + 255) / 256)

namespace cpm {

// Scratch: [0, MAX_POINTS) holds w = E u on B+, then 2 doubles per block of
// the residual kernel hold its partial max|r| and sum r^2.
static __device__ __align__(256) double g_noalloc_scratch[CPM_NOALLOC_MAX_POINTS_VALUE +
                                                          2 * CPM_NOALLOC_MAX_BLOCKS];

// Residual r_i = f_i - c_i u_i + (M u)_i in the difference form, reduced per
// block (the residual itself is not stored).
__global__ void __launch_bounds__(256) k_resid_partials_noalloc(LevelView<double> L,
                                                                const double* __restrict__ u,
                                                                const double* __restrict__ w,
                                                                const double* __restrict__ f,
                                                                const double* __restrict__ cvec,
                                                                double cval, double* part) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0, s = 0.0;
  if (i < L.nB) {
    const double wi = w[i];
    double lap = 0.0;
    for (int q = 0; q < 2 * L.dim; ++q) lap += w[__ldg(L.nbr + (int64_t)q * L.nB + i)] - wi;
    const double ui = u[i];
    const double Mu = lap * L.inv_h2 + L.gamma * (wi - ui);
    const double r = f[i] - (cvec ? cvec[i] : cval) * ui + Mu;
    m = fabs(r);
    s = r * r;
  }
  __shared__ double sm[8], ss[8];
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sm[wid] = m; ss[wid] = s; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double M = 0.0, S = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { M = fmax(M, sm[q]); S += ss[q]; }
    part[2 * blockIdx.x] = M;
    part[2 * blockIdx.x + 1] = S;
  }
}

// norms[0] = max|r|, norms[1] = sum r^2 (fixed reduction order).
__global__ void k_final_noalloc(const double* part, int nblocks, double* norms) {
  double m = 0.0, s = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    m = fmax(m, part[2 * i]);
    s += part[2 * i + 1];
  }
  __shared__ double sm[32], ss[32];
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sm[wid] = m; ss[wid] = s; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double M = 0.0, S = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { M = fmax(M, sm[q]); S += ss[q]; }
    norms[0] = M;
    norms[1] = S;
  }
}

// Device address of the scratch array for the calling thread's current
// context (host code cannot pass the symbol itself to a kernel: in host code
// it names a host-side stand-in, not device memory).  The address is looked up
// with cudaGetSymbolAddress on the first call in a context and cached with the
// context's unique id (cuCtxGetId), so a context torn down and created again
// (cudaDeviceReset) gets a fresh lookup instead of a dangling address.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

static uint64_t current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  CPM_CHECK(get_current && get_id, CPM_ERR_CUDA, "driver entry points cuCtxGetCurrent/cuCtxGetId unavailable");
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return (uint64_t)id + 1;  // 0 is reserved for "no valid context"
}

static double* scratch_address() {
  static std::mutex mu;
  static uint64_t ctx_of[128] = {0};
  static double* addr[128] = {nullptr};
  int dev = 0;
  CPM_CUDA_TRY(cudaGetDevice(&dev));
  CPM_CHECK(dev >= 0 && dev < 128, CPM_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(mu);
  const uint64_t id = current_context_id();
  if (id == 0 || id != ctx_of[dev] || !addr[dev]) {
    void* p = nullptr;
    CPM_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));  // makes the context current
    addr[dev] = static_cast<double*>(p);
    ctx_of[dev] = current_context_id();
  }
  return addr[dev];
}

void residual_norms_noalloc(const LevelView<double>& v, const double* f, const double* u,
                            const double* cvec, double cval, double* norms, cudaStream_t st) {
  CPM_CHECK(v.nplus <= CPM_NOALLOC_MAX_POINTS_VALUE, CPM_ERR_ARG,
            "cpm_residual_norms_noalloc: the finest level has more than 1048576 band + ghost "
            "points (the fixed scratch size); use cpm_residual_norms");
  double* scratch = scratch_address();
  double* w = scratch;
  double* part = scratch + CPM_NOALLOC_MAX_POINTS_VALUE;
  launch_extend<double>(v, u, w, (int32_t)v.nplus, st);
  const int nblocks = (v.nB + 255) / 256;
  if (nblocks > 0) {
    k_resid_partials_noalloc<<<nblocks, 256, 0, st>>>(v, u, w, f, cvec, cval, part);
    count_launch();
  }
  k_final_noalloc<<<1, 1024, 0, st>>>(part, nblocks, norms);
  count_launch();
  CPM_CUDA_TRY(cudaGetLastError());
}

}  // namespace cpm
