// Device operators of one level: the closest-point extension E (Sec. 3.1,
// Eq. 3.1), the operator M = diag(L) + (L - diag L) E (Sec. 2.3 Eq. 2.10,
// Remark 3.2), Jacobi smoothing (Eq. 4.1, Eq. 4.2), residuals, closest-point
// restriction and prolongation (Sec. 4.3), norms, and the setup kernels for
// diag(M) and the coarsest-level matrix.
#include <cmath>

#include "ops.cuh"
#include "gemv.cuh"

#include <atomic>

namespace cpm {

static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

static std::atomic<int64_t> g_launches{0};
static thread_local bool g_capturing = false;
void count_launch(int64_t n) {
  if (!g_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}
void set_capturing(bool on) { g_capturing = on; }
int64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

// ----------------------------------------------------------------- weights
// 1-D cubic Lagrange weights at fraction s for nodes -1, 0, 1, 2
// (the closed forms of the proof of Theorem 3.3, a = s dx):
//   l_-1 = -s(s-1)(s-2)/6, l_0 = (s+1)(s-1)(s-2)/2,
//   l_1  = -(s+1)s(s-2)/2, l_2 = (s+1)s(s-1)/6.
template <typename T>
__device__ __forceinline__ void cubic_w(T s, T w[4]) {
  const T sm1 = s - T(1), sm2 = s - T(2), sp1 = s + T(1);
  const T a = s * sm1, b = sp1 * sm2;
  w[0] = -(a * sm2) * T(1.0 / 6.0);
  w[1] = (b * sm1) * T(0.5);
  w[2] = -(b * s) * T(0.5);
  w[3] = (a * sp1) * T(1.0 / 6.0);
}

// ----------------------------------------------------------------- block reduce
__device__ inline void block_max_sum(double m, double s, double* part) {
  __shared__ double sm[32], ss[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sm[wid] = m; ss[wid] = s; }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    m = lane < nw ? sm[lane] : 0.0;
    s = lane < nw ? ss[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (lane == 0) {
      part[2 * blockIdx.x] = m;
      part[2 * blockIdx.x + 1] = s;
    }
  }
}

// ----------------------------------------------------------------- M stencil
template <typename T, int DIM, int MODE>
__global__ void __launch_bounds__(256) k_lap(LevelView<T> L, const T* u, const T* __restrict__ w,
                                             const T* __restrict__ f, const T* __restrict__ cvec,
                                             T cval, const T* __restrict__ dA, T omega, T* out,
                                             T* u_inout, double* part, const T* __restrict__ refv) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  double rm = 0.0, rs = 0.0;
  if (i < L.nB) {
    const T wi = w[i];
    const T ui = u[i];
    T s = T(0), Mu;
    if (MODE == LAP_RESID_REL) {
      const T ri = refv[i];
#pragma unroll
      for (int q = 0; q < 2 * DIM; ++q) {
        const int32_t k = __ldg(L.nbr + (int64_t)q * L.nB + i);
        s += (refv[k] - ri) + (w[k] - wi);
      }
      Mu = s * L.inv_h2 + L.gamma * ((ri - ui) + wi);
    } else {
#pragma unroll
      for (int q = 0; q < 2 * DIM; ++q) s += w[__ldg(L.nbr + (int64_t)q * L.nB + i)] - wi;
      Mu = s * L.inv_h2 + L.gamma * (wi - ui);
    }
    if (MODE == LAP_APPLY) {
      out[i] = Mu;
    } else {
      const T c = cvec ? cvec[i] : cval;
      const T r = f[i] - c * ui + Mu;
      if (MODE == LAP_RESID || MODE == LAP_RESID_REL) {
        out[i] = r;
        rm = fabs((double)r);
        rs = (double)r * (double)r;
      } else {
        u_inout[i] = ui + r * dA[i];
      }
    }
  }
  if ((MODE == LAP_RESID || MODE == LAP_RESID_REL) && part) block_max_sum(rm, rs, part);
}

template <int DIM, int MODE, typename T>
static void lap_dispatch(const LevelView<T>& L, const T* u, const T* w, const T* f, const T* cvec,
                         T cval, const T* dA, T omega, T* out, T* u_inout, double* part,
                         cudaStream_t st) {
  k_lap<T, DIM, MODE><<<nblk(L.nB, 256), 256, 0, st>>>(L, u, w, f, cvec, cval, dA, omega, out,
                                                         u_inout, part, nullptr);
  count_launch();
}

template <typename T>
void launch_lap(const LevelView<T>& L, LapMode mode, const T* u, const T* w, const T* f,
                const T* cvec, T cval, const T* dA, T omega, T* out, T* u_inout, double* part,
                int nblocks_part, cudaStream_t st) {
  (void)nblocks_part;
  if (L.nB <= 0) return;
  if (L.dim == 3) {
    if (mode == LAP_APPLY) lap_dispatch<3, LAP_APPLY>(L, u, w, f, cvec, cval, dA, omega, out, u_inout, part, st);
    if (mode == LAP_RESID) lap_dispatch<3, LAP_RESID>(L, u, w, f, cvec, cval, dA, omega, out, u_inout, part, st);
    if (mode == LAP_JACOBI) lap_dispatch<3, LAP_JACOBI>(L, u, w, f, cvec, cval, dA, omega, out, u_inout, part, st);
  } else {
    if (mode == LAP_APPLY) lap_dispatch<2, LAP_APPLY>(L, u, w, f, cvec, cval, dA, omega, out, u_inout, part, st);
    if (mode == LAP_RESID) lap_dispatch<2, LAP_RESID>(L, u, w, f, cvec, cval, dA, omega, out, u_inout, part, st);
    if (mode == LAP_JACOBI) lap_dispatch<2, LAP_JACOBI>(L, u, w, f, cvec, cval, dA, omega, out, u_inout, part, st);
  }
}

void launch_resid_rel(const LevelView<double>& L, const double* u, const double* delta,
                      const double* refv, const double* f, const double* cvec, double cval,
                      double* r, double* part, cudaStream_t st) {
  if (L.nB <= 0) return;
  if (L.dim == 3)
    k_lap<double, 3, LAP_RESID_REL><<<nblk(L.nB, 256), 256, 0, st>>>(
        L, u, delta, f, cvec, cval, nullptr, 0.0, r, nullptr, part, refv);
  else
    k_lap<double, 2, LAP_RESID_REL><<<nblk(L.nB, 256), 256, 0, st>>>(
        L, u, delta, f, cvec, cval, nullptr, 0.0, r, nullptr, part, refv);
  count_launch();
}

// ----------------------------------------------------------------- Ruuth-Merriman
template <typename T, int DIM, bool JAC>
__global__ void __launch_bounds__(256) k_rm(LevelView<T> L, const T* __restrict__ u,
                                            const T* __restrict__ f, const T* __restrict__ cvec,
                                            T cval, T omega, T* __restrict__ out) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.nB) return;
  T s = T(0);
#pragma unroll
  for (int q = 0; q < 2 * DIM; ++q) {
    const int32_t j = __ldg(L.nbr + (int64_t)q * L.nB + i);
    if (j < L.nB) s += u[j];  // band-restricted Laplacian: ghost neighbours dropped
  }
  const T c = cvec ? cvec[i] : cval;
  const T diag = c + L.gamma;
  const T ui = u[i];
  const T r = f[i] - diag * ui + s * L.inv_h2;
  out[i] = JAC ? ui + omega * r / diag : r;
}

template <typename T>
void launch_rm_jacobi(const LevelView<T>& L, const T* u, const T* f, const T* cvec, T cval, T omega,
                      T* out, cudaStream_t st) {
  if (L.dim == 3) k_rm<T, 3, true><<<nblk(L.nB, 256), 256, 0, st>>>(L, u, f, cvec, cval, omega, out);
  else k_rm<T, 2, true><<<nblk(L.nB, 256), 256, 0, st>>>(L, u, f, cvec, cval, omega, out);
  count_launch();
}
template <typename T>
void launch_rm_resid(const LevelView<T>& L, const T* u, const T* f, const T* cvec, T cval, T* out,
                     cudaStream_t st) {
  if (L.dim == 3) k_rm<T, 3, false><<<nblk(L.nB, 256), 256, 0, st>>>(L, u, f, cvec, cval, T(0), out);
  else k_rm<T, 2, false><<<nblk(L.nB, 256), 256, 0, st>>>(L, u, f, cvec, cval, T(0), out);
  count_launch();
}

// ----------------------------------------------------------------- transfers
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_transfer(TransferView<T> tv, const T* __restrict__ src,
                                                  T* __restrict__ dst, bool add) {
  const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= tv.n) return;
  const T sx = __ldg(tv.fr + j), sy = __ldg(tv.fr + tv.n + j);
  const T sz = DIM == 3 ? __ldg(tv.fr + 2 * tv.n + j) : T(0);
  const T wx[2] = {T(1) - sx, sx}, wy[2] = {T(1) - sy, sy}, wz[2] = {T(1) - sz, sz};
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < (DIM == 3 ? 2 : 1); ++c) {
    T accy = T(0);
#pragma unroll
    for (int bb = 0; bb < 2; ++bb) {
      const int q = 4 * c + 2 * bb;
      const T v0 = __ldg(src + __ldg(tv.src_idx + (int64_t)q * tv.n + j));
      const T v1 = __ldg(src + __ldg(tv.src_idx + (int64_t)(q + 1) * tv.n + j));
      accy += wy[bb] * (wx[0] * v0 + wx[1] * v1);
    }
    acc += (DIM == 3 ? wz[c] : T(1)) * accy;
  }
  dst[j] = add ? dst[j] + acc : acc;
}

template <typename T>
void launch_transfer(const TransferView<T>& tv, const T* src, T* dst, bool add, cudaStream_t st) {
  if (tv.n <= 0) return;
  if (tv.dim == 3) k_transfer<T, 3><<<nblk(tv.n, 256), 256, 0, st>>>(tv, src, dst, add);
  else k_transfer<T, 2><<<nblk(tv.n, 256), 256, 0, st>>>(tv, src, dst, add);
  count_launch();
}

// ----------------------------------------------------------------- norms
template <typename T>
__global__ void k_norm_partials(const T* __restrict__ x, int64_t n, double* part) {
  double m = 0.0, s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)x[i];
    m = fmax(m, fabs(v));
    s += v * v;
  }
  block_max_sum(m, s, part);
}

template <typename T>
void launch_norm_partials(const T* x, int64_t n, double* part, cudaStream_t st) {
  k_norm_partials<T><<<kNormBlocks, 256, 0, st>>>(x, n, part);
  count_launch();
}

// out[0] = max|x|, out[1] = sum x^2, out[2] = 1 / max|x| (0 if max is 0).
__global__ void k_norm_final(const double* part, int nblocks, double* out) {
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
    out[0] = M;
    out[1] = S;
    out[2] = M > 0.0 ? 1.0 / M : 0.0;
  }
}

void launch_norm_final(const double* part, int nblocks, double* out, cudaStream_t st) {
  k_norm_final<<<1, 1024, 0, st>>>(part, nblocks, out);
  count_launch();
}

// ----------------------------------------------------------------- mixed precision
__global__ void k_scale_to_f32(const double* __restrict__ r, const double* __restrict__ norms,
                               float* __restrict__ r32, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r32[i] = (float)(r[i] * norms[2]);
}
void launch_scale_to_f32(const double* r, const double* norms, float* r32, int64_t n, cudaStream_t st) {
  k_scale_to_f32<<<nblk(n, 256), 256, 0, st>>>(r, norms, r32, n);
  count_launch();
}

__global__ void k_axpy_scaled(double* __restrict__ u, const float* __restrict__ d,
                              const double* __restrict__ norms, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) u[i] += norms[0] * (double)d[i];
}
void launch_axpy_scaled(double* u, const float* d, const double* norms, int64_t n, cudaStream_t st) {
  k_axpy_scaled<<<nblk(n, 256), 256, 0, st>>>(u, d, norms, n);
  count_launch();
}

__global__ void k_axpy64(double* __restrict__ u, const double* __restrict__ d, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) u[i] += d[i];
}
void launch_axpy64(double* u, const double* d, int64_t n, cudaStream_t st) {
  k_axpy64<<<nblk(n, 256), 256, 0, st>>>(u, d, n);
  count_launch();
}

template <typename T>
__global__ void k_cast_to_f64(const T* x, double* y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (double)x[i];
}
template <typename T>
__global__ void k_cast_from_f64(const double* x, T* y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (T)x[i];
}
template <typename T>
void launch_cast_to_f64(const T* x, double* y, int64_t n, cudaStream_t st) {
  k_cast_to_f64<T><<<nblk(n, 256), 256, 0, st>>>(x, y, n);
}
template <typename T>
void launch_cast_from_f64(const double* x, T* y, int64_t n, cudaStream_t st) {
  k_cast_from_f64<T><<<nblk(n, 256), 256, 0, st>>>(x, y, n);
}

// ----------------------------------------------------------------- coarse solve
// x_g = Ainv b_g with the FP64 inverse (chunked dense product, FP64 accumulation).
template <typename T>
void launch_coarse_gemv(const double* Ainv, const T* const* b, T* const* x, int G, int32_t n,
                        cudaStream_t st) {
  launch_dense_gemv<double, T, false>(Ainv, b, x, G, n, st);
  count_launch((G + kGemvMaxVectors - 1) / kGemvMaxVectors);
}

// ----------------------------------------------------------------- setup: diag(M)
// M_ii = -gamma + (1/dx^2) sum_{k in N(i)} E_{k,i}: the weight of node i in
// the cubic stencil of cp(x_k) for each Laplacian neighbour k of i.
template <int DIM>
__global__ void k_diag_M(LevelView<double> L, double* __restrict__ diagM) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.nB) return;
  const uint64_t ki = L.key[i];
  const int own[3] = {key_x(ki), key_y(ki), key_z(ki)};
  const int d[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  double s = 0.0;
  for (int q = 0; q < 2 * DIM; ++q) {
    const int32_t kk = node_index(L.bv, own[0] + d[q][0], own[1] + d[q][1], own[2] + d[q][2]);
    if (kk < 0) continue;
    const uint64_t key = L.key[kk];
    const int base[3] = {key_x(key) + key_ox(key), key_y(key) + key_oy(key), key_z(key) + key_oz(key)};
    double wprod = 1.0;
    bool inside = true;
    for (int a = 0; a < DIM; ++a) {
      const int off = own[a] - base[a];
      if (off < 0 || off > 3) { inside = false; break; }
      double w[4];
      cubic_w(L.fr[a * L.nplus + kk], w);
      wprod *= w[off];
    }
    if (inside) s += wprod;
  }
  diagM[i] = -L.gamma + s * L.inv_h2;
}

void launch_diag_M(const LevelView<double>& L, double* diagM, cudaStream_t st) {
  if (L.dim == 3) k_diag_M<3><<<nblk(L.nB, 256), 256, 0, st>>>(L, diagM);
  else k_diag_M<2><<<nblk(L.nB, 256), 256, 0, st>>>(L, diagM);
}

// ----------------------------------------------------------------- setup: dense A
// Row i of A = diag(c) - M: A_ii += c_i + gamma, A_ij -= E_{k,j}/dx^2 for each
// neighbour k of i and stencil node j of cp(x_k).  One thread per row.
template <int DIM, typename M>
__global__ void k_assemble_A(LevelView<double> L, const double* cvec, double cval, M* A) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t n = L.nB;
  if (i >= n) return;
  M* row = A + (size_t)i * n;
  row[i] += (M)((cvec ? cvec[i] : cval) + L.gamma);
  const uint64_t ki = L.key[i];
  const int own[3] = {key_x(ki), key_y(ki), key_z(ki)};
  const int d[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  for (int q = 0; q < 2 * DIM; ++q) {
    const int32_t kk = node_index(L.bv, own[0] + d[q][0], own[1] + d[q][1], own[2] + d[q][2]);
    if (kk < 0) continue;
    const uint64_t key = L.key[kk];
    const int bx = key_x(key) + key_ox(key), by = key_y(key) + key_oy(key),
              bz = key_z(key) + key_oz(key);
    double wx[4], wy[4], wz[4] = {1.0, 0.0, 0.0, 0.0};
    cubic_w(L.fr[kk], wx);
    cubic_w(L.fr[L.nplus + kk], wy);
    if (DIM == 3) cubic_w(L.fr[2 * L.nplus + kk], wz);
    for (int c = 0; c < (DIM == 3 ? 4 : 1); ++c)
      for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) {
          const int32_t j = band_index(L.bv, bx + a, by + b, DIM == 3 ? bz + c : 0);
          if (j >= 0) row[j] -= (M)(wx[a] * wy[b] * wz[c] * L.inv_h2);
        }
  }
}

template <typename M>
void launch_assemble_A(const LevelView<double>& L, const double* cvec, double cval, M* A,
                       cudaStream_t st) {
  if (L.dim == 3) k_assemble_A<3, M><<<nblk(L.nB, 128), 128, 0, st>>>(L, cvec, cval, A);
  else k_assemble_A<2, M><<<nblk(L.nB, 128), 128, 0, st>>>(L, cvec, cval, A);
}
template void launch_assemble_A<double>(const LevelView<double>&, const double*, double, double*,
                                        cudaStream_t);
template void launch_assemble_A<float>(const LevelView<double>&, const double*, double, float*,
                                       cudaStream_t);

// ----------------------------------------------------------------- setup: inverse
// Gauss-Jordan with partial pivoting, in place: at step k the pivot row p
// (max |A[i][k]|, i >= k) is swapped into row k, row k is scaled by the
// reciprocal pivot (with A[k][k] replaced by 1 first), and every other row i
// subtracts A[i][k] times row k (with A[i][k] replaced by 0 first).  Row
// swaps permute the columns of the computed inverse; they are undone at the
// end in reverse order.
__global__ void k_gj_pivot(const double* A, int32_t n, int32_t k, int32_t* piv, int32_t* err) {
  double best = -1.0;
  int32_t arg = k;
  for (int32_t i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double v = fabs(A[(size_t)i * n + k]);
    if (v > best) { best = v; arg = i; }
  }
  __shared__ double sv[1024];
  __shared__ int32_t si[1024];
  sv[threadIdx.x] = best;
  si[threadIdx.x] = arg;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = sv[threadIdx.x + s];
      const int32_t oi = si[threadIdx.x + s];
      if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    piv[k] = si[0];
    if (!(sv[0] > 1e-300)) atomicOr(err, 1);
  }
}

__global__ void k_gj_swap_scale(double* A, int32_t n, int32_t k, const int32_t* piv, double* col) {
  const int32_t p = piv[k];
  double* rk = A + (size_t)k * n;
  if (p != k) {
    double* rp = A + (size_t)p * n;
    for (int32_t j = threadIdx.x; j < n; j += blockDim.x) {
      const double t = rk[j];
      rk[j] = rp[j];
      rp[j] = t;
    }
    __syncthreads();
  }
  __shared__ double pivinv;
  if (threadIdx.x == 0) {
    const double a = rk[k];
    pivinv = a != 0.0 ? 1.0 / a : 0.0;
    rk[k] = 1.0;
  }
  __syncthreads();
  for (int32_t j = threadIdx.x; j < n; j += blockDim.x) rk[j] *= pivinv;
  (void)col;
}

__global__ void k_gj_save_col(const double* A, int32_t n, int32_t k, double* col) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) col[i] = A[(size_t)i * n + k];
}

__global__ void k_gj_eliminate(double* A, int32_t n, int32_t k, const double* __restrict__ col) {
  const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t i = blockIdx.y;
  if (j >= n || i == k) return;
  const double m = col[i];
  if (m == 0.0) return;
  const double akj = A[(size_t)k * n + j];
  double* aij = A + (size_t)i * n + j;
  *aij = (j == k ? 0.0 : *aij) - m * akj;
}

__global__ void k_gj_swap_cols(double* A, int32_t n, int32_t k, const int32_t* piv) {
  const int32_t p = piv[k];
  if (p == k) return;
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* r = A + (size_t)i * n;
  const double t = r[k];
  r[k] = r[p];
  r[p] = t;
}

void invert_dense(double* A, int32_t n, cudaStream_t st, int32_t* err) {
  DBuf<int32_t> piv(n);
  DBuf<double> col(n);
  const dim3 eg(nblk(n, 256), n);
  for (int32_t k = 0; k < n; ++k) {
    k_gj_pivot<<<1, 1024, 0, st>>>(A, n, k, piv.get(), err);
    k_gj_swap_scale<<<1, 1024, 0, st>>>(A, n, k, piv.get(), col.get());
    k_gj_save_col<<<nblk(n, 256), 256, 0, st>>>(A, n, k, col.get());
    k_gj_eliminate<<<eg, 256, 0, st>>>(A, n, k, col.get());
  }
  for (int32_t k = n - 1; k >= 0; --k)
    k_gj_swap_cols<<<nblk(n, 256), 256, 0, st>>>(A, n, k, piv.get());
  CPM_CUDA_TRY(cudaGetLastError());
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
}

// ----------------------------------------------------------------- instantiations
#define CPM_INST(T)                                                                              \
  template void launch_lap<T>(const LevelView<T>&, LapMode, const T*, const T*, const T*,        \
                              const T*, T, const T*, T, T*, T*, double*, int, cudaStream_t);      \
  template void launch_rm_jacobi<T>(const LevelView<T>&, const T*, const T*, const T*, T, T, T*, \
                                    cudaStream_t);                                               \
  template void launch_rm_resid<T>(const LevelView<T>&, const T*, const T*, const T*, T, T*,     \
                                   cudaStream_t);                                                \
  template void launch_transfer<T>(const TransferView<T>&, const T*, T*, bool, cudaStream_t);    \
  template void launch_norm_partials<T>(const T*, int64_t, double*, cudaStream_t);               \
  template void launch_cast_to_f64<T>(const T*, double*, int64_t, cudaStream_t);                 \
  template void launch_cast_from_f64<T>(const double*, T*, int64_t, cudaStream_t);               \
  template void launch_coarse_gemv<T>(const double*, const T* const*, T* const*, int, int32_t, \
                                      cudaStream_t);
CPM_INST(double)
CPM_INST(float)

}  // namespace cpm
