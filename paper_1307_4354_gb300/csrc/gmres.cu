// Restarted GMRES on the coarsest level, for levels too large for a dense
// inverse (a Krylov solve of the coarsest system of Algorithm 4.1 step 2 in
// place of the direct one).  Everything stays on the device, with a fixed
// number of steps and restarts and no host synchronisation, so that it can be
// recorded in the V-cycle's CUDA graph:
//
//   x = 0; repeat `restarts` times:
//     r = b - A x, beta = ||r||, v_0 = -r / beta, g = beta e_0
//     for j < m:  z = P v_j,  w = (-A) z                (P = omega diag(A)^-1)
//                 h = V_j^T w, w -= V_j h, twice        (classical Gram-Schmidt,
//                 H[:, j] = h1 + h2                      reorthogonalised)
//                 H[j+1, j] = ||w||, v_{j+1} = w / ||w||
//                 Givens rotations on H[:, j] and g
//     y = R^-1 g (back substitution),  x += P V y
//
// The Krylov operator is -A with right-hand side -r (the residual kernel
// gives f - c z + M z = -A z for f = 0), so the correction solves A x = r.
#include <cmath>

#include "gmres.cuh"

namespace cpm {

static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr int kGmBlocks = 2 * 152;
constexpr int kGmThreads = 256;

// part[b * nv + i] = partial sum over block b of w . V_i, i < nv.
template <typename T>
__global__ void __launch_bounds__(kGmThreads) k_gm_dots(const T* __restrict__ w, const T* __restrict__ V,
                                                        int nv, int64_t n, double* part) {
  double acc[kGmresMaxM + 1];
#pragma unroll
  for (int i = 0; i <= kGmresMaxM; ++i) acc[i] = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double wk = (double)w[k];
#pragma unroll
    for (int i = 0; i <= kGmresMaxM; ++i)
      if (i < nv) acc[i] += wk * (double)V[(int64_t)i * n + k];
  }
  __shared__ double red[kGmThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < nv; ++i) {
    double s = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < kGmThreads / 32; ++q) t += red[q];
      part[(int64_t)blockIdx.x * nv + i] = t;
    }
    __syncthreads();
  }
}

// out[i] (+)= sum over blocks of part[b * nv + i] (fixed order).
__global__ void k_gm_dots_final(const double* part, int nblocks, int nv, double* out, bool add) {
  const int i = threadIdx.x;
  if (i >= nv) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * nv + i];
  out[i] = add ? out[i] + s : s;
}

// w -= sum_i h[i] V_i, i < nv.
template <typename T>
__global__ void k_gm_orth(T* __restrict__ w, const T* __restrict__ V, int nv, const double* h, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s = (double)w[k];
  for (int i = 0; i < nv; ++i) s -= h[i] * (double)V[(int64_t)i * n + k];
  w[k] = (T)s;
}

// dst = sign * src / sqrt(nrm2[0]) (0 where the norm vanishes); *hout = sqrt(nrm2[0]).
template <typename T>
__global__ void k_gm_normalise(T* dst, const T* src, const double* nrm2, double sign, int64_t n,
                               double* hout) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double nr = sqrt(nrm2[0]);
  if (k == 0 && hout) *hout = nr;
  if (k >= n) return;
  dst[k] = nr > 1e-300 ? (T)(sign * (double)src[k] / nr) : T(0);
}

// z = P v (P = omega / diag(A) per point).
template <typename T>
__global__ void k_gm_precond(T* z, const T* v, const T* dA, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) z[k] = v[k] * dA[k];
}

// Column j of H (column-major, ld = m + 1): the previous rotations, a new one
// zeroing H[j+1, j], and g rotated.  At j = m - 1 also y = R^-1 g.
__global__ void k_gm_givens(double* H, double* cs, double* sn, double* g, double* y, int j, int m) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* h = H + (int64_t)j * (m + 1);
  for (int i = 0; i < j; ++i) {
    const double a = h[i], b = h[i + 1];
    h[i] = cs[i] * a + sn[i] * b;
    h[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double a = h[j], b = h[j + 1];
  const double r = sqrt(a * a + b * b);
  const double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
  cs[j] = c;
  sn[j] = s;
  h[j] = r;
  h[j + 1] = 0.0;
  const double gj = g[j];
  g[j] = c * gj;
  g[j + 1] = -s * gj;
  if (j == m - 1) {
    for (int i = m - 1; i >= 0; --i) {
      double t = g[i];
      for (int k = i + 1; k < m; ++k) t -= H[(int64_t)k * (m + 1) + i] * y[k];
      const double d = H[(int64_t)i * (m + 1) + i];
      y[i] = d != 0.0 ? t / d : 0.0;
    }
  }
}

// g = beta e_0 (beta = sqrt(nrm2[0])).
__global__ void k_gm_init_g(double* g, const double* nrm2, int m) {
  const int i = threadIdx.x;
  if (i <= m) g[i] = i == 0 ? sqrt(nrm2[0]) : 0.0;
}

// x += P sum_j y_j V_j.
template <typename T>
__global__ void k_gm_update(T* x, const T* V, const double* y, const T* dA, int m, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s = 0.0;
  for (int j = 0; j < m; ++j) s += y[j] * (double)V[(int64_t)j * n + k];
  x[k] = (T)((double)x[k] + s * (double)dA[k]);
}

template <typename T>
void GmresWork<T>::alloc(int64_t n_, int m_) {
  n = n_;
  m = m_;
  V.alloc((size_t)(m + 1) * n);
  z.alloc(n);
  zero.alloc(n);
  r.alloc(n);
  H.alloc((size_t)(m + 1) * m);
  cs.alloc(m);
  sn.alloc(m);
  g.alloc(m + 1);
  y.alloc(m);
  h.alloc(2 * (m + 1));
  nrm.alloc(2);
  part.alloc((size_t)kGmBlocks * (m + 1));
}

template <typename T>
static void dots(const T* w, const T* V, int nv, int64_t n, double* part, double* out, bool add,
                 cudaStream_t st) {
  k_gm_dots<T><<<kGmBlocks, kGmThreads, 0, st>>>(w, V, nv, n, part);
  k_gm_dots_final<<<1, 32, 0, st>>>(part, kGmBlocks, nv, out, add);
  count_launch(2);
}

template <typename T>
void gmres_solve(const GmresOps<T>& op, GmresWork<T>& G, const T* b, T* x, const T* dA, int restarts,
                 cudaStream_t st) {
  const int64_t n = G.n;
  const int m = G.m;
  const unsigned gb = nblk(n, 256);
  CPM_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * n, st));
  CPM_CUDA_TRY(cudaMemsetAsync(G.zero.get(), 0, sizeof(T) * n, st));
  CPM_CUDA_TRY(cudaMemsetAsync(G.H.get(), 0, sizeof(double) * (m + 1) * m, st));
  for (int rs = 0; rs < restarts; ++rs) {
    op.residual(b, x, G.r.get(), st);  // r = b - A x
    dots<T>(G.r.get(), G.r.get(), 1, n, G.part.get(), G.nrm.get(), false, st);
    k_gm_init_g<<<1, 64, 0, st>>>(G.g.get(), G.nrm.get(), m);
    k_gm_normalise<T><<<gb, 256, 0, st>>>(G.V.get(), G.r.get(), G.nrm.get(), -1.0, n, nullptr);
    count_launch(2);
    for (int j = 0; j < m; ++j) {
      T* vj = G.V.get() + (int64_t)j * n;
      T* w = G.V.get() + (int64_t)(j + 1) * n;
      k_gm_precond<T><<<gb, 256, 0, st>>>(G.z.get(), vj, dA, n);
      count_launch();
      op.residual(G.zero.get(), G.z.get(), w, st);  // w = 0 - c z + M z = -A z
      double* hcol = G.H.get() + (int64_t)j * (m + 1);
      for (int pass = 0; pass < 2; ++pass) {
        dots<T>(w, G.V.get(), j + 1, n, G.part.get(), G.h.get() + pass * (m + 1), false, st);
        k_gm_orth<T><<<gb, 256, 0, st>>>(w, G.V.get(), j + 1, G.h.get() + pass * (m + 1), n);
        k_gm_dots_final<<<1, 32, 0, st>>>(G.h.get() + pass * (m + 1), 1, j + 1, hcol, pass > 0);
        count_launch(2);
      }
      dots<T>(w, w, 1, n, G.part.get(), G.nrm.get() + 1, false, st);
      k_gm_normalise<T><<<gb, 256, 0, st>>>(w, w, G.nrm.get() + 1, 1.0, n, hcol + j + 1);
      k_gm_givens<<<1, 1, 0, st>>>(G.H.get(), G.cs.get(), G.sn.get(), G.g.get(), G.y.get(), j, m);
      count_launch(2);
    }
    k_gm_update<T><<<gb, 256, 0, st>>>(x, G.V.get(), G.y.get(), dA, m, n);
    count_launch();
  }
  CPM_CUDA_TRY(cudaGetLastError());
}

template struct GmresWork<double>;
template struct GmresWork<float>;
template void gmres_solve<double>(const GmresOps<double>&, GmresWork<double>&, const double*, double*,
                                  const double*, int, cudaStream_t);
template void gmres_solve<float>(const GmresOps<float>&, GmresWork<float>&, const float*, float*,
                                 const float*, int, cudaStream_t);

}  // namespace cpm
