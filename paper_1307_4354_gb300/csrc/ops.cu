// Device operators of one level: the closest-point extension E (Sec. 3.1,
// Eq. 3.1), the operator M = diag(L) + (L - diag L) E (Sec. 2.3 Eq. 2.10,
// Remark 3.2), Jacobi smoothing (Eq. 4.1, Eq. 4.2), residuals, closest-point
// restriction and prolongation (Sec. 4.3), norms, and the setup kernels for
// diag(M) and the coarsest-level matrix.
#include <cmath>
#include <cstring>

#include "ops.cuh"
#include "gemv.cuh"
#include "pair.cuh"

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
// Stencil passes on B, one warp per brick (lane l handles nodes l and l + 32
// of the 4x4x4 brick; in 2-D lanes 0..15 the 16 nodes of a 4x4 brick).  The
// Laplacian neighbours of a node are found by brick addressing: a neighbour
// inside the brick is a local position of the same brick, one across a face
// is a local position of the face-neighbour brick, and its index in B+ is
// start + popcount of the occupancy mask below it (band mask first, then
// ghost mask).  The brick tables are warp-uniform loads, so the pass reads
// no per-point index table: per point only u, f, diag and w (and writes the
// result).
// Occupancy masks and starts of one slot of a brick record.
struct SlotTab {
  uint64_t bm, gm;
  int32_t bs, gs;
};
template <bool BAND_ONLY>
__device__ __forceinline__ SlotTab slot_tab(const BrickRec* R, int q) {
  SlotTab t;
  t.bm = __ldg(&R->bm[q]);
  t.bs = __ldg(&R->bs[q]);
  t.gm = BAND_ONLY ? 0ull : __ldg(&R->gm[q]);
  t.gs = BAND_ONLY ? 0 : __ldg(&R->gs[q]);
  return t;
}
// Index in B+ (or in B only) of local node l of a brick, -1 if absent.
__device__ __forceinline__ int32_t tab_index(const SlotTab& t, int l, int32_t nB) {
  const uint64_t bit = 1ull << l;
  if (t.bm & bit) return t.bs + __popcll(t.bm & (bit - 1ull));
  if (t.gm & bit) return nB + t.gs + __popcll(t.gm & (bit - 1ull));
  return -1;
}
// The 2d neighbours (-x, +x, -y, +y, -z, +z) of local node l: inside the
// brick (its own tables, already in registers) or across a face (the tables
// of record slot q + 1, loaded only for nodes on that face).
template <int DIM, bool BAND_ONLY>
__device__ __forceinline__ void brick_neighbours(const BrickRec* R, const SlotTab& own, int l,
                                                 int32_t nB, int32_t k[6]) {
  const int x = l & 3, y = (l >> 2) & 3, z = l >> 4;
  const int step[3] = {1, 4, 16};
  const int pos[3] = {x, y, z};
#pragma unroll
  for (int q = 0; q < 2 * DIM; ++q) {
    const int a = q >> 1;
    const bool up = q & 1;
    const bool face = up ? pos[a] == 3 : pos[a] == 0;
    const int ln = face ? (up ? l - 3 * step[a] : l + 3 * step[a]) : (up ? l + step[a] : l - step[a]);
    k[q] = tab_index(face ? slot_tab<BAND_ONLY>(R, q + 1) : own, ln, nB);
  }
}

// Threads per brick of the stencil passes: 64 (one node each) or 32 (two).
#ifndef CPM_LAP_TPB
#define CPM_LAP_TPB 64
#endif
constexpr int kLapTPB = CPM_LAP_TPB;
static_assert(kLapTPB == 32 || kLapTPB == 64, "threads per brick");

// Stencil passes over the per-point neighbour table (1) or by brick
// addressing (0).
#ifndef CPM_LAP_INDEXED
#define CPM_LAP_INDEXED 1
#endif
constexpr bool kLapIndexed = CPM_LAP_INDEXED != 0;

template <typename T>
static unsigned lap_grid(const LevelView<T>& L) {
  return kLapIndexed ? nblk(L.nB, 256) : nblk((int64_t)L.bv.nbricks * kLapTPB, 256);
}
int lap_blocks_f64(const LevelView<double>& L) { return (int)lap_grid(L); }

// MODE (LapMode, plus the Ruuth-Merriman pieces):
//   APPLY : out = M u
//   RESID : out = f - c u + M u, block partials of max|out|, sum out^2
//   JACOBI: u += (f - c u + M u) * dA (in place)
//   RESID_REL: RESID from the relative extension (w = delta, refv)
//   RM_JAC / RM_RES: band-restricted Laplacian L_B on u (ghost neighbours
//           dropped): out = u + omega (f - (cI - L_B) u) / (c + gamma), or
//           out = f - (cI - L_B) u
constexpr int LAP_RM_JAC = 8, LAP_RM_RES = 9, LAP_BAND = 10, LAP_VARD = 11;
template <typename T, int DIM, int MODE>
__global__ void __launch_bounds__(256) k_lap(LevelView<T> L, const T* u, const T* __restrict__ w,
                                             const T* __restrict__ f, const T* __restrict__ cvec,
                                             T cval, const T* __restrict__ dA, T omega, T* out,
                                             T* u_inout, double* part, const T* __restrict__ refv) {
  constexpr bool RM = MODE == LAP_RM_JAC || MODE == LAP_RM_RES || MODE == LAP_BAND || MODE == LAP_VARD;
  const int32_t b = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) / kLapTPB);
  const int lane = threadIdx.x % kLapTPB;
  double rm = 0.0, rs = 0.0;
  const BrickRec* R = L.bv.brec + (b < L.bv.nbricks ? b : 0);
  const uint64_t bm = b < L.bv.nbricks ? __ldg(&R->bm[0]) : 0ull;
  if (bm) {
    const SlotTab own = slot_tab<RM>(R, 0);
    const int32_t bs = own.bs;
#pragma unroll
    for (int h = 0; h < (DIM == 3 ? 64 / kLapTPB : 1); ++h) {
      const int l = lane + kLapTPB * h;
      if ((DIM == 2 && l >= 16) || !((bm >> l) & 1ull)) continue;
      if ((MODE == LAP_JAC_RED || MODE == LAP_JAC_BLACK) &&
          node_colour_local(l) != (MODE == LAP_JAC_BLACK ? 1 : 0))
        continue;
      const int32_t i = bs + __popcll(bm & ((1ull << l) - 1ull));
      int32_t k[6];
      brick_neighbours<DIM, RM>(R, own, l, L.nB, k);
      const T ui = u[i];
      if (MODE == LAP_VARD) {  // out = L~ u, refv = the diffusion coefficient a
        const T ai = refv[i];
        T s = T(0);
#pragma unroll
        for (int q = 0; q < 2 * DIM; ++q)
          if (k[q] >= 0) s += (T(0.5) * (ai + refv[k[q]])) * (u[k[q]] - ui);
        out[i] = s * L.inv_h2;
        continue;
      }
      if (RM) {
        T s = T(0);
#pragma unroll
        for (int q = 0; q < 2 * DIM; ++q)
          if (k[q] >= 0) s += u[k[q]];
        if (MODE == LAP_BAND) {  // out = L_B u
          out[i] = s * L.inv_h2 - L.gamma * ui;
          continue;
        }
        const T c = cvec ? cvec[i] : cval;
        const T diag = c + L.gamma;
        const T r = f[i] - diag * ui + s * L.inv_h2;
        out[i] = MODE == LAP_RM_JAC ? ui + omega * r / diag : r;
        continue;
      }
      const T wi = w[i];
      T s = T(0), Mu;
      if (MODE == LAP_RESID_REL || MODE == LAP_JAC_REL) {
        const T ri = refv[i];
#pragma unroll
        for (int q = 0; q < 2 * DIM; ++q) {
          const int32_t kk = k[q] < 0 ? i : k[q];
          s += (refv[kk] - ri) + (w[kk] - wi);
        }
        Mu = s * L.inv_h2 + L.gamma * ((ri - ui) + wi);
      } else {
#pragma unroll
        for (int q = 0; q < 2 * DIM; ++q) s += w[k[q] < 0 ? i : k[q]] - wi;
        Mu = s * L.inv_h2 + L.gamma * (wi - ui);
      }
      if (MODE == LAP_APPLY) {
        out[i] = Mu;
      } else {
        const T c = cvec ? cvec[i] : cval;
        const T r = f[i] - c * ui + Mu;
        if (MODE == LAP_RESID || MODE == LAP_RESID_REL) {
          out[i] = r;
          rm = fmax(rm, fabs((double)r));
          rs += (double)r * (double)r;
        } else {
          u_inout[i] = ui + r * dA[i];
        }
      }
    }
  }
  if ((MODE == LAP_RESID || MODE == LAP_RESID_REL) && part) block_max_sum(rm, rs, part);
}

// The same passes with one thread per band point and its 2d neighbours read
// from the per-point index table (B+ indices, the node itself where a
// neighbour is missing).  Ruuth-Merriman modes drop ghost neighbours.
template <typename T, int DIM, int MODE>
__global__ void __launch_bounds__(256) k_lap_idx(LevelView<T> L, const T* u, const T* __restrict__ w,
                                                 const T* __restrict__ f, const T* __restrict__ cvec,
                                                 T cval, const T* __restrict__ dA, T omega, T* out,
                                                 T* u_inout, double* part, const T* __restrict__ refv) {
  constexpr bool RM = MODE == LAP_RM_JAC || MODE == LAP_RM_RES || MODE == LAP_BAND || MODE == LAP_VARD;
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  double rm = 0.0, rs = 0.0;
  bool active = i < L.nB;
  if (active && (MODE == LAP_JAC_RED || MODE == LAP_JAC_BLACK)) {
    const uint64_t kk = __ldg(L.key + i);
    active = ((key_x(kk) + key_y(kk) + (DIM == 3 ? key_z(kk) : 0)) & 1) == (MODE == LAP_JAC_BLACK ? 1 : 0);
  }
  if (active) {
    int32_t k[6];
#pragma unroll
    for (int q = 0; q < 2 * DIM; ++q) k[q] = __ldg(L.nbr + (int64_t)q * L.nB + i);
    const T ui = u[i];
    if (MODE == LAP_VARD) {  // out = L~ u, refv = the diffusion coefficient a
      const T ai = refv[i];
      T s = T(0);
#pragma unroll
      for (int q = 0; q < 2 * DIM; ++q)
        if (k[q] < L.nB && k[q] != i) s += (T(0.5) * (ai + refv[k[q]])) * (u[k[q]] - ui);
      out[i] = s * L.inv_h2;
    } else if (RM) {
      T s = T(0);
#pragma unroll
      for (int q = 0; q < 2 * DIM; ++q)
        if (k[q] < L.nB && k[q] != i) s += u[k[q]];
      if (MODE == LAP_BAND) {
        out[i] = s * L.inv_h2 - L.gamma * ui;
      } else {
        const T c = cvec ? cvec[i] : cval;
        const T diag = c + L.gamma;
        const T r = f[i] - diag * ui + s * L.inv_h2;
        out[i] = MODE == LAP_RM_JAC ? ui + omega * r / diag : r;
      }
    } else {
      const T wi = w[i];
      T s = T(0), Mu;
      if (MODE == LAP_RESID_REL || MODE == LAP_JAC_REL) {
        const T ri = refv[i];
#pragma unroll
        for (int q = 0; q < 2 * DIM; ++q) s += (refv[k[q]] - ri) + (w[k[q]] - wi);
        Mu = s * L.inv_h2 + L.gamma * ((ri - ui) + wi);
      } else {
#pragma unroll
        for (int q = 0; q < 2 * DIM; ++q) s += w[k[q]] - wi;
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
  }
  if ((MODE == LAP_RESID || MODE == LAP_RESID_REL) && part) block_max_sum(rm, rs, part);
}

template <int DIM, int MODE, typename T>
static void lap_dispatch(const LevelView<T>& L, const T* u, const T* w, const T* f, const T* cvec,
                         T cval, const T* dA, T omega, T* out, T* u_inout, double* part,
                         const T* refv, cudaStream_t st) {
  if (kLapIndexed)
    k_lap_idx<T, DIM, MODE><<<lap_grid(L), 256, 0, st>>>(L, u, w, f, cvec, cval, dA, omega, out,
                                                          u_inout, part, refv);
  else
    k_lap<T, DIM, MODE><<<lap_grid(L), 256, 0, st>>>(L, u, w, f, cvec, cval, dA, omega, out, u_inout,
                                                      part, refv);
  count_launch();
}

template <int MODE, typename T>
static void lap_dim(const LevelView<T>& L, const T* u, const T* w, const T* f, const T* cvec, T cval,
                    const T* dA, T omega, T* out, T* u_inout, double* part, const T* refv,
                    cudaStream_t st) {
  if (L.nB <= 0) return;
  if (L.dim == 3)
    lap_dispatch<3, MODE>(L, u, w, f, cvec, cval, dA, omega, out, u_inout, part, refv, st);
  else
    lap_dispatch<2, MODE>(L, u, w, f, cvec, cval, dA, omega, out, u_inout, part, refv, st);
}

template <typename T>
void launch_lap(const LevelView<T>& L, LapMode mode, const T* u, const T* w, const T* f,
                const T* cvec, T cval, const T* dA, T omega, T* out, T* u_inout, double* part,
                int nblocks_part, cudaStream_t st) {
  (void)nblocks_part;
  if (mode == LAP_APPLY) lap_dim<LAP_APPLY>(L, u, w, f, cvec, cval, dA, omega, out, u_inout, part, (const T*)nullptr, st);
  if (mode == LAP_RESID) lap_dim<LAP_RESID>(L, u, w, f, cvec, cval, dA, omega, out, u_inout, part, (const T*)nullptr, st);
  if (mode == LAP_JACOBI) lap_dim<LAP_JACOBI>(L, u, w, f, cvec, cval, dA, omega, out, u_inout, part, (const T*)nullptr, st);
  if (mode == LAP_JAC_RED) lap_dim<LAP_JAC_RED>(L, u, w, f, cvec, cval, dA, omega, out, u_inout, part, (const T*)nullptr, st);
  if (mode == LAP_JAC_BLACK) lap_dim<LAP_JAC_BLACK>(L, u, w, f, cvec, cval, dA, omega, out, u_inout, part, (const T*)nullptr, st);
}

template <typename T>
void launch_lap_rel(const LevelView<T>& L, LapMode mode, const T* u, const T* delta, const T* refv,
                    const T* f, const T* cvec, T cval, const T* dA, T* out, T* u_inout, double* part,
                    cudaStream_t st) {
  if (mode == LAP_RESID_REL)
    lap_dim<LAP_RESID_REL>(L, u, delta, f, cvec, cval, dA, T(0), out, u_inout, part, refv, st);
  else
    lap_dim<LAP_JAC_REL>(L, u, delta, f, cvec, cval, dA, T(0), out, u_inout, part, refv, st);
}

void launch_resid_rel(const LevelView<double>& L, const double* u, const double* delta,
                      const double* refv, const double* f, const double* cvec, double cval,
                      double* r, double* part, cudaStream_t st) {
  lap_dim<LAP_RESID_REL>(L, u, delta, f, cvec, cval, (const double*)nullptr, 0.0, r, (double*)nullptr,
                         part, refv, st);
}

// ---------------------------------------------------- outer residual, FP32 pairs
// r = f - c u + M u on B from the pair extension (delta_j pairs, ref_j floats):
// M u_i = S / dx^2 + gamma ((ref_i - u_i) + delta_i) with
// S = sum over the 2d neighbours k of (ref_k - ref_i) + (delta_k - delta_i),
// summed in pairs (the reference differences are exact TwoSums of floats),
// scaled by 1/dx^2 and gamma as pairs.  FP64 work per point: ref_i - u_i,
// f - c u_i and the sum with M u_i, and r^2 for the norm (the maximum is taken
// on the bit patterns of |r|).  Each thread takes kPairPts points (strided by
// the block), so the block's norm reduction is shared by several points.
constexpr int kPairPts = 4;

// Largest |x| and sum of x^2 over the block into part[2 b], part[2 b + 1];
// m holds the bit pattern of a non-negative double (ordered as an integer).
__device__ inline void block_maxbits_sum(unsigned long long m, double s, double* part) {
  __shared__ unsigned long long sm[32];
  __shared__ double ss[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sm[wid] = m; ss[wid] = s; }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    m = lane < nw ? sm[lane] : 0ull;
    s = lane < nw ? ss[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
      s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (lane == 0) {
      part[2 * blockIdx.x] = __longlong_as_double((long long)m);
      part[2 * blockIdx.x + 1] = s;
    }
  }
}

template <int DIM>
__global__ void __launch_bounds__(256) k_resid_pair(LevelView<double> L, const double* __restrict__ u,
                                                    const float2* __restrict__ dp,
                                                    const float* __restrict__ rp,
                                                    const double* __restrict__ f,
                                                    const double* __restrict__ cvec, double cval,
                                                    float2 ih2, float2 gam, double* __restrict__ r,
                                                    double* part) {
  unsigned long long rm = 0ull;
  double rs = 0.0;
#pragma unroll
  for (int j = 0; j < kPairPts; ++j) {
    const int32_t i = (blockIdx.x * kPairPts + j) * blockDim.x + threadIdx.x;
    if (i >= L.nB) continue;  // (not break: the points' loads can then overlap)
    int32_t k[2 * DIM];
#pragma unroll
    for (int q = 0; q < 2 * DIM; ++q) k[q] = __ldg(L.nbr + (int64_t)q * L.nB + i);
    const float ri = __ldg(rp + i);
    const float2 di = __ldg(dp + i);
    float sh = 0.f, sl = 0.f;
#pragma unroll
    for (int q = 0; q < 2 * DIM; ++q) {
      const float rk = __ldg(rp + k[q]);
      const float2 dk = __ldg(dp + k[q]);
      float ah, al, bh, bl, ch, cl, t;
      two_sum(rk, -ri, ah, al);
      two_sum(dk.x, -di.x, bh, bl);
      two_sum(ah, bh, ch, cl);
      two_sum(sh, ch, sh, t);
      sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(al, bl), __fadd_rn(cl, t)));
      sl = __fadd_rn(sl, __fsub_rn(dk.y, di.y));
    }
    float Sh, Sl, lh, ll;
    fast_two_sum(sh, sl, Sh, Sl);
    pair_mul(Sh, Sl, ih2.x, ih2.y, lh, ll);             // S / dx^2
    const double ui = u[i];
    const float2 e = pair_split(pair_f2d(ri) - ui);      // ref_i - u_i
    float th, tl, gh, gl, mh, ml;
    pair_add(e.x, e.y, di.x, di.y, th, tl);
    pair_mul(th, tl, gam.x, gam.y, gh, gl);             // gamma ((ref_i - u_i) + delta_i)
    pair_add(lh, ll, gh, gl, mh, ml);                   // M u_i
    const double c = cvec ? cvec[i] : cval;
    const double res = (f[i] - c * ui) + pair_to_f64(mh, ml);
    r[i] = res;
    rm = max(rm, (unsigned long long)__double_as_longlong(res) & 0x7FFFFFFFFFFFFFFFull);  // |res|
    rs += res * res;
  }
  if (part) block_maxbits_sum(rm, rs, part);
}

int resid_pair_blocks(const LevelView<double>& L) {
  return (int)((L.nB + 256 * kPairPts - 1) / (256 * kPairPts));
}

void launch_resid_pair(const LevelView<double>& L, const double* u, const float2* delta,
                       const float* refv, const double* f, const double* cvec, double cval, double* r,
                       double* part, cudaStream_t st) {
  if (L.nB <= 0) return;
  const unsigned nb = (unsigned)resid_pair_blocks(L);
  const double ih2 = (double)L.inv_h2, gam = (double)L.gamma;
  const float ih2h = (float)ih2, gamh = (float)gam;
  const float2 ih2p = make_float2(ih2h, (float)(ih2 - (double)ih2h));
  const float2 gamp = make_float2(gamh, (float)(gam - (double)gamh));
  if (L.dim == 3)
    k_resid_pair<3><<<nb, 256, 0, st>>>(L, u, delta, refv, f, cvec, cval, ih2p, gamp, r, part);
  else
    k_resid_pair<2><<<nb, 256, 0, st>>>(L, u, delta, refv, f, cvec, cval, ih2p, gamp, r, part);
  count_launch();
}

// ------------------------------------------------- pointwise FP64 residual check
// After an outer residual in FP32 pairs that meets the tolerance only within
// its error estimate, only the band points whose |r_i| exceeds thr = (tol -
// estimate) max|f| can violate the tolerance.  k_check_select lists them (at
// most cap; *count may exceed cap, the list is then incomplete) and
// k_check_points evaluates r_i there in FP64, in the relative form with the
// point's own value as the common reference: delta_j = sum_m E_jm (u_m - u_i)
// for j = i and its 2d neighbours (cubic weights from the fractions, stencil
// nodes through the brick tables), M u_i = sum_q (delta_kq - delta_i) / dx^2 +
// gamma delta_i, r_i = f_i - c_i u_i + M u_i; the maximum |r_i| goes to *maxbits
// (bit pattern of a non-negative double).  The stencil rows of one point are
// summed with shared-memory atomics, so the last bits of r_i may vary from
// run to run.
__global__ void k_check_select(const double* __restrict__ r, int32_t nB, unsigned long long thr_bits,
                               int32_t* __restrict__ list, int32_t cap, int32_t* count) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nB) return;
  const unsigned long long a = (unsigned long long)__double_as_longlong(r[i]) & 0x7FFFFFFFFFFFFFFFull;
  if (a > thr_bits) {
    const int32_t p = atomicAdd(count, 1);
    if (p < cap) list[p] = i;
  }
}

// One warp per candidate point i: the 2d + 1 extension values it needs (at i
// and at its Laplacian neighbours) are split into 4-node rows of their cubic
// stencils, spread over the lanes, and summed per value in shared memory.
constexpr int kCheckWarps = 4;

template <int DIM>
__global__ void __launch_bounds__(kCheckWarps * 32) k_check_points(
    LevelView<double> L, const double* __restrict__ u, const double* __restrict__ f,
    const double* __restrict__ cvec, double cval, const int32_t* __restrict__ list,
    const int32_t* count, int32_t cap, unsigned long long* maxbits) {
  constexpr int R = DIM == 3 ? 16 : 4;  // stencil rows of 4 nodes per value
  constexpr int NJ = 2 * DIM + 1;       // values: the point, then its neighbours
  __shared__ double part[kCheckWarps][NJ];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t n = min(*count, cap);
  for (int32_t t = blockIdx.x * kCheckWarps + warp; t < n; t += gridDim.x * kCheckWarps) {
    const int32_t i = list[t];
    const double ui = u[i];
    if (lane < NJ) part[warp][lane] = 0.0;
    __syncwarp();
    for (int e = lane; e < NJ * R; e += 32) {
      const int jj = e / R, row = e % R;
      const int32_t j = jj == 0 ? i : __ldg(L.nbr + (int64_t)(jj - 1) * L.nB + i);
      const uint64_t kk = __ldg(L.key + j);
      const int bx = key_x(kk) + key_ox(kk), by = key_y(kk) + key_oy(kk);
      const int bz = DIM == 3 ? key_z(kk) + key_oz(kk) : 0;
      const int b = row & 3, c = row >> 2;
      double w[3][4];  // cubic Lagrange weights at nodes -1, 0, 1, 2 per axis
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const double sf = __ldg(L.fr + a * L.nplus + j);
        const double sm1 = sf - 1.0, sm2 = sf - 2.0, sp1 = sf + 1.0;
        const double p = sf * sm1, q = sp1 * sm2;
        w[a][0] = -(p * sm2) * (1.0 / 6.0);
        w[a][1] = (q * sm1) * 0.5;
        w[a][2] = -(q * sf) * 0.5;
        w[a][3] = (p * sp1) * (1.0 / 6.0);
      }
      double acc = 0.0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int32_t m = band_index(L.bv, bx + a, by + b, bz + c);
        acc += w[0][a] * ((m >= 0 ? __ldg(u + m) : ui) - ui);
      }
      atomicAdd(&part[warp][jj], w[1][b] * (DIM == 3 ? w[2][c] : 1.0) * acc);
    }
    __syncwarp();
    if (lane == 0) {
      const double di = part[warp][0];
      double s = 0.0;
      for (int q = 1; q < NJ; ++q) s += part[warp][q] - di;
      const double c = cvec ? cvec[i] : cval;
      const double r = f[i] - c * ui + (s * L.inv_h2 + L.gamma * di);
      atomicMax(maxbits, (unsigned long long)__double_as_longlong(r) & 0x7FFFFFFFFFFFFFFFull);
    }
    __syncwarp();
  }
}

void launch_pointwise_check(const LevelView<double>& L, const double* u, const double* f,
                            const double* cvec, double cval, const double* r, double thr,
                            int32_t* list, int32_t cap, int32_t* count, unsigned long long* maxbits,
                            cudaStream_t st) {
  CPM_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int32_t), st));
  CPM_CUDA_TRY(cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long), st));
  if (L.nB <= 0) return;
  unsigned long long thr_bits = 0ull;
  if (thr > 0.0) std::memcpy(&thr_bits, &thr, sizeof(thr));
  k_check_select<<<nblk(L.nB, 256), 256, 0, st>>>(r, L.nB, thr_bits, list, cap, count);
  const unsigned grid = 2 * 152;  // warps loop over the candidates
  if (L.dim == 3)
    k_check_points<3><<<grid, kCheckWarps * 32, 0, st>>>(L, u, f, cvec, cval, list, count, cap, maxbits);
  else
    k_check_points<2><<<grid, kCheckWarps * 32, 0, st>>>(L, u, f, cvec, cval, list, count, cap, maxbits);
  count_launch(2);
}

// ----------------------------------------------------------------- Ruuth-Merriman
template <typename T>
void launch_rm_jacobi(const LevelView<T>& L, const T* u, const T* f, const T* cvec, T cval, T omega,
                      T* out, cudaStream_t st) {
  lap_dim<LAP_RM_JAC>(L, u, (const T*)nullptr, f, cvec, cval, (const T*)nullptr, omega, out,
                      (T*)nullptr, nullptr, (const T*)nullptr, st);
}
template <typename T>
void launch_rm_resid(const LevelView<T>& L, const T* u, const T* f, const T* cvec, T cval, T* out,
                     cudaStream_t st) {
  lap_dim<LAP_RM_RES>(L, u, (const T*)nullptr, f, cvec, cval, (const T*)nullptr, T(0), out,
                      (T*)nullptr, nullptr, (const T*)nullptr, st);
}

// ----------------------------------------------------------------- paper form
// The paper's own scheme (Sec. 3.1, Eq. 3.3): M u = E_1 (L_B u) - gamma (u - E_3 u)
// on B, with L_B the band-restricted 2d+1-point Laplacian, E_1 linear and
// E_3 cubic interpolation at cp.  Given v = L_B u (launch_lap_band) and
// w = E_3 u on B (launch_extend over B), one thread per band point gathers v
// at the 2^d linear-stencil nodes of cp(x_i) (the middle nodes of its cubic
// stencil, same fractions) through the brick tables.
template <typename T>
void launch_lap_band(const LevelView<T>& L, const T* u, T* v, cudaStream_t st) {
  lap_dim<LAP_BAND>(L, u, (const T*)nullptr, (const T*)nullptr, (const T*)nullptr, T(0),
                    (const T*)nullptr, T(0), v, (T*)nullptr, nullptr, (const T*)nullptr, st);
}

template <typename T>
void launch_lap_vard(const LevelView<T>& L, const T* u, const T* a, T* v, cudaStream_t st) {
  lap_dim<LAP_VARD>(L, u, (const T*)nullptr, (const T*)nullptr, (const T*)nullptr, T(0),
                    (const T*)nullptr, T(0), v, (T*)nullptr, nullptr, a, st);
}

template <typename T, int DIM, int MODE>
__global__ void __launch_bounds__(256) k_paper(LevelView<T> L, const T* u, const T* __restrict__ v,
                                               const T* __restrict__ w, const T* __restrict__ f,
                                               const T* __restrict__ cvec, T cval,
                                               const T* __restrict__ dA, T* out, T* u_inout,
                                               double* part, const T* __restrict__ avec) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  double rm = 0.0, rs = 0.0;
  const uint64_t k = i < L.nB ? __ldg(L.key + i) : 0ull;
  const bool skip = (MODE == LAP_JAC_RED || MODE == LAP_JAC_BLACK) &&
                    ((key_x(k) + key_y(k) + (DIM == 3 ? key_z(k) : 0)) & 1) != (MODE == LAP_JAC_BLACK ? 1 : 0);
  if (i < L.nB && !skip) {
    const int bx = key_x(k) + key_ox(k) + 1, by = key_y(k) + key_oy(k) + 1;
    const int bz = DIM == 3 ? key_z(k) + key_oz(k) + 1 : 0;
    const T sx = __ldg(L.fr + i), sy = __ldg(L.fr + L.nplus + i);
    const T sz = DIM == 3 ? __ldg(L.fr + 2 * L.nplus + i) : T(0);
    const T wx[2] = {T(1) - sx, sx}, wy[2] = {T(1) - sy, sy}, wz[2] = {T(1) - sz, sz};
    T e1v = T(0);
#pragma unroll
    for (int c = 0; c < (DIM == 3 ? 2 : 1); ++c) {
      T accy = T(0);
#pragma unroll
      for (int bb = 0; bb < 2; ++bb) {
        const int32_t j0 = band_index(L.bv, bx, by + bb, bz + c);
        const int32_t j1 = band_index(L.bv, bx + 1, by + bb, bz + c);
        accy += wy[bb] * (wx[0] * v[j0 < 0 ? i : j0] + wx[1] * v[j1 < 0 ? i : j1]);
      }
      e1v += (DIM == 3 ? wz[c] : T(1)) * accy;
    }
    const T ui = u[i];
    const T g = avec ? L.gamma * avec[i] : L.gamma;  // side-condition weight gamma a_i
    const T Mu = e1v - g * (ui - w[i]);
    if (MODE == LAP_APPLY) {
      out[i] = Mu;
    } else {
      const T cc = cvec ? cvec[i] : cval;
      const T r = f[i] - cc * ui + Mu;
      if (MODE == LAP_RESID) {
        out[i] = r;
        rm = fabs((double)r);
        rs = (double)r * (double)r;
      } else {
        u_inout[i] = ui + r * dA[i];
      }
    }
  }
  if (MODE == LAP_RESID && part) block_max_sum(rm, rs, part);
}

int paper_blocks(const LevelView<double>& L) { return (int)nblk(L.nB, 256); }

template <typename T>
void launch_paper(const LevelView<T>& L, LapMode mode, const T* u, const T* v, const T* w, const T* f,
                  const T* cvec, T cval, const T* dA, T* out, T* u_inout, double* part,
                  const T* avec, cudaStream_t st) {
  if (L.nB <= 0) return;
  const unsigned g = nblk(L.nB, 256);
#define CPM_PAPER(DIM, MODE) \
  k_paper<T, DIM, MODE><<<g, 256, 0, st>>>(L, u, v, w, f, cvec, cval, dA, out, u_inout, part, avec)
  if (L.dim == 3) {
    if (mode == LAP_APPLY) CPM_PAPER(3, LAP_APPLY);
    else if (mode == LAP_RESID) CPM_PAPER(3, LAP_RESID);
    else if (mode == LAP_JAC_RED) CPM_PAPER(3, LAP_JAC_RED);
    else if (mode == LAP_JAC_BLACK) CPM_PAPER(3, LAP_JAC_BLACK);
    else CPM_PAPER(3, LAP_JACOBI);
  } else {
    if (mode == LAP_APPLY) CPM_PAPER(2, LAP_APPLY);
    else if (mode == LAP_RESID) CPM_PAPER(2, LAP_RESID);
    else if (mode == LAP_JAC_RED) CPM_PAPER(2, LAP_JAC_RED);
    else if (mode == LAP_JAC_BLACK) CPM_PAPER(2, LAP_JAC_BLACK);
    else CPM_PAPER(2, LAP_JACOBI);
  }
#undef CPM_PAPER
  count_launch();
}

// ----------------------------------------------------------------- transfers
// Closest-point restriction / prolongation (Sec. 4.3): linear interpolation
// at each target's cp from the 2^d source nodes around it.  The nodes are
// found from the packed base node through the source brick map and masks
// (cached loads shared by neighbouring targets), not from a per-target index
// table.
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_transfer(TransferView<T> tv, const T* __restrict__ src,
                                                  T* __restrict__ dst, bool add) {
  const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= tv.n) return;
  const T sx = __ldg(tv.fr + j), sy = __ldg(tv.fr + tv.n + j);
  const T sz = DIM == 3 ? __ldg(tv.fr + 2 * tv.n + j) : T(0);
  const T wx[2] = {T(1) - sx, sx}, wy[2] = {T(1) - sy, sy}, wz[2] = {T(1) - sz, sz};
  int x = 0, y = 0, z = 0;
  if (!tv.idx) {
    const uint64_t kb = __ldg(tv.base + j);
    x = (int)(kb & 0xffffu);
    y = (int)((kb >> 16) & 0xffffu);
    z = (int)((kb >> 32) & 0xffffu);
  }
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < (DIM == 3 ? 2 : 1); ++c) {
    T accy = T(0);
#pragma unroll
    for (int bb = 0; bb < 2; ++bb) {
      const int q = 4 * c + 2 * bb;
      const int32_t i0 = tv.idx ? __ldg(tv.idx + (int64_t)q * tv.n + j) : band_index(tv.src, x, y + bb, z + c);
      const int32_t i1 = tv.idx ? __ldg(tv.idx + (int64_t)(q + 1) * tv.n + j)
                                : band_index(tv.src, x + 1, y + bb, z + c);
      const T v0 = __ldg(src + (i0 < 0 ? 0 : i0));
      const T v1 = __ldg(src + (i1 < 0 ? 0 : i1));
      accy += wy[bb] * (wx[0] * v0 + wx[1] * v1);
    }
    acc += (DIM == 3 ? wz[c] : T(1)) * accy;
  }
  dst[j] = add ? dst[j] + acc : acc;
}

// Cubic restriction / prolongation: degree-3 interpolation at the target's cp
// from the 4^d source nodes around it (base = floor - 1), tensor-product
// Lagrange weights, contracted x, then y, then z.
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_transfer3(TransferView<T> tv, const T* __restrict__ src,
                                                   T* __restrict__ dst, bool add) {
  const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= tv.n) return;
  const uint64_t kb = __ldg(tv.base + j);
  const int x = (int)(kb & 0xffffu), y = (int)((kb >> 16) & 0xffffu), z = (int)((kb >> 32) & 0xffffu);
  T wx[4], wy[4], wz[4] = {T(1), T(0), T(0), T(0)};
  cubic_w(__ldg(tv.fr + j), wx);
  cubic_w(__ldg(tv.fr + tv.n + j), wy);
  if (DIM == 3) cubic_w(__ldg(tv.fr + 2 * tv.n + j), wz);
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < (DIM == 3 ? 4 : 1); ++c) {
    T accy = T(0);
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      T accx = T(0);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int32_t i = band_index(tv.src, x + a, y + bb, z + c);
        accx += wx[a] * __ldg(src + (i < 0 ? 0 : i));
      }
      accy += wy[bb] * accx;
    }
    acc += wz[c] * accy;
  }
  dst[j] = add ? dst[j] + acc : acc;
}

template <typename T>
void launch_transfer(const TransferView<T>& tv, const T* src, T* dst, bool add, cudaStream_t st) {
  if (tv.n <= 0) return;
  if (tv.deg == 3) {
    if (tv.dim == 3) k_transfer3<T, 3><<<nblk(tv.n, 256), 256, 0, st>>>(tv, src, dst, add);
    else k_transfer3<T, 2><<<nblk(tv.n, 256), 256, 0, st>>>(tv, src, dst, add);
  } else {
    if (tv.dim == 3) k_transfer<T, 3><<<nblk(tv.n, 256), 256, 0, st>>>(tv, src, dst, add);
    else k_transfer<T, 2><<<nblk(tv.n, 256), 256, 0, st>>>(tv, src, dst, add);
  }
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

// out[0] = max|x|, out[1] = sum x^2, out[2] = 1 / max|x| (0 if max is 0);
// out[3] = the largest of the kPairSlots float slots of dmax (non-negative,
// compared as integers), which are reset to 0, or 0 without dmax.
__global__ void k_norm_final(const double* part, int nblocks, double* out, uint32_t* dmax) {
  __shared__ uint32_t dm;
  if (threadIdx.x == 0) dm = 0u;
  __syncthreads();
  if (dmax) {
    for (int i = threadIdx.x; i < kPairSlots; i += blockDim.x) {
      atomicMax(&dm, dmax[i]);
      dmax[i] = 0u;
    }
  }
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
    out[3] = (double)__uint_as_float(dm);
  }
}

void launch_norm_final(const double* part, int nblocks, double* out, cudaStream_t st, uint32_t* dmax) {
  k_norm_final<<<1, 1024, 0, st>>>(part, nblocks, out, dmax);
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

// ----------------------------------------------------------------- setup: paper form
// diag(M_p)_ii = sum_j (E_1)_ij (L_B)_ji - gamma (1 - (E_3)_ii): over the 2^d
// linear-stencil nodes j of cp(x_i), (L_B)_ji is -2d/dx^2 for j = i and
// 1/dx^2 for a Laplacian neighbour j of i; (E_3)_ii is the cubic weight of
// node i in its own stencil (0 if it lies outside).
// Variable diffusion (a != null): (L~)_ji = (a_j + a_i) / (2 dx^2) for a
// Laplacian neighbour j of i in B, (L~)_ii = -sum over the neighbours k of i
// in B of (a_i + a_k) / (2 dx^2), and the side condition is weighted by
// gamma a_i.
__device__ __forceinline__ double vard_ii(const LevelView<double>& L, const double* a, int x, int y,
                                          int z, int dim, int32_t i) {
  const int d[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  double s = 0.0;
  for (int q = 0; q < 2 * dim; ++q) {
    const int32_t k = band_index(L.bv, x + d[q][0], y + d[q][1], z + d[q][2]);
    if (k >= 0) s -= 0.5 * (a[i] + a[k]) * L.inv_h2;
  }
  return s;
}

template <int DIM>
__global__ void k_diag_Mp(LevelView<double> L, double* __restrict__ diagM, const double* __restrict__ acoef) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.nB) return;
  const uint64_t k = L.key[i];
  const int own[3] = {key_x(k), key_y(k), key_z(k)};
  const int b3[3] = {key_x(k) + key_ox(k), key_y(k) + key_oy(k), key_z(k) + key_oz(k)};
  double s[3], w3[3][4];
  for (int a = 0; a < DIM; ++a) {
    s[a] = L.fr[a * L.nplus + i];
    cubic_w(s[a], w3[a]);
  }
  double e1l = 0.0;
  for (int c = 0; c < (DIM == 3 ? 2 : 1); ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const int j[3] = {b3[0] + 1 + a, b3[1] + 1 + b, DIM == 3 ? b3[2] + 1 + c : 0};
        const double w1 = (a ? s[0] : 1.0 - s[0]) * (b ? s[1] : 1.0 - s[1]) *
                          (DIM == 3 ? (c ? s[2] : 1.0 - s[2]) : 1.0);
        int dist = 0;
        for (int q = 0; q < DIM; ++q) dist += abs(j[q] - own[q]);
        if (!acoef) {
          if (dist == 0) e1l += w1 * (-L.gamma);
          else if (dist == 1) e1l += w1 * L.inv_h2;
        } else if (dist == 0) {
          e1l += w1 * vard_ii(L, acoef, own[0], own[1], own[2], DIM, i);
        } else if (dist == 1) {
          const int32_t jj = band_index(L.bv, j[0], j[1], j[2]);
          if (jj >= 0) e1l += w1 * 0.5 * (acoef[jj] + acoef[i]) * L.inv_h2;
        }
      }
  double e3 = 1.0;
  for (int q = 0; q < DIM; ++q) {
    const int off = own[q] - b3[q];
    e3 = (off < 0 || off > 3) ? 0.0 : e3 * w3[q][off];
  }
  diagM[i] = e1l - (acoef ? L.gamma * acoef[i] : L.gamma) * (1.0 - e3);
}

void launch_diag_Mp(const LevelView<double>& L, double* diagM, const double* a, cudaStream_t st) {
  if (L.dim == 3) k_diag_Mp<3><<<nblk(L.nB, 256), 256, 0, st>>>(L, diagM, a);
  else k_diag_Mp<2><<<nblk(L.nB, 256), 256, 0, st>>>(L, diagM, a);
}

// Row i of A_p = cI - M_p = (c + gamma) I - E_1 L_B - gamma E_3.  One thread per row.
template <int DIM, typename M>
__global__ void k_assemble_Ap(LevelView<double> L, const double* cvec, double cval, M* A,
                              const double* acoef) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t n = L.nB;
  if (i >= n) return;
  M* row = A + (size_t)i * n;
  const double gi = acoef ? L.gamma * acoef[i] : L.gamma;
  row[i] += (M)((cvec ? cvec[i] : cval) + gi);
  const uint64_t k = L.key[i];
  const int b3[3] = {key_x(k) + key_ox(k), key_y(k) + key_oy(k), key_z(k) + key_oz(k)};
  double s[3] = {0.0, 0.0, 0.0}, w3[3][4] = {{1.0, 0.0, 0.0, 0.0}, {1.0, 0.0, 0.0, 0.0}, {1.0, 0.0, 0.0, 0.0}};
  for (int a = 0; a < DIM; ++a) {
    s[a] = L.fr[a * L.nplus + i];
    cubic_w(s[a], w3[a]);
  }
  for (int c = 0; c < (DIM == 3 ? 4 : 1); ++c)
    for (int b = 0; b < 4; ++b)
      for (int a = 0; a < 4; ++a) {
        const int32_t j = band_index(L.bv, b3[0] + a, b3[1] + b, DIM == 3 ? b3[2] + c : 0);
        if (j >= 0) row[j] -= (M)(gi * w3[0][a] * w3[1][b] * w3[2][c]);
      }
  const int d[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  for (int c = 0; c < (DIM == 3 ? 2 : 1); ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const int jx = b3[0] + 1 + a, jy = b3[1] + 1 + b, jz = DIM == 3 ? b3[2] + 1 + c : 0;
        const double w1 = (a ? s[0] : 1.0 - s[0]) * (b ? s[1] : 1.0 - s[1]) *
                          (DIM == 3 ? (c ? s[2] : 1.0 - s[2]) : 1.0);
        const int32_t jj = band_index(L.bv, jx, jy, jz);
        if (!acoef) {
          if (jj >= 0) row[jj] -= (M)(w1 * -L.gamma);
          for (int q = 0; q < 2 * DIM; ++q) {
            const int32_t kk = band_index(L.bv, jx + d[q][0], jy + d[q][1], jz + d[q][2]);
            if (kk >= 0) row[kk] -= (M)(w1 * L.inv_h2);
          }
        } else if (jj >= 0) {  // row jj of L~ (its own band-restricted neighbours)
          for (int q = 0; q < 2 * DIM; ++q) {
            const int32_t kk = band_index(L.bv, jx + d[q][0], jy + d[q][1], jz + d[q][2]);
            if (kk < 0) continue;
            const double face = 0.5 * (acoef[jj] + acoef[kk]) * L.inv_h2;
            row[kk] -= (M)(w1 * face);
            row[jj] += (M)(w1 * face);
          }
        }
      }
}

template <typename M>
void launch_assemble_Ap(const LevelView<double>& L, const double* cvec, double cval, M* A,
                        const double* a, cudaStream_t st) {
  if (L.dim == 3) k_assemble_Ap<3, M><<<nblk(L.nB, 128), 128, 0, st>>>(L, cvec, cval, A, a);
  else k_assemble_Ap<2, M><<<nblk(L.nB, 128), 128, 0, st>>>(L, cvec, cval, A, a);
}
template void launch_assemble_Ap<double>(const LevelView<double>&, const double*, double, double*,
                                         const double*, cudaStream_t);
template void launch_assemble_Ap<float>(const LevelView<double>&, const double*, double, float*,
                                        const double*, cudaStream_t);

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
  template void launch_lap_band<T>(const LevelView<T>&, const T*, T*, cudaStream_t);            \
  template void launch_lap_rel<T>(const LevelView<T>&, LapMode, const T*, const T*, const T*,   \
                                  const T*, const T*, T, const T*, T*, T*, double*, cudaStream_t); \
  template void launch_paper<T>(const LevelView<T>&, LapMode, const T*, const T*, const T*,     \
                                const T*, const T*, T, const T*, T*, T*, double*, const T*,      \
                                cudaStream_t);                                                   \
  template void launch_lap_vard<T>(const LevelView<T>&, const T*, const T*, T*, cudaStream_t);  \
  template void launch_norm_partials<T>(const T*, int64_t, double*, cudaStream_t);               \
  template void launch_cast_to_f64<T>(const T*, double*, int64_t, cudaStream_t);                 \
  template void launch_cast_from_f64<T>(const double*, T*, int64_t, cudaStream_t);               \
  template void launch_coarse_gemv<T>(const double*, const T* const*, T* const*, int, int32_t, \
                                      cudaStream_t);
CPM_INST(double)
CPM_INST(float)

}  // namespace cpm
