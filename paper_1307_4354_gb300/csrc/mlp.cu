// Learned smoother: a per-band-point network (31 -> 64 -> 64 -> 1) that
// replaces the first pre-smoothing Jacobi sweep (Eq. 4.1) of the finest
// level, with plain weighted Jacobi as its fallback and judge.  The paper has
// no learned component.
//
// Features of band point i: the residual at the 3x3x3 grid neighbourhood of
// x_i (0 off the band) divided by s_i = max |r| over it, (x_i - cp(x_i))/dx,
// and dx^2 M_ii.  Correction du_i = s_i dx^2 y_i, y = w3 . relu(W2^T
// relu(W1^T x + b1) + b2) + b3.
//
// Forward: BF16 weights and features, FP32 accumulation on the tensor cores
// (warp-level mma.sync m16n8k16, one warp per 16 points).  Training: the loss
// of a residual field r is ||r - A du||^2 / ||r||^2; its gradient with
// respect to du is -2 A^T (r - A du) / ||r||^2 (A^T through a transposed
// neighbour gather and a transposed extension scatter over the extension
// tiles), back-propagated through the network on the tensor cores (the three
// contractions as BF16 mma.sync with FP32 accumulation, bias gradients in
// FP32), reduced per CTA and summed in a fixed order; Adam on FP32 master
// weights.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "mlp.cuh"

namespace cpm {

static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ----------------------------------------------------------------- static data
// nbr27[q * nB + i]: band index of x_i + (a, b, c) dx, q = (a+1) + 3(b+1) + 9(c+1),
// or -1; stat[a * nB + i]: (x_i - cp_i)/dx for a < 3, dx^2 M_ii for a = 3.
__global__ void k_mlp_static(BrickView v, const uint64_t* key, const double* cp, int64_t nplus,
                             int32_t nB, double lo, double dx, const double* diagM, int32_t* nbr27,
                             float* stat) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nB) return;
  const uint64_t k = key[i];
  const int x = key_x(k), y = key_y(k), z = key_z(k);
  int q = 0;
  for (int c = -1; c <= 1; ++c)
    for (int b = -1; b <= 1; ++b)
      for (int a = -1; a <= 1; ++a, ++q) nbr27[(int64_t)q * nB + i] = band_index(v, x + a, y + b, z + c);
  const int own[3] = {x, y, z};
  for (int a = 0; a < 3; ++a) {
    const double xa = lo + own[a] * dx;
    stat[(int64_t)a * nB + i] = (float)((xa - cp[a * nplus + i]) / dx);
  }
  stat[(int64_t)3 * nB + i] = (float)(dx * dx * diagM[i]);
}

// ----------------------------------------------------------------- forward
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kFwdWarps = 8;
constexpr int kW1S = 40;  // padded row (k) stride of the transposed W1 in shared memory (bf16)
constexpr int kW2S = 72;  // same for W2
constexpr int kXS = 40;   // padded row stride of the per-warp feature tile

struct MlpFwdArgs {
  const float* params;   // FP32 master parameters (layout in mlp.cuh)
  const float* r;        // residual on B (FP32)
  const int32_t* nbr27;
  const float* stat;
  int32_t nB;
  float dx2;
  float* du;             // out: correction (mode 0) ...
  float* u;              // ... or u += correction (mode 1)
  // training outputs (mode 0, may be null)
  __nv_bfloat16* Xs;     // nB x 32
  __nv_bfloat16* H1;     // nB x 64
  __nv_bfloat16* H2;     // nB x 64
  float* S;              // nB
};

template <int MODE>
__global__ void __launch_bounds__(kFwdWarps * 32) k_mlp_forward(MlpFwdArgs A) {
  __shared__ __align__(16) __nv_bfloat16 w1t[64 * kW1S];  // w1t[n][k] = W1[k][n]
  __shared__ __align__(16) __nv_bfloat16 w2t[64 * kW2S];
  __shared__ float bias1[64], bias2[64], w3s[64];
  __shared__ __align__(16) __nv_bfloat16 xs[kFwdWarps][16 * kXS];
  __shared__ float ss[kFwdWarps][16];
  for (int q = threadIdx.x; q < 64 * 32; q += blockDim.x) {
    const int n = q & 63, k = q >> 6;
    w1t[n * kW1S + k] = __float2bfloat16_rn(A.params[kOffW1 + k * 64 + n]);
  }
  for (int q = threadIdx.x; q < 64 * 64; q += blockDim.x) {
    const int n = q & 63, k = q >> 6;
    w2t[n * kW2S + k] = __float2bfloat16_rn(A.params[kOffW2 + k * 64 + n]);
  }
  for (int q = threadIdx.x; q < 64; q += blockDim.x) {
    bias1[q] = A.params[kOffB1 + q];
    bias2[q] = A.params[kOffB2 + q];
    w3s[q] = A.params[kOffW3 + q];
  }
  __syncthreads();
  const float b3 = A.params[kOffB3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  __nv_bfloat16* xw = xs[warp];
  const int64_t ngroups = ((int64_t)A.nB + 15) / 16;
  for (int64_t grp = (int64_t)blockIdx.x * kFwdWarps + warp; grp < ngroups;
       grp += (int64_t)gridDim.x * kFwdWarps) {
    const int64_t p0 = grp * 16;
    // features: lanes 0..15 one point each
    if (lane < 16) {
      const int64_t p = p0 + lane;
      float f[32];
      float smax = 0.f;
      if (p < A.nB) {
#pragma unroll
        for (int q = 0; q < 27; ++q) {
          const int32_t j = __ldg(A.nbr27 + (int64_t)q * A.nB + p);
          f[q] = j >= 0 ? __ldg(A.r + j) : 0.f;
          smax = fmaxf(smax, fabsf(f[q]));
        }
        const float inv = smax > 0.f ? 1.f / smax : 0.f;
#pragma unroll
        for (int q = 0; q < 27; ++q) f[q] *= inv;
#pragma unroll
        for (int q = 0; q < 4; ++q) f[27 + q] = __ldg(A.stat + (int64_t)q * A.nB + p);
      } else {
#pragma unroll
        for (int q = 0; q < 31; ++q) f[q] = 0.f;
      }
      f[31] = 0.f;
#pragma unroll
      for (int q = 0; q < 32; q += 2)
        *reinterpret_cast<uint32_t*>(&xw[lane * kXS + q]) = pack_bf16(f[q], f[q + 1]);
      ss[warp][lane] = smax;
      if (MODE == 0 && A.Xs && p < A.nB) {
        uint4* dst = reinterpret_cast<uint4*>(A.Xs + p * 32);
        const uint4* src = reinterpret_cast<const uint4*>(&xw[lane * kXS]);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = src[q];
      }
    }
    __syncwarp();
    // layer 1: [16 x 32] x [32 x 64]
    uint32_t a[2][4];
#pragma unroll
    for (int kc = 0; kc < 2; ++kc) {
      a[kc][0] = *reinterpret_cast<const uint32_t*>(&xw[g * kXS + kc * 16 + 2 * t]);
      a[kc][1] = *reinterpret_cast<const uint32_t*>(&xw[(g + 8) * kXS + kc * 16 + 2 * t]);
      a[kc][2] = *reinterpret_cast<const uint32_t*>(&xw[g * kXS + kc * 16 + 8 + 2 * t]);
      a[kc][3] = *reinterpret_cast<const uint32_t*>(&xw[(g + 8) * kXS + kc * 16 + 8 + 2 * t]);
    }
    float h[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int n = nt * 8 + 2 * t;
      h[nt][0] = h[nt][2] = bias1[n];
      h[nt][1] = h[nt][3] = bias1[n + 1];
#pragma unroll
      for (int kc = 0; kc < 2; ++kc) {
        const __nv_bfloat16* wb = &w1t[(nt * 8 + g) * kW1S + kc * 16 + 2 * t];
        mma_bf16(h[nt], a[kc], *reinterpret_cast<const uint32_t*>(wb),
                 *reinterpret_cast<const uint32_t*>(wb + 8));
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) h[nt][e] = fmaxf(h[nt][e], 0.f);
    }
    // relu(h1) as the A operand of layer 2 (C tiles 2j, 2j+1 form k-chunk j)
    uint32_t a2[4][4];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      a2[kc][0] = pack_bf16(h[2 * kc][0], h[2 * kc][1]);
      a2[kc][1] = pack_bf16(h[2 * kc][2], h[2 * kc][3]);
      a2[kc][2] = pack_bf16(h[2 * kc + 1][0], h[2 * kc + 1][1]);
      a2[kc][3] = pack_bf16(h[2 * kc + 1][2], h[2 * kc + 1][3]);
    }
    if (MODE == 0 && A.H1) {
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        const int64_t r0 = p0 + g, r1 = p0 + g + 8;
        const int c0 = kc * 16 + 2 * t;
        if (r0 < A.nB) {
          *reinterpret_cast<uint32_t*>(A.H1 + r0 * 64 + c0) = a2[kc][0];
          *reinterpret_cast<uint32_t*>(A.H1 + r0 * 64 + c0 + 8) = a2[kc][2];
        }
        if (r1 < A.nB) {
          *reinterpret_cast<uint32_t*>(A.H1 + r1 * 64 + c0) = a2[kc][1];
          *reinterpret_cast<uint32_t*>(A.H1 + r1 * 64 + c0 + 8) = a2[kc][3];
        }
      }
    }
    // layer 2: [16 x 64] x [64 x 64], then relu and the dot with w3
    float y0 = 0.f, y1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int n = nt * 8 + 2 * t;
      float c[4] = {bias2[n], bias2[n + 1], bias2[n], bias2[n + 1]};
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        const __nv_bfloat16* wb = &w2t[(nt * 8 + g) * kW2S + kc * 16 + 2 * t];
        mma_bf16(c, a2[kc], *reinterpret_cast<const uint32_t*>(wb),
                 *reinterpret_cast<const uint32_t*>(wb + 8));
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) c[e] = fmaxf(c[e], 0.f);
      if (MODE == 0 && A.H2) {
        const int64_t r0 = p0 + g, r1 = p0 + g + 8;
        if (r0 < A.nB) *reinterpret_cast<uint32_t*>(A.H2 + r0 * 64 + n) = pack_bf16(c[0], c[1]);
        if (r1 < A.nB) *reinterpret_cast<uint32_t*>(A.H2 + r1 * 64 + n) = pack_bf16(c[2], c[3]);
      }
      y0 += c[0] * w3s[n] + c[1] * w3s[n + 1];
      y1 += c[2] * w3s[n] + c[3] * w3s[n + 1];
    }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
    if (t == 0) {
      const int64_t r0 = p0 + g, r1 = p0 + g + 8;
      if (r0 < A.nB) {
        const float d = ss[warp][g] * A.dx2 * (y0 + b3);
        if (MODE == 1) A.u[r0] += d; else A.du[r0] = d;
        if (MODE == 0 && A.S) A.S[r0] = ss[warp][g];
      }
      if (r1 < A.nB) {
        const float d = ss[warp][g + 8] * A.dx2 * (y1 + b3);
        if (MODE == 1) A.u[r1] += d; else A.du[r1] = d;
        if (MODE == 0 && A.S) A.S[r1] = ss[warp][g + 8];
      }
    }
    __syncwarp();
  }
}

// ----------------------------------------------------------------- backward
// The backward pass runs on a fixed grid of kBwdCtas CTAs, each writing one
// partial gradient (kBwdCtas x 25 KB whatever the band size).
constexpr int kBwdCtas = 2 * 152;

// Tensor-core backward.  A CTA of 4 warps loops over groups of 16 points;
// per group the three contractions run as BF16 mma.sync.m16n8k16 with FP32
// accumulation:
//   dz1 = (dz2 W2^T) [h1 > 0]    M = 16 points, N = 64, K = 64  (warp w: dz1 columns 16w..16w+15)
//   dW2 += H1^T dz2              M = 64, N = 64, K = 16 points (warp w: rows 16w..16w+15)
//   dW1 += X^T dz1               M = 32, N = 64, K = 16 points (warp w: columns 16w..16w+15)
// with dz2 = dy w3 [h2 > 0].  The operands sit in shared memory transposed so
// that the K index (the points) is contiguous; the dW accumulators stay in
// registers across all the CTA's groups; bias gradients are FP32 sums by 65
// threads.  Each CTA writes one partial gradient, summed by k_grad_reduce.
constexpr int kTcWarps = 4;
constexpr int kTcS = 24;   // row stride (bf16) of the transposed 16-point tiles
constexpr int kTcW2 = 72;  // row stride (bf16) of W2 in shared memory

__global__ void __launch_bounds__(kTcWarps * 32) k_mlp_backward_tc(const float* params, const float* dy,
                                                                   const __nv_bfloat16* Xs,
                                                                   const __nv_bfloat16* H1,
                                                                   const __nv_bfloat16* H2, int32_t nB,
                                                                   float* part) {
  __shared__ __align__(16) __nv_bfloat16 w2s[64 * kTcW2];   // w2s[k][j] = W2[k][j]
  __shared__ __align__(16) __nv_bfloat16 xT[32 * kTcS];     // xT[f][p]
  __shared__ __align__(16) __nv_bfloat16 h1T[64 * kTcS];    // h1T[k][p]
  __shared__ __align__(16) __nv_bfloat16 dz2T[64 * kTcS];   // dz2T[j][p]
  __shared__ __align__(16) __nv_bfloat16 dz1T[64 * kTcS];   // dz1T[k][p]
  __shared__ __align__(16) __nv_bfloat16 dz2r[16 * kTcW2];  // dz2r[p][j] (A operand of dz1)
  __shared__ float h1f[16][65], h2f[16][65], dz1f[16][65], w3s[64], dys[16];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  for (int q = tid; q < 64 * 64; q += blockDim.x)
    w2s[(q >> 6) * kTcW2 + (q & 63)] = __float2bfloat16_rn(params[kOffW2 + q]);
  for (int q = tid; q < 64; q += blockDim.x) w3s[q] = params[kOffW3 + q];
  float acc2[8][4], acc1[2][2][4];  // dW2 rows 16w.., dW1 (m-tile, n-tile of the warp)
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc2[a][e] = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc1[a][b][e] = 0.f;
  float sb1 = 0.f, sb2 = 0.f, sw3 = 0.f, sb3 = 0.f;  // bias sums of threads 0..64
  const int64_t ngroups = ((int64_t)nB + 15) / 16;
  __syncthreads();
  for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int64_t p0 = grp * 16;
    // operands of this group
    for (int q = tid; q < 16 * 64; q += blockDim.x) {
      const int p = q >> 6, j = q & 63;
      const int64_t gp = p0 + p;
      const bool ok = gp < nB;
      const float h1v = ok ? __bfloat162float(H1[gp * 64 + j]) : 0.f;
      const float h2v = ok ? __bfloat162float(H2[gp * 64 + j]) : 0.f;
      const float dyv = ok ? dy[gp] : 0.f;
      const float d2 = h2v > 0.f ? dyv * w3s[j] : 0.f;
      h1f[p][j] = h1v;
      h2f[p][j] = h2v;
      h1T[j * kTcS + p] = __float2bfloat16_rn(h1v);
      dz2T[j * kTcS + p] = __float2bfloat16_rn(d2);
      dz2r[p * kTcW2 + j] = __float2bfloat16_rn(d2);
      if (j < 32) xT[j * kTcS + p] = ok ? Xs[gp * 32 + j] : __float2bfloat16_rn(0.f);
      if (j == 0) dys[p] = dyv;
    }
    __syncthreads();
    // dz1 columns 16 warp .. 16 warp + 15: A = dz2 (points x j), B[j][k] = W2[k][j]
    {
      float c[2][4];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) c[nt][e] = 0.f;
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        uint32_t a[4];
        a[0] = *reinterpret_cast<const uint32_t*>(&dz2r[g * kTcW2 + kc * 16 + 2 * t]);
        a[1] = *reinterpret_cast<const uint32_t*>(&dz2r[(g + 8) * kTcW2 + kc * 16 + 2 * t]);
        a[2] = *reinterpret_cast<const uint32_t*>(&dz2r[g * kTcW2 + kc * 16 + 8 + 2 * t]);
        a[3] = *reinterpret_cast<const uint32_t*>(&dz2r[(g + 8) * kTcW2 + kc * 16 + 8 + 2 * t]);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int n = 16 * warp + 8 * nt + g;
          const __nv_bfloat16* wb = &w2s[n * kTcW2 + kc * 16 + 2 * t];
          mma_bf16(c[nt], a, *reinterpret_cast<const uint32_t*>(wb),
                   *reinterpret_cast<const uint32_t*>(wb + 8));
        }
      }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int k0 = 16 * warp + 8 * nt + 2 * t;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int p = g + (e >> 1) * 8, k = k0 + (e & 1);
          const float v = h1f[p][k] > 0.f ? c[nt][e] : 0.f;
          dz1f[p][k] = v;
          dz1T[k * kTcS + p] = __float2bfloat16_rn(v);
        }
      }
    }
    __syncthreads();
    // dW2 rows 16 warp ..: A[k][p] = h1T, B[p][j] = dz2T (as [j][p])
    {
      uint32_t a[4];
      const int m0 = 16 * warp;
      a[0] = *reinterpret_cast<const uint32_t*>(&h1T[(m0 + g) * kTcS + 2 * t]);
      a[1] = *reinterpret_cast<const uint32_t*>(&h1T[(m0 + g + 8) * kTcS + 2 * t]);
      a[2] = *reinterpret_cast<const uint32_t*>(&h1T[(m0 + g) * kTcS + 8 + 2 * t]);
      a[3] = *reinterpret_cast<const uint32_t*>(&h1T[(m0 + g + 8) * kTcS + 8 + 2 * t]);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const __nv_bfloat16* bb = &dz2T[(nt * 8 + g) * kTcS + 2 * t];
        mma_bf16(acc2[nt], a, *reinterpret_cast<const uint32_t*>(bb),
                 *reinterpret_cast<const uint32_t*>(bb + 8));
      }
    }
    // dW1 columns 16 warp ..: A[f][p] = xT, B[p][k] = dz1T (as [k][p])
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      uint32_t a[4];
      a[0] = *reinterpret_cast<const uint32_t*>(&xT[(16 * mt + g) * kTcS + 2 * t]);
      a[1] = *reinterpret_cast<const uint32_t*>(&xT[(16 * mt + g + 8) * kTcS + 2 * t]);
      a[2] = *reinterpret_cast<const uint32_t*>(&xT[(16 * mt + g) * kTcS + 8 + 2 * t]);
      a[3] = *reinterpret_cast<const uint32_t*>(&xT[(16 * mt + g + 8) * kTcS + 8 + 2 * t]);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const __nv_bfloat16* bb = &dz1T[(16 * warp + 8 * nt + g) * kTcS + 2 * t];
        mma_bf16(acc1[mt][nt], a, *reinterpret_cast<const uint32_t*>(bb),
                 *reinterpret_cast<const uint32_t*>(bb + 8));
      }
    }
    // bias gradients (FP32)
    if (tid < 64) {
      for (int p = 0; p < 16; ++p) {
        sb1 += dz1f[p][tid];
        const float d2 = h2f[p][tid] > 0.f ? dys[p] * w3s[tid] : 0.f;
        sb2 += d2;
        sw3 += dys[p] * h2f[p][tid];
      }
    } else if (tid == 64) {
      for (int p = 0; p < 16; ++p) sb3 += dys[p];
    }
    __syncthreads();
  }
  float* out = part + (int64_t)blockIdx.x * kNParams;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = 16 * warp + g + (e >> 1) * 8, j = nt * 8 + 2 * t + (e & 1);
      out[kOffW2 + k * 64 + j] = acc2[nt][e];
    }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int f = 16 * mt + g + (e >> 1) * 8, k = 16 * warp + 8 * nt + 2 * t + (e & 1);
        out[kOffW1 + f * 64 + k] = acc1[mt][nt][e];
      }
  if (tid < 64) {
    out[kOffB1 + tid] = sb1;
    out[kOffB2 + tid] = sb2;
    out[kOffW3 + tid] = sw3;
  } else if (tid == 64) {
    out[kOffB3] = sb3;
  }
}

// grad[q] = sum over CTAs of part[c][q] (fixed order).
__global__ void k_grad_reduce(const float* part, int nparts, float* grad) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= kNParams) return;
  float s = 0.f;
  for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * kNParams + q];
  grad[q] = s;
}

// Adam (Kingma & Ba) on the FP32 master parameters.
__global__ void k_adam(float* params, const float* grad, float* m, float* v, float lr, float b1,
                       float b2, float eps, float bc1, float bc2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= kNParams) return;
  if (q >= kOffW1 + 31 * 64 && q < kOffW1 + 32 * 64) return;  // zero-feature row stays 0
  const float g = grad[q];
  const float mq = b1 * m[q] + (1.f - b1) * g;
  const float vq = b2 * v[q] + (1.f - b2) * g * g;
  m[q] = mq;
  v[q] = vq;
  params[q] -= lr * (mq / bc1) / (sqrtf(vq / bc2) + eps);
}

// ----------------------------------------------------------------- A^T
// t[k] = sum of z_i over the grid neighbours i of k (k in B+) that are in B.
__global__ void k_nbr_transpose(BrickView v, const uint64_t* key, int64_t nplus, int dim,
                                const float* z, float* t) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nplus) return;
  const uint64_t kk = key[k];
  const int x = key_x(kk), y = key_y(kk), zc = key_z(kk);
  const int d[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  float s = 0.f;
  for (int q = 0; q < 2 * dim; ++q) {
    const int32_t i = band_index(v, x + d[q][0], y + d[q][1], zc + d[q][2]);
    if (i >= 0) s += z[i];
  }
  t[k] = s;
}

// out[j] += sum_k E_{kj} t[k]: each extension tile scatters its points'
// weighted values into its shared-memory box, then adds the box to out.
__global__ void __launch_bounds__(64) k_extend_transpose(LevelView<float> L, const float* t,
                                                         float* out) {
  __shared__ float box[7 * 7 * 7];
  __shared__ uint64_t sm_mask[8];
  __shared__ int32_t sm_start[8];
  const int32_t tile = blockIdx.x;
  for (int q = threadIdx.x; q < 343; q += blockDim.x) box[q] = 0.f;
  if (threadIdx.x < 8) {
    sm_mask[threadIdx.x] = L.tile_mask[8 * (int64_t)tile + threadIdx.x];
    sm_start[threadIdx.x] = L.tile_bstart[8 * (int64_t)tile + threadIdx.x];
  }
  __syncthreads();
  const int32_t beg = L.tile_start[tile], end = L.tile_start[tile + 1];
  const int64_t np = L.nplus;
  for (int32_t k = beg + threadIdx.x; k < end; k += blockDim.x) {
    const uint32_t rec = L.erec[k];
    const int lx = rec & 3, ly = (rec >> 2) & 3, lz = (rec >> 4) & 3;
    float wx[4], wy[4], wz[4];
    const float s3[3] = {L.efr[k], L.efr[np + k], L.efr[2 * np + k]};
    float* ws[3] = {wx, wy, wz};
    for (int a = 0; a < 3; ++a) {
      const float s = s3[a], sm1 = s - 1.f, sm2 = s - 2.f, sp1 = s + 1.f;
      const float p = s * sm1, q = sp1 * sm2;
      ws[a][0] = (p * sm2) * (-1.f / 6.f);
      ws[a][1] = (q * sm1) * 0.5f;
      ws[a][2] = (q * s) * -0.5f;
      ws[a][3] = (p * sp1) * (1.f / 6.f);
    }
    const float tv = t[rec >> 6];
    for (int c = 0; c < 4; ++c)
      for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a)
          atomicAdd(&box[((lz + c) * 7 + ly + b) * 7 + lx + a], wx[a] * wy[b] * wz[c] * tv);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 343; q += blockDim.x) {
    const float val = box[q];
    if (val == 0.f) continue;
    const int x = q % 7, y = (q / 7) % 7, z = q / 49;
    const int j = (x >> 2) | ((y >> 2) << 1) | ((z >> 2) << 2);
    const uint64_t bit = 1ull << ((x & 3) | ((y & 3) << 2) | ((z & 3) << 4));
    const uint64_t m = sm_mask[j];
    if (m & bit) atomicAdd(out + sm_start[j] + __popcll(m & (bit - 1)), val);
  }
}

// dy = -2 (A^T z) s dx^2 / ||r||^2 with A^T z = (c + gamma) z - ext^T / dx^2.
__global__ void k_mlp_dy(const float* z, const float* et, const float* cvec, float cval, float gamma,
                         float inv_h2, const float* S, float dx2, const double* nr2, int32_t nB,
                         float* dy) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nB) return;
  const float c = cvec ? cvec[i] : cval;
  const float atz = (c + gamma) * z[i] - et[i] * inv_h2;
  dy[i] = (float)(-2.0 / nr2[0]) * atz * S[i] * dx2;
}

// z = r - (c du - M du) given Mdu; partial sums of z^2 and r^2 per block.
__global__ void k_mlp_resid(const float* r, const float* du, const float* Mdu, const float* cvec,
                            float cval, int32_t nB, float* z, double* part) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  double zz = 0.0, rr = 0.0;
  if (i < nB) {
    const float c = cvec ? cvec[i] : cval;
    const float zi = r[i] - (c * du[i] - Mdu[i]);
    z[i] = zi;
    zz = (double)zi * zi;
    rr = (double)r[i] * r[i];
  }
  __shared__ double s1[8], s2[8];
  for (int o = 16; o > 0; o >>= 1) {
    zz += __shfl_xor_sync(0xffffffffu, zz, o);
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
  }
  if ((threadIdx.x & 31) == 0) { s1[threadIdx.x >> 5] = zz; s2[threadIdx.x >> 5] = rr; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += s1[q]; b += s2[q]; }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

__global__ void k_mlp_loss_final(const double* part, int nblocks, double* out) {
  if (threadIdx.x != 0) return;
  double a = 0, b = 0;
  for (int q = 0; q < nblocks; ++q) { a += part[2 * q]; b += part[2 * q + 1]; }
  out[0] = a;  // ||z||^2
  out[1] = b;  // ||r||^2
}

// ----------------------------------------------------------------- host side
void MlpLevelData::build(const Level& lev, const double* diagM, cudaStream_t st) {
  nB = lev.nB;
  nbr27.alloc((size_t)27 * nB);
  stat.alloc((size_t)4 * nB);
  k_mlp_static<<<nblk(nB, 256), 256, 0, st>>>(lev.view(), lev.key.get(), lev.cp.get(), lev.nplus(), nB,
                                              lev.lo, lev.dx, diagM, nbr27.get(), stat.get());
  CPM_CUDA_TRY(cudaGetLastError());
}

void mlp_forward(const float* params, const MlpLevelData& D, const float* r, float dx2, float* du,
                 float* u_add, const MlpTrainBuffers* tb, cudaStream_t st) {
  MlpFwdArgs a{};
  a.params = params;
  a.r = r;
  a.nbr27 = D.nbr27.get();
  a.stat = D.stat.get();
  a.nB = D.nB;
  a.dx2 = dx2;
  a.du = du;
  a.u = u_add;
  if (tb) {
    a.Xs = tb->Xs.get();
    a.H1 = tb->H1.get();
    a.H2 = tb->H2.get();
    a.S = tb->S.get();
  }
  const int64_t groups = ((int64_t)D.nB + 15) / 16;
  const unsigned grid = (unsigned)std::min<int64_t>((groups + kFwdWarps - 1) / kFwdWarps, 152 * 8);
  if (u_add)
    k_mlp_forward<1><<<grid, kFwdWarps * 32, 0, st>>>(a);
  else
    k_mlp_forward<0><<<grid, kFwdWarps * 32, 0, st>>>(a);
  count_launch();
}

void MlpTrainBuffers::ensure(int32_t nB, int64_t nplus) {
  nparts = kBwdCtas;
  if (nB <= n && nplus <= np) return;  // capacity suffices
  n = nB;
  np = nplus;
  Xs.alloc((size_t)nB * 32);
  H1.alloc((size_t)nB * 64);
  H2.alloc((size_t)nB * 64);
  S.alloc(nB);
  du.alloc(nB);
  Mdu.alloc(nB);
  z.alloc(nB);
  w.alloc(nplus);
  t.alloc(nplus);
  et.alloc(nB);
  dy.alloc(nB);
  nparts = kBwdCtas;
  part.alloc((size_t)nparts * kNParams);
  lpart.alloc(2 * (size_t)((nB + 255) / 256));
  loss.alloc(2);
  grad.alloc(kNParams);
}

// Loss and gradient of one residual field (FP32 on level 0 of the view L).
void mlp_loss_grad(const float* params, const MlpLevelData& D, const LevelView<float>& L,
                   const float* cvec, float cval, const float* r, MlpTrainBuffers& tb,
                   cudaStream_t st) {
  const int32_t nB = L.nB;
  const float dx2 = 1.f / L.inv_h2;
  tb.ensure(nB, L.nplus);
  mlp_forward(params, D, r, dx2, tb.du.get(), nullptr, &tb, st);
  // M du (extension over B+ then the stencil)
  launch_extend<float>(L, tb.du.get(), tb.w.get(), (int32_t)L.nplus, st);
  launch_lap<float>(L, LAP_APPLY, tb.du.get(), tb.w.get(), nullptr, nullptr, 0.f, nullptr, 0.f,
                    tb.Mdu.get(), nullptr, nullptr, 0, st);
  const int nb256 = (int)((nB + 255) / 256);
  k_mlp_resid<<<nb256, 256, 0, st>>>(r, tb.du.get(), tb.Mdu.get(), cvec, cval, nB, tb.z.get(),
                                      tb.lpart.get());
  k_mlp_loss_final<<<1, 32, 0, st>>>(tb.lpart.get(), nb256, tb.loss.get());
  // A^T z = (c + gamma) z - E^T (N^T z) / dx^2
  k_nbr_transpose<<<nblk(L.nplus, 256), 256, 0, st>>>(L.bv, L.key, L.nplus, L.dim, tb.z.get(),
                                                       tb.t.get());
  CPM_CUDA_TRY(cudaMemsetAsync(tb.et.get(), 0, sizeof(float) * nB, st));
  k_extend_transpose<<<L.ntiles, 64, 0, st>>>(L, tb.t.get(), tb.et.get());
  k_mlp_dy<<<nb256, 256, 0, st>>>(tb.z.get(), tb.et.get(), cvec, cval, L.gamma, L.inv_h2, tb.S.get(),
                                   dx2, tb.loss.get() + 1, nB, tb.dy.get());
  k_mlp_backward_tc<<<tb.nparts, kTcWarps * 32, 0, st>>>(params, tb.dy.get(), tb.Xs.get(), tb.H1.get(),
                                                         tb.H2.get(), nB, tb.part.get());
  k_grad_reduce<<<nblk(kNParams, 256), 256, 0, st>>>(tb.part.get(), tb.nparts, tb.grad.get());
  count_launch(9);
  CPM_CUDA_TRY(cudaGetLastError());
}

void mlp_adam(float* params, const float* grad, float* m, float* v, int64_t step, float lr,
              cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - std::pow(b1, (float)step), bc2 = 1.f - std::pow(b2, (float)step);
  k_adam<<<nblk(kNParams, 256), 256, 0, st>>>(params, grad, m, v, lr, b1, b2, 1e-8f, bc1, bc2);
  count_launch();
}

}  // namespace cpm
