// Device operators of one level (extension E, the operator M, Jacobi,
// residuals, closest-point transfers, norms) and their launchers.
#pragma once

#include "cpm_internal.cuh"

namespace cpm {

// Plain-pointer view of one level for precision T.
template <typename T>
struct LevelView {
  BrickView bv;
  const uint64_t* key;  // B+ keys
  const T* fr;          // d x nplus fractions (SoA, band order)
  int64_t nplus;
  int32_t nB;
  int dim;
  T inv_h2;   // 1/dx^2
  T gamma;    // 2d/dx^2
  // extension tiles (ext.cu)
  const uint32_t* tile_brick;
  const uint32_t* tile_box;
  const uint64_t* tile_mask;
  const int32_t* tile_bstart;
  const int32_t* tile_start;
  const int32_t* tile_mid;  // per tile: end of its points of B
  const uint32_t* erec;
  const float* efr;     // E-order FP32 fractions
  const double* ew64;   // E-order FP64 weights
  const float2* ewp;    // E-order weights as FP32 pairs (finest level, pair residual)
  int32_t ntiles;
  int ext_variant;            // FP32 extension work decomposition (ExtVariant)
  const uint32_t* echunk;     // chunk records (ext.cu)
  const int32_t* tile_cstart; // ntiles + 1 chunk offsets
  const int32_t* tile_cmid;   // per tile: end of its chunks of B
  const int32_t* nbr;   // 2d x nB neighbour indices into B+
};

// Transfer records: for each target point, the base node of its linear
// (2^d) or cubic (4^d) stencil in the source grid (packed x | y << 16 | z << 32)
// and the fractions (SoA, d x n).  The stencil nodes are located through the source
// level's brick tables.
template <typename T>
struct TransferView {
  const uint64_t* base;    // n packed base nodes in the source grid
  const T* fr;
  BrickView src;           // brick tables of the source level
  int32_t n;               // number of target points
  int dim;
  int deg;                 // 1: linear (2^d nodes from base), 3: cubic (4^d nodes)
  const int32_t* idx;      // linear: 2^d x n source band indices, or null (brick lookups)
};

enum LapMode { LAP_APPLY = 0, LAP_RESID = 1, LAP_JACOBI = 2, LAP_RESID_REL = 3,
               LAP_JAC_RED = 4, LAP_JAC_BLACK = 5,  // Jacobi update of one colour only
               LAP_JAC_REL = 6 };                    // Jacobi update from the relative extension
// Red (0) / black (1): parity of the sum of the grid coordinates.  Bricks start
// at multiples of 4, so the parity of the local coordinates inside a brick is
// that of the global ones.
__host__ __device__ inline int node_colour_local(int l) { return ((l & 3) + ((l >> 2) & 3) + (l >> 4)) & 1; }

enum ExtVariant { EXT_TILES = 0, EXT_PIPE = 1, EXT_CHUNKS = 2 };
// Time the three FP32 extension variants on a level (over B+, one warm-up and
// three timed launches each, CUDA events on st) and return the fastest; ms[v]
// gets each variant's time.  u, w: device scratch of nB and nB + nG floats.
int tune_extension(const LevelView<float>& L, const float* u, float* w, cudaStream_t st, float ms[3]);

// w = E u on the first npts points of B+ (npts = nB or nB + nG).
template <typename T>
void launch_extend(const LevelView<T>& L, const T* u, T* w, int32_t npts, cudaStream_t st);

// Extension over B+ in relative form: delta_j = (E u)_j - ref_j with
// ref_j = u at a reference node of j's tile (see k_extend_tiles).
template <typename T>
void launch_extend_rel(const LevelView<T>& L, const T* u, T* delta, T* refv, cudaStream_t st);
// RESID_REL / JAC_REL passes from delta and refv (launch_lap with refv).
template <typename T>
void launch_lap_rel(const LevelView<T>& L, LapMode mode, const T* u, const T* delta, const T* refv,
                    const T* f, const T* cvec, T cval, const T* dA, T* out, T* u_inout, double* part,
                    cudaStream_t st);
// FP64 residual r = f - c u + M u from the relative extension: every
// difference w_k - w_i = (ref_k - ref_i) + (delta_k - delta_i) and
// w_i - u_i = (ref_i - u_i) + delta_i is formed from exact inputs, so the
// rounding floor is relative to the differences, not to |u| / dx^2.  Per-block
// partial (max|r|, sum r^2) into part (nblk(nB, 256) blocks).
void launch_resid_rel(const LevelView<double>& L, const double* u, const double* delta,
                      const double* refv, const double* f, const double* cvec, double cval,
                      double* r, double* part, cudaStream_t st);

// Stencil pass on B from w = E u:
//   APPLY : out = M u
//   RESID : out = f - c u + M u  (and block partials of max|out|, sum out^2
//           into part[2*block], part[2*block+1] if part != nullptr)
//   JACOBI: u += (f - c u + M u) * wdA, wdA = omega / dA (in place, out unused)
template <typename T>
void launch_lap(const LevelView<T>& L, LapMode mode, const T* u, const T* w, const T* f,
                const T* cvec, T cval, const T* dA, T omega, T* out, T* u_inout, double* part,
                int nblocks_part, cudaStream_t st);

// Number of blocks (2 partial doubles each) of a RESID / RESID_REL stencil pass.
int lap_blocks_f64(const LevelView<double>& L);

// The outer residual in FP32-pair arithmetic (relative form, see k_extend_pair
// and k_resid_pair): launch_extend_pair fills delta (pairs) and refv (floats)
// over B+ (needs L.ewp), launch_resid_pair forms r = f - c u + M u on B with
// norm partials of resid_pair_blocks(L) blocks into part.
// kPairSlots slots collect the largest |u - ref| staged by any tile (as float
// bits, one atomic max per tile into slot tile mod kPairSlots), which bounds
// the size of the rounding errors of the pair arithmetic.
constexpr int kPairSlots = 1024;
void launch_extend_pair(const LevelView<double>& L, const double* u, float2* delta, float* refv,
                        uint32_t* dmax, cudaStream_t st);
void launch_resid_pair(const LevelView<double>& L, const double* u, const float2* delta,
                       const float* refv, const double* f, const double* cvec, double cval, double* r,
                       double* part, cudaStream_t st);
int resid_pair_blocks(const LevelView<double>& L);
// Pointwise FP64 check of a pair residual r: lists the band points with
// |r_i| > thr (at most cap; *count gets the number of candidates, which may
// exceed cap) and sets *maxbits to the bit pattern of the largest |r_i| there,
// evaluated in FP64 (see k_check_points).
void launch_pointwise_check(const LevelView<double>& L, const double* u, const double* f,
                            const double* cvec, double cval, const double* r, double thr,
                            int32_t* list, int32_t cap, int32_t* count, unsigned long long* maxbits,
                            cudaStream_t st);

// The paper's scheme M_p u = E_1 (L_B u) - gamma (u - E_3 u) (Eq. 3.3):
// v = L_B u on B (band-restricted Laplacian); then, with w = E_3 u on B,
//   APPLY : out = M_p u
//   RESID : out = f - c u + M_p u (block partials into part, paper_blocks blocks)
//   JACOBI: u += (f - c u + M_p u) dA (in place)
template <typename T>
void launch_lap_band(const LevelView<T>& L, const T* u, T* v, cudaStream_t st);
// avec != null: the variable-diffusion form (Sec. 4.5.6) E_1 L~ - diag(gamma a)
// (I - E_3), v = L~ u from launch_lap_vard.
template <typename T>
void launch_paper(const LevelView<T>& L, LapMode mode, const T* u, const T* v, const T* w, const T* f,
                  const T* cvec, T cval, const T* dA, T* out, T* u_inout, double* part,
                  const T* avec, cudaStream_t st);
// v = L~ u = sum over axes of D^b diag(A^f a) D^f u on B (band-restricted).
template <typename T>
void launch_lap_vard(const LevelView<T>& L, const T* u, const T* a, T* v, cudaStream_t st);
int paper_blocks(const LevelView<double>& L);
// diag(M_p) and the dense A_p = cI - M_p (setup, FP64 records); a != null:
// the variable-diffusion form.
void launch_diag_Mp(const LevelView<double>& L, double* diagM, const double* a, cudaStream_t st);
template <typename M>
void launch_assemble_Ap(const LevelView<double>& L, const double* cvec, double cval, M* A,
                        const double* a, cudaStream_t st);

// RM smoother pieces: u += omega (f - (cI - L_B) u) / (c + gamma) with the
// band-restricted Laplacian, written to out (out may not alias u).
template <typename T>
void launch_rm_jacobi(const LevelView<T>& L, const T* u, const T* f, const T* cvec, T cval, T omega,
                      T* out, cudaStream_t st);
// r = f - (cI - L_B) u
template <typename T>
void launch_rm_resid(const LevelView<T>& L, const T* u, const T* f, const T* cvec, T cval, T* out,
                     cudaStream_t st);

// dst[j] = sum of linear-interpolation weights times src (restriction), or
// dst[j] += (prolongation with add).
template <typename T>
void launch_transfer(const TransferView<T>& tv, const T* src, T* dst, bool add, cudaStream_t st);

// Norm partials of a vector and the final reduction to out[0] = max|x|,
// out[1] = sum x^2 (device doubles).
constexpr int kNormBlocks = 1216;  // 152 SMs x 8
template <typename T>
void launch_norm_partials(const T* x, int64_t n, double* part, cudaStream_t st);
// out[0..3] = max, sum of squares, 1/max of the partials' vector, and the
// largest value in dmax's kPairSlots slots (0 without dmax; the slots are reset).
void launch_norm_final(const double* part, int nblocks, double* out, cudaStream_t st,
                       uint32_t* dmax = nullptr);

// Mixed precision helpers.
void launch_scale_to_f32(const double* r, const double* norms, float* r32, int64_t n, cudaStream_t st);
void launch_axpy_scaled(double* u, const float* d, const double* norms, int64_t n, cudaStream_t st);
void launch_axpy64(double* u, const double* d, int64_t n, cudaStream_t st);
template <typename T>
void launch_cast_to_f64(const T* x, double* y, int64_t n, cudaStream_t st);
template <typename T>
void launch_cast_from_f64(const double* x, T* y, int64_t n, cudaStream_t st);

// Coarsest direct solve x_g = Ainv b_g, g < G (FP64 matrix, FP64 accumulation).
template <typename T>
void launch_coarse_gemv(const double* Ainv, const T* const* b, T* const* x, int G, int32_t n,
                        cudaStream_t st);

// Residual norms of the finest level with the library's fixed device scratch
// (noalloc.cu); norms[0] = max|r|, norms[1] = sum r^2 (device).
void residual_norms_noalloc(const LevelView<double>& v, const double* f, const double* u,
                            const double* cvec, double cval, double* norms, cudaStream_t st);

// Coarsest solve with an FP32 explicit inverse (coarse32.cu): x_g (+)= Ainv b_g.
template <typename T>
void launch_coarse_gemv32(const float* Ainv, const T* const* b, T* const* x, int G, int32_t n, bool add,
                          cudaStream_t st);
// A (row-major FP32, overwritten) -> X = A^-1 (library LU, setup only).
void invert_dense_f32(float* A, float* X, int32_t n, cudaStream_t st, int32_t* err);

// Setup kernels.
void launch_diag_M(const LevelView<double>& L, double* diagM, cudaStream_t st);
template <typename M>
void launch_assemble_A(const LevelView<double>& L, const double* cvec, double cval, M* A,
                       cudaStream_t st);
// In-place Gauss-Jordan inversion with partial pivoting (row-major n x n).
void invert_dense(double* A, int32_t n, cudaStream_t st, int32_t* err);

}  // namespace cpm
