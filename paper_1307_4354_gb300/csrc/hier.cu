// Multigrid hierarchy, V-cycle (Algorithm 4.1), outer solve loop and the
// C ABI entry points declared in include/cpm.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "gmres.cuh"
#include "gemv.cuh"
#include "mlp.cuh"

namespace cpm {

thread_local std::string g_last_error;
int64_t launches_total();
void set_last_error(const std::string& msg) { g_last_error = msg; }

static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ----------------------------------------------------------------- transfer records
// For each target point (its cp), the base node floor((cp - lo)/dx_src) of the
// linear stencil in the source grid and the fractions; every stencil node
// must be a band node of the source level.
__global__ void k_transfer_records(const double* cp, int64_t cp_stride, int32_t n, int dim, int deg,
                                   double lo, double dx, BrickView src, uint64_t* base,
                                   double* fr64, float* fr32, int32_t* err) {
  const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int b[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) {
    const double t = __ddiv_rn(__dadd_rn(cp[a * cp_stride + j], -lo), dx);
    const double fl = floor(t);
    const double s = __dadd_rn(t, -fl);
    b[a] = (int)fl - (deg == 3 ? 1 : 0);
    fr64[(int64_t)a * n + j] = s;
    fr32[(int64_t)a * n + j] = (float)s;
  }
  bool ok = b[0] >= 0 && b[1] >= 0 && b[2] >= 0;
  const int np1 = deg + 1;
  for (int c = 0; c < (dim == 3 ? np1 : 1); ++c)
    for (int bb = 0; bb < np1; ++bb)
      for (int a = 0; a < np1; ++a)
        if (band_index(src, b[0] + a, b[1] + bb, b[2] + c) < 0) ok = false;
  if (!ok) atomicOr(err, 4);
  base[j] = ok ? ((uint64_t)b[0] | ((uint64_t)b[1] << 16) | ((uint64_t)b[2] << 32)) : 0ull;
}

// dA = c - diag(M) in FP64 and FP32.
// wdA = omega / (c - diag(M)): the Jacobi step size (Eq. 4.1), FP64 and FP32.
__global__ void k_diag_A(const double* diagM, const double* cvec, double cval, double omega,
                         double* dA64, float* dA32, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = omega / ((cvec ? cvec[i] : cval) - diagM[i]);
  dA64[i] = v;
  dA32[i] = (float)v;
}

// Linear transfers read their 2^d source indices from a per-target table (1)
// or find them through the source brick tables (0).
#ifndef CPM_TRANSFER_INDEXED
#define CPM_TRANSFER_INDEXED 1
#endif

// dst (n rows of ld floats) = src (n x n, row-major) rounded to FP32, the
// padding columns n .. ld-1 zero.
__global__ void k_round_f32(const double* src, int32_t n, int32_t ld, float* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * ld) return;
  const int64_t r = i / ld, c = i - r * ld;
  dst[i] = c < n ? (float)src[r * n + c] : 0.f;
}
// Largest coarsest level whose FP64 inverse also gets an FP32 copy (256 MB).
constexpr int32_t kCoarseF32CopyMax = 8192;
// Most candidate points of a pointwise FP64 check of a pair residual.
constexpr int32_t kCheckCap = 1 << 16;

__global__ void k_transfer_index(const uint64_t* base, int32_t n, int dim, BrickView src, int32_t* idx) {
  const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint64_t kb = base[j];
  const int x = (int)(kb & 0xffffu), y = (int)((kb >> 16) & 0xffffu), z = (int)((kb >> 32) & 0xffffu);
  for (int c = 0; c < (dim == 3 ? 2 : 1); ++c)
    for (int bb = 0; bb < 2; ++bb)
      for (int a = 0; a < 2; ++a) {
        const int32_t i = band_index(src, x + a, y + bb, z + c);
        idx[(int64_t)(4 * c + 2 * bb + a) * n + j] = i < 0 ? 0 : i;
      }
}

struct Transfer {
  DBuf<uint64_t> base;
  DBuf<int32_t> idx;  // linear, indexed: 2^d x n source indices
  BrickView src{};
  int deg = 1;
  DBuf<double> fr64;
  DBuf<float> fr32;
  int32_t n = 0;
};

template <typename T>
struct Work {
  DBuf<T> u, f, r, w, tmp, v, refv;
  void alloc(int64_t nB, int64_t nplus, bool paper, bool relative) {
    if (relative) refv.alloc(nplus);  // reference values of the relative extension
    u.alloc(nB);
    f.alloc(nB);
    r.alloc(nB);
    w.alloc(nplus);
    tmp.alloc(nB);
    if (paper) v.alloc(nB);  // L_B u of the paper-form operator
  }
};

struct HLevel {
  std::unique_ptr<Level> lev;
  DBuf<double> c64;   // per-point c (empty: scalar)
  DBuf<float> c32;
  DBuf<double> a64;   // diffusion coefficient (CPM_OP_VARDIFF)
  DBuf<float> a32;
  DBuf<double> dA64;  // omega / (c - diag(M))
  DBuf<float> dA32;
  DBuf<double> dM64;  // diag(M)
  Transfer R;  // restriction: targets = B of level l+1, source = this level
  Transfer P;  // prolongation: targets = B of this level, source = level l+1

  template <typename T>
  LevelView<T> view() const;
  template <typename T>
  const T* cvec() const;
  template <typename T>
  const T* dA() const;
};

template <>
LevelView<double> HLevel::view<double>() const {
  LevelView<double> v;
  v.bv = lev->view();
  v.key = lev->key.get();
  v.fr = lev->fr64.get();
  v.nplus = lev->nplus();
  v.nB = lev->nB;
  v.dim = lev->dim;
  v.inv_h2 = 1.0 / (lev->dx * lev->dx);
  v.gamma = 2.0 * lev->dim / (lev->dx * lev->dx);
  v.tile_brick = lev->tile_brick.get();
  v.tile_box = lev->tile_box.get();
  v.tile_mask = lev->tile_mask.get();
  v.tile_bstart = lev->tile_bstart.get();
  v.tile_start = lev->tile_start.get();
  v.tile_mid = lev->tile_mid.get();
  v.erec = lev->erec.get();
  v.efr = lev->efr32.get();
  v.ew64 = lev->ew64.get();
  v.ewp = lev->ewp.get();
  v.ntiles = lev->ntiles;
  v.ext_variant = lev->ext_variant;
  v.echunk = lev->echunk.get();
  v.tile_cstart = lev->tile_cstart.get();
  v.tile_cmid = lev->tile_cmid.get();
  v.nbr = lev->nbr.get();
  return v;
}
template <>
LevelView<float> HLevel::view<float>() const {
  LevelView<float> v;
  v.bv = lev->view();
  v.key = lev->key.get();
  v.fr = lev->fr32.get();
  v.nplus = lev->nplus();
  v.nB = lev->nB;
  v.dim = lev->dim;
  v.inv_h2 = (float)(1.0 / (lev->dx * lev->dx));
  v.gamma = (float)(2.0 * lev->dim / (lev->dx * lev->dx));
  v.tile_brick = lev->tile_brick.get();
  v.tile_box = lev->tile_box.get();
  v.tile_mask = lev->tile_mask.get();
  v.tile_bstart = lev->tile_bstart.get();
  v.tile_start = lev->tile_start.get();
  v.tile_mid = lev->tile_mid.get();
  v.erec = lev->erec.get();
  v.efr = lev->efr32.get();
  v.ew64 = lev->ew64.get();
  v.ewp = lev->ewp.get();
  v.ntiles = lev->ntiles;
  v.ext_variant = lev->ext_variant;
  v.echunk = lev->echunk.get();
  v.tile_cstart = lev->tile_cstart.get();
  v.tile_cmid = lev->tile_cmid.get();
  v.nbr = lev->nbr.get();
  return v;
}
template <> const double* HLevel::cvec<double>() const { return c64.get(); }
template <> const float* HLevel::cvec<float>() const { return c32.get(); }
template <typename T> static const T* avec_of(const HLevel& lv);
template <> const double* avec_of<double>(const HLevel& lv) { return lv.a64.get(); }
template <> const float* avec_of<float>(const HLevel& lv) { return lv.a32.get(); }
template <> const double* HLevel::dA<double>() const { return dA64.get(); }
template <> const float* HLevel::dA<float>() const { return dA32.get(); }

template <typename T>
static TransferView<T> tview(const Transfer& t, int dim);
template <>
TransferView<double> tview<double>(const Transfer& t, int dim) {
  return TransferView<double>{t.base.get(), t.fr64.get(), t.src, t.n, dim, t.deg, t.idx.get()};
}
template <>
TransferView<float> tview<float>(const Transfer& t, int dim) {
  return TransferView<float>{t.base.get(), t.fr32.get(), t.src, t.n, dim, t.deg, t.idx.get()};
}

}  // namespace cpm

using namespace cpm;

// Everything one solve mutates: per-level work vectors, the finest-level
// solve vectors, norms, a stream and the captured graphs.  A hierarchy owns one
// workspace; a batch gives every (hierarchy, right-hand side) its own.
struct Workspace {
  std::vector<cpm::Work<double>> w64;
  std::vector<cpm::Work<float>> w32;
  cpm::DBuf<double> part;   // norm partials (2 per block)
  int part_blocks = 0;
  cpm::DBuf<double> own_norms;  // [max, sumsq, 1/max, -] unless norms points elsewhere
  double* norms = nullptr;
  cpm::DBuf<double> normf;  // norms of f
  cpm::DBuf<double> u_own, f_own, r64, d64;
  cpm::DBuf<double> refv;   // per point of the finest B+: the extension's reference value (FP64 form)
  cpm::DBuf<float2> dpair;  // pair form: delta_j = (E u)_j - ref_j over the finest B+
  cpm::DBuf<float> rpair;   // pair form: ref_j
  cpm::DBuf<uint32_t> dmax; // pair form: slots of the largest staged |u - ref| (norms[3])
  cpm::DBuf<int32_t> chk_list, chk_count;      // pointwise FP64 check: candidate points
  cpm::DBuf<unsigned long long> chk_max;       // and the largest |r| among them (bits)
  cpm::DBuf<float> r32, d32;
  cpm::GmresWork<double> gm64;  // coarsest-level GMRES (coarse mode 3)
  cpm::GmresWork<float> gm32;
  cudaStream_t hs = nullptr;
  cudaEvent_t ev = nullptr;
  // outer residual of this solve's steps in FP32 pairs (until a check in FP64
  // disagrees with the convergence test, see solve_ws)
  bool pair = false;
  // graphs of one outer step: FP64, mixed, mixed with the learned smoother;
  // + 3 for the same with the outer residual in FP32 pairs
  cudaGraphExec_t graph[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int64_t graph_kernels[6] = {0, 0, 0, 0, 0, 0};
  int32_t graph_inner[6] = {0, 0, 0, 0, 0, 0};
  double* pinned = nullptr;
  template <typename T>
  cpm::Work<T>& work(int l);
  ~Workspace() {
    for (auto& g : graph)
      if (g) cudaGraphExecDestroy(g);
    if (ev) cudaEventDestroy(ev);
    if (hs) cudaStreamDestroy(hs);
    if (pinned) cudaFreeHost(pinned);
  }
};
template <> cpm::Work<double>& Workspace::work<double>(int l) { return w64[l]; }
template <> cpm::Work<float>& Workspace::work<float>(int l) { return w32[l]; }
template <typename T> static cpm::GmresWork<T>& gmres_work(Workspace& W);
template <> cpm::GmresWork<double>& gmres_work<double>(Workspace& W) { return W.gm64; }
template <> cpm::GmresWork<float>& gmres_work<float>(Workspace& W) { return W.gm32; }

struct cpm_hier_s {
  cpm_surface surface;
  cpm_mg_opts opts;
  double c = 1.0;
  std::vector<HLevel> L;
  DBuf<double> Ainv;     // coarse_mode 0: FP64 inverse
  DBuf<float> Ainv32;    // coarse_mode 1: FP32 inverse
  DBuf<float> Ainv_f32;  // coarse_mode 0: the FP64 inverse rounded to FP32, for FP32
                         // V-cycles (FP32 GEMV at twice the bandwidth and off the FP64
                         // pipe); built when it takes at most kCoarseF32CopyMax points;
                         // rows padded with zeros to ld_f32 (a multiple of 4) columns
  int32_t ld_f32 = 0;
  int32_t nc = 0;
  int32_t coarse_mode = 0;    // 0: FP64 inverse, 1: FP32 inverse (+FP64 refinement), 2: sweeps,
                              // 3: GMRES
  int32_t coarse_sweeps = 0;
  int32_t coarse_restarts = 3;
  bool pair_resid = false;    // outer residual in FP32 pairs (k_extend_pair + k_resid_pair)
  cpm_mlp mlp = nullptr;
  std::unique_ptr<cpm::MlpLevelData> mlpd;
  bool learned_active = false;
  Workspace ws;
};

namespace cpm {
// Allocate the work vectors of every level and the solve vectors.
static void alloc_workspace(const cpm_hier_s& H, Workspace& W, double* norms_slot = nullptr) {
  W.w64.resize(H.L.size());
  W.w32.resize(H.L.size());
  for (size_t l = 0; l < H.L.size(); ++l) {
    const int64_t nB = H.L[l].lev->nB, np = H.L[l].lev->nplus();
    const bool paper = H.opts.op_form != CPM_OP_MBR;
    W.w64[l].alloc(nB, np, paper, H.opts.relative != 0);
    W.w32[l].alloc(nB, np, paper, H.opts.relative != 0);
  }
  const int64_t nB0 = H.L[0].lev->nB;
  W.part_blocks = std::max<int>(std::max(lap_blocks_f64(H.L[0].view<double>()),
                                          paper_blocks(H.L[0].view<double>())),
                                 kNormBlocks);
  W.part.alloc(2 * (size_t)W.part_blocks);
  W.own_norms.alloc(4);
  W.norms = norms_slot ? norms_slot : W.own_norms.get();
  W.normf.alloc(4);
  W.u_own.alloc(nB0);
  W.f_own.alloc(nB0);
  W.r64.alloc(nB0);
  W.d64.alloc(nB0);
  W.refv.alloc(H.L[0].lev->nplus());  // FP64 form (also the check of the pair form)
  if (H.pair_resid) {
    W.dpair.alloc(H.L[0].lev->nplus());
    W.rpair.alloc(H.L[0].lev->nplus());
    W.dmax.alloc(kPairSlots);
    CPM_CUDA_TRY(cudaMemset(W.dmax.get(), 0, sizeof(uint32_t) * kPairSlots));
    W.chk_list.alloc(kCheckCap);
    W.chk_count.alloc(1);
    W.chk_max.alloc(1);
  }
  W.r32.alloc(nB0);
  W.d32.alloc(nB0);
  if (H.coarse_mode == 3) {
    const int64_t nc = H.L.back().lev->nB;
    W.gm64.alloc(nc, kGmresMaxM);
    W.gm32.alloc(nc, kGmresMaxM);
  }
  CPM_CUDA_TRY(cudaStreamCreateWithFlags(&W.hs, cudaStreamNonBlocking));
  CPM_CUDA_TRY(cudaEventCreateWithFlags(&W.ev, cudaEventDisableTiming));
  CPM_CUDA_TRY(cudaMallocHost(&W.pinned, 8 * sizeof(double)));
}
}  // namespace cpm

namespace cpm {

// ----------------------------------------------------------------- level ops
// The operator of level l in the hierarchy's form: M u (APPLY), the residual
// f - A u (RESID, block partials into part when given) or one weighted Jacobi
// sweep on A u = f in place (JACOBI).  MBR form: w = E u on B+, then the
// stencil on w; paper form: v = L_B u and w = E_3 u on B, then E_1 v - gamma
// (u - w).
template <typename T>
static void level_op(cpm_hier_s* H, Workspace& W, int l, LapMode mode, const T* f, const T* u,
                     T* out, double* part, cudaStream_t st) {
  HLevel& lv = H->L[l];
  const LevelView<T> v = lv.view<T>();
  Work<T>& w = W.work<T>(l);
  const bool upd = mode == LAP_JACOBI || mode == LAP_JAC_RED || mode == LAP_JAC_BLACK;
  const T* dA = upd ? lv.dA<T>() : nullptr;
  T* u_inout = upd ? const_cast<T*>(u) : nullptr;
  if (H->opts.op_form == CPM_OP_PAPER || H->opts.op_form == CPM_OP_VARDIFF) {
    const T* a = H->opts.op_form == CPM_OP_VARDIFF ? avec_of<T>(lv) : nullptr;
    if (a)
      launch_lap_vard<T>(v, u, a, w.v.get(), st);
    else
      launch_lap_band<T>(v, u, w.v.get(), st);
    launch_extend<T>(v, u, w.w.get(), v.nB, st);
    launch_paper<T>(v, mode, u, w.v.get(), w.w.get(), f, lv.cvec<T>(), (T)H->c, dA, out, u_inout,
                    part, a, st);
  } else if (H->opts.relative && (mode == LAP_RESID || mode == LAP_JACOBI)) {
    launch_extend_rel<T>(v, u, w.w.get(), w.refv.get(), st);
    launch_lap_rel<T>(v, mode == LAP_RESID ? LAP_RESID_REL : LAP_JAC_REL, u, w.w.get(), w.refv.get(), f,
                      lv.cvec<T>(), (T)H->c, dA, out, u_inout, part, st);
  } else {
    launch_extend<T>(v, u, w.w.get(), (int32_t)v.nplus, st);
    launch_lap<T>(v, mode, u, w.w.get(), f, lv.cvec<T>(), (T)H->c, dA, (T)H->opts.omega, out,
                  u_inout, part, 0, st);
  }
}

template <typename T>
static void smooth(cpm_hier_s* H, Workspace& W, int l, const T* f, T* u, int sweeps,
                   cudaStream_t st) {
  HLevel& lv = H->L[l];
  const LevelView<T> v = lv.view<T>();
  Work<T>& w = W.work<T>(l);
  const T omega = (T)H->opts.omega;
  const T cval = (T)H->c;
  for (int s = 0; s < sweeps; ++s) {
    if (H->opts.smoother == CPM_SMOOTH_RM) {
      launch_rm_jacobi<T>(v, u, f, lv.cvec<T>(), cval, omega, w.tmp.get(), st);
      launch_extend<T>(v, w.tmp.get(), u, v.nB, st);
    } else if (H->opts.smoother == CPM_SMOOTH_RBGS) {
      level_op<T>(H, W, l, LAP_JAC_RED, f, u, nullptr, nullptr, st);
      level_op<T>(H, W, l, LAP_JAC_BLACK, f, u, nullptr, nullptr, st);
    } else {
      level_op<T>(H, W, l, LAP_JACOBI, f, u, nullptr, nullptr, st);
    }
  }
}

// r = f - A u (Jacobi smoother) or f - (cI - L) u (Ruuth-Merriman, Algorithm 4.1 step 2).
template <typename T>
static void transfer_residual(cpm_hier_s* H, Workspace& W, int l, const T* f, const T* u, T* r,
                              cudaStream_t st) {
  HLevel& lv = H->L[l];
  const LevelView<T> v = lv.view<T>();
  Work<T>& w = W.work<T>(l);
  if (H->opts.smoother == CPM_SMOOTH_RM) {
    launch_rm_resid<T>(v, u, f, lv.cvec<T>(), (T)H->c, r, st);
  } else if (H->opts.residual_mode == 1) {
    level_op<T>(H, W, l, LAP_RESID, f, u, r, nullptr, st);
  } else {
    // f - A (E u): first E u on B, then the residual of that re-extended iterate
    launch_extend<T>(v, u, w.tmp.get(), v.nB, st);
    level_op<T>(H, W, l, LAP_RESID, f, w.tmp.get(), r, nullptr, st);
  }
}

// Systems that share one hierarchy and run one V-cycle in lockstep on one
// stream: every step is issued for each member in turn (so each member's
// arithmetic is exactly that of its own V-cycle), and the coarsest direct
// solve reads the dense inverse once for all members.
constexpr int kMaxGroup = 16;

// Coarsest level: explicit FP64 or FP32 inverse, or weighted Jacobi sweeps from zero.
template <typename T>
static void coarse_solve(cpm_hier_s* H, Workspace* const* W, int G, const T* const* f, T* const* u,
                         cudaStream_t st) {
  const int l = (int)H->L.size() - 1;
  if (H->coarse_mode == 0) {
    if constexpr (sizeof(T) == 4) {
      if (H->Ainv_f32.n > 0) {
        launch_dense_gemv_v4<T>(H->Ainv_f32.get(), H->ld_f32, f, u, G, H->nc, st);
        count_launch((G + kGemvMaxVectors - 1) / kGemvMaxVectors);
        return;
      }
    }
    launch_coarse_gemv<T>(H->Ainv.get(), f, u, G, H->nc, st);
    return;
  }
  if (H->coarse_mode == 1) {
    launch_coarse_gemv32<T>(H->Ainv32.get(), f, u, G, H->nc, false, st);
    if constexpr (sizeof(T) == 8) {
      // two steps of iterative refinement with the FP64 residual of the level
      HLevel& lv = H->L[l];
      const LevelView<double> v = lv.view<double>();
      const double* r[kMaxGroup];
      for (int g = 0; g < G; ++g) r[g] = W[g]->w64[l].r.get();
      for (int it = 0; it < 2; ++it) {
        for (int g = 0; g < G; ++g)
          level_op<double>(H, *W[g], l, LAP_RESID, f[g], u[g], W[g]->w64[l].r.get(), nullptr, st);
        launch_coarse_gemv32<double>(H->Ainv32.get(), r, u, G, H->nc, true, st);
      }
    }
    return;
  }
  HLevel& lv = H->L[l];
  if (H->coarse_mode == 3) {
    for (int g = 0; g < G; ++g) {
      Workspace& Wg = *W[g];
      GmresOps<T> op;
      op.residual = [H, &Wg, l](const T* ff, const T* uu, T* rr, cudaStream_t s2) {
        level_op<T>(H, Wg, l, LAP_RESID, ff, uu, rr, nullptr, s2);
      };
      gmres_solve<T>(op, gmres_work<T>(Wg), f[g], u[g], lv.dA<T>(), H->coarse_restarts, st);
    }
    return;
  }
  for (int g = 0; g < G; ++g) {
    CPM_CUDA_TRY(cudaMemsetAsync(u[g], 0, sizeof(T) * lv.lev->nB, st));
    for (int s = 0; s < H->coarse_sweeps; ++s)
      level_op<T>(H, *W[g], l, LAP_JACOBI, f[g], u[g], nullptr, nullptr, st);
  }
}

// V-cycle of Algorithm 4.1 from level l for G systems in lockstep.
template <typename T>
static void vcycle_level(cpm_hier_s* H, Workspace* const* W, int G, int l, const T* const* f,
                         T* const* u, cudaStream_t st) {
  const int nl = (int)H->L.size();
  if (l == nl - 1) {
    coarse_solve<T>(H, W, G, f, u, st);
    return;
  }
  HLevel& lv = H->L[l];
  HLevel& cv = H->L[l + 1];
  const T* cf[kMaxGroup];
  T* cu[kMaxGroup];
  for (int g = 0; g < G; ++g) {
    Work<T>& w = W[g]->work<T>(l);
    Work<T>& cw = W[g]->work<T>(l + 1);
    int pre = H->opts.nu1;
    if constexpr (sizeof(T) == 4) {
      if (l == 0 && H->learned_active && pre > 0) {
        // learned smoother in place of the first Jacobi sweep: r = f - A u, u += net(r)
        const LevelView<float> v = lv.view<float>();
        launch_extend<float>(v, u[g], w.w.get(), (int32_t)v.nplus, st);
        launch_lap<float>(v, LAP_RESID, u[g], w.w.get(), f[g], lv.cvec<float>(), (float)H->c, nullptr,
                          0.f, w.r.get(), nullptr, nullptr, 0, st);
        mlp_forward(H->mlp->params.get(), *H->mlpd, w.r.get(), 1.f / v.inv_h2, nullptr, u[g], nullptr,
                    st);
        --pre;
      }
    }
    smooth<T>(H, *W[g], l, f[g], u[g], pre, st);
    transfer_residual<T>(H, *W[g], l, f[g], u[g], w.r.get(), st);
    launch_transfer<T>(tview<T>(lv.R, lv.lev->dim), w.r.get(), cw.f.get(), false, st);
    if (l + 1 < nl - 1)
      CPM_CUDA_TRY(cudaMemsetAsync(cw.u.get(), 0, sizeof(T) * cv.lev->nB, st));
    cf[g] = cw.f.get();
    cu[g] = cw.u.get();
  }
  // V-cycle: one cycle of the next level from zero; W-cycle: a second one
  // from the first's result (the coarsest level is solved once)
  const int ncyc = l + 1 == nl - 1 ? 1 : H->opts.cycle;
  for (int q = 0; q < ncyc; ++q) vcycle_level<T>(H, W, G, l + 1, cf, cu, st);
  for (int g = 0; g < G; ++g) {
    launch_transfer<T>(tview<T>(lv.P, lv.lev->dim), cu[g], u[g], true, st);
    smooth<T>(H, *W[g], l, f[g], u[g], H->opts.nu2, st);
  }
}

template <typename T>
static void vcycle_level(cpm_hier_s* H, Workspace& W, int l, const T* f, T* u, cudaStream_t st) {
  Workspace* w = &W;
  vcycle_level<T>(H, &w, 1, l, &f, &u, st);
}

// Full multigrid from zero (remark at Algorithm 4.1): f restricted to every
// level (into the levels' work f), the coarsest level solved, then on each
// finer level the prolonged coarse solution starts one cycle of that level.
// A level's work f and u are free again once the level above has taken its
// start value from them.
template <typename T>
static void fmg(cpm_hier_s* H, Workspace& W, const T* f, T* u, cudaStream_t st) {
  const int nl = (int)H->L.size();
  std::vector<const T*> fl(nl);
  fl[0] = f;
  for (int l = 0; l + 1 < nl; ++l) {
    launch_transfer<T>(tview<T>(H->L[l].R, H->L[l].lev->dim), fl[l], W.work<T>(l + 1).f.get(), false, st);
    fl[l + 1] = W.work<T>(l + 1).f.get();
  }
  T* uc = nl == 1 ? u : W.work<T>(nl - 1).u.get();
  Workspace* w = &W;
  coarse_solve<T>(H, &w, 1, &fl[nl - 1], &uc, st);
  for (int l = nl - 2; l >= 0; --l) {
    T* ul = l == 0 ? u : W.work<T>(l).u.get();
    launch_transfer<T>(tview<T>(H->L[l].P, H->L[l].lev->dim), W.work<T>(l + 1).u.get(), ul, false, st);
    vcycle_level<T>(H, W, l, fl[l], ul, st);
  }
}

// Outer residual r = f - A u on the finest level with norms into W.norms, in
// the relative form (differences formed from exact inputs; its rounding floor
// is far below that of w = E u followed by the stencil at fine dx), evaluated
// in FP32 pairs on the FP32 pipe (default) or in FP64.
static void outer_residual(cpm_hier_s* H, Workspace& W, const double* f, const double* u, double* r,
                           cudaStream_t st, bool pair) {
  HLevel& lv = H->L[0];
  const LevelView<double> v = lv.view<double>();
  if (H->opts.op_form != CPM_OP_MBR) {  // direct form of Eq. 3.3
    level_op<double>(H, W, 0, LAP_RESID, f, u, r, W.part.get(), st);
    launch_norm_final(W.part.get(), paper_blocks(v), W.norms, st);
    return;
  }
  if (pair && H->pair_resid) {
    launch_extend_pair(v, u, W.dpair.get(), W.rpair.get(), W.dmax.get(), st);
    launch_resid_pair(v, u, W.dpair.get(), W.rpair.get(), f, lv.c64.get(), H->c, r, W.part.get(), st);
    launch_norm_final(W.part.get(), resid_pair_blocks(v), W.norms, st, W.dmax.get());
    return;
  }
  launch_extend_rel(v, u, W.w64[0].w.get(), W.refv.get(), st);
  launch_resid_rel(v, u, W.w64[0].w.get(), W.refv.get(), f, lv.c64.get(), H->c, r, W.part.get(), st);
  launch_norm_final(W.part.get(), lap_blocks_f64(v), W.norms, st);
}

// One outer iteration after the residual, for G systems of one hierarchy in
// lockstep: u += V(0, r), then the new residual.
static void outer_step(cpm_hier_s* H, Workspace* const* W, int G, int mode, int inner,
                       cudaStream_t st, bool first_fmg = false) {
  const int64_t nB = H->L[0].lev->nB;
  if (mode == CPM_SOLVE_F64) {
    const double* r[kMaxGroup];
    double* d[kMaxGroup];
    for (int g = 0; g < G; ++g) {
      CPM_CUDA_TRY(cudaMemsetAsync(W[g]->d64.get(), 0, sizeof(double) * nB, st));
      r[g] = W[g]->r64.get();
      d[g] = W[g]->d64.get();
    }
    if (first_fmg)
      for (int g = 0; g < G; ++g) fmg<double>(H, *W[g], r[g], d[g], st);
    else
      vcycle_level<double>(H, W, G, 0, r, d, st);
    for (int g = 0; g < G; ++g) launch_axpy64(W[g]->u_own.get(), W[g]->d64.get(), nB, st);
  } else {
    const float* r[kMaxGroup];
    float* d[kMaxGroup];
    for (int g = 0; g < G; ++g) {
      launch_scale_to_f32(W[g]->r64.get(), W[g]->norms, W[g]->r32.get(), nB, st);
      CPM_CUDA_TRY(cudaMemsetAsync(W[g]->d32.get(), 0, sizeof(float) * nB, st));
      r[g] = W[g]->r32.get();
      d[g] = W[g]->d32.get();
    }
    for (int j = 0; j < inner; ++j) {
      if (first_fmg && j == 0)
        for (int g = 0; g < G; ++g) fmg<float>(H, *W[g], r[g], d[g], st);
      else
        vcycle_level<float>(H, W, G, 0, r, d, st);
    }
    for (int g = 0; g < G; ++g) launch_axpy_scaled(W[g]->u_own.get(), W[g]->d32.get(), W[g]->norms, nB, st);
  }
  for (int g = 0; g < G; ++g)
    outer_residual(H, *W[g], W[g]->f_own.get(), W[g]->u_own.get(), W[g]->r64.get(), st, W[g]->pair);
}

static void outer_step(cpm_hier_s* H, Workspace& W, int mode, int inner, cudaStream_t st,
                       bool first_fmg = false) {
  Workspace* w = &W;
  outer_step(H, &w, 1, mode, inner, st, first_fmg);
}

}  // namespace cpm

// ----------------------------------------------------------------- C ABI
#define CPM_API_BEGIN try {
#define CPM_API_END                                                    \
  }                                                                    \
  catch (const cpm::Error& e) {                                        \
    cpm::set_last_error(e.msg);                                        \
    return e.status;                                                   \
  }                                                                    \
  catch (const std::bad_alloc&) {                                      \
    cpm::set_last_error("host allocation failed");                     \
    return CPM_ERR_OOM;                                                \
  }                                                                    \
  catch (...) {                                                        \
    cpm::set_last_error("unexpected exception");                       \
    return CPM_ERR_CUDA;                                               \
  }                                                                    \
  return CPM_OK;

extern "C" {

const char* cpm_status_str(cpm_status s) {
  switch (s) {
    case CPM_OK: return "ok";
    case CPM_ERR_ARG: return "invalid argument";
    case CPM_ERR_OOM: return "out of device memory";
    case CPM_ERR_CUDA: return "CUDA error";
    case CPM_ERR_REACH: return "band wider than the closest-point reach";
    case CPM_ERR_DIVERGED: return "diverged";
    case CPM_ERR_NOT_CONVERGED: return "not converged";
    case CPM_ERR_TIMEOUT: return "timeout";
    case CPM_ERR_CHECKED: return "device check failed";
    case CPM_ERR_SINGULAR: return "singular coarsest matrix";
  }
  return "unknown status";
}

const char* cpm_last_error(void) { return cpm::g_last_error.c_str(); }

static void check_surface(const cpm_surface* s) {
  CPM_CHECK(s != nullptr, CPM_ERR_ARG, "surface is NULL");
  CPM_CHECK(s->kind >= CPM_CIRCLE && s->kind <= CPM_DZIUK, CPM_ERR_ARG, "unknown surface kind");
  const int np = s->kind == CPM_TORUS ? 2 : (s->kind == CPM_ELLIPSOID ? 3 : (s->kind == CPM_DZIUK ? 0 : 1));
  for (int i = 0; i < np; ++i)
    CPM_CHECK(s->param[i] > 0 && std::isfinite(s->param[i]), CPM_ERR_ARG,
              "surface parameters must be positive");
  if (s->kind == CPM_TORUS)
    CPM_CHECK(s->param[1] < s->param[0], CPM_ERR_ARG, "torus needs r < R");
}

static double default_lambda2(int dim) { return dim == 3 ? 17.0 : 13.0; }

static int grid_n(const cpm_grid* g) {
  if (g->n > 0) return (int)g->n;
  return (int)std::llround(-2.0 * g->lo / g->dx) + 1;
}

cpm_status cpm_build_band(const cpm_surface* surface, const cpm_grid* grid, cpm_stream stream,
                          cpm_band* out) {
  CPM_API_BEGIN
  CPM_CHECK(out != nullptr && grid != nullptr, CPM_ERR_ARG, "NULL argument");
  *out = nullptr;
  check_surface(surface);
  CPM_CHECK(grid->dx > 0 && std::isfinite(grid->dx), CPM_ERR_ARG, "dx must be positive");
  CPM_CHECK(grid->lo < 0 && std::isfinite(grid->lo), CPM_ERR_ARG, "lo must be negative");
  const int dim = surface_dim(*surface);
  const double lam2 = grid->lambda2 > 0 ? grid->lambda2 : default_lambda2(dim);
  std::unique_ptr<cpm_band_s> b(new cpm_band_s);
  b->surface = *surface;
  build_level(*surface, grid->lo, grid->dx, grid_n(grid), lam2, (cudaStream_t)stream, b->lev);
  *out = b.release();
  CPM_API_END
}

cpm_status cpm_band_info(cpm_band band, int64_t* n_band, int64_t* n_ghost) {
  CPM_API_BEGIN
  CPM_CHECK(band != nullptr, CPM_ERR_ARG, "band is NULL");
  if (n_band) *n_band = band->lev.nB;
  if (n_ghost) *n_ghost = band->lev.nG;
  CPM_API_END
}

static void export_level(const Level& L, int32_t* ijk, double* cp, int32_t* base) {
  const int64_t np = L.nplus();
  const int d = L.dim;
  std::vector<uint64_t> key(np);
  CPM_CUDA_TRY(cudaDeviceSynchronize());
  CPM_CUDA_TRY(cudaMemcpy(key.data(), L.key.get(), np * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  if (cp) {
    std::vector<double> c((size_t)d * np);
    CPM_CUDA_TRY(cudaMemcpy(c.data(), L.cp.get(), c.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < np; ++i)
      for (int a = 0; a < d; ++a) cp[i * d + a] = c[(size_t)a * np + i];
  }
  for (int64_t i = 0; i < np; ++i) {
    const uint64_t k = key[i];
    const int own[3] = {key_x(k), key_y(k), key_z(k)};
    const int off[3] = {key_ox(k), key_oy(k), key_oz(k)};
    for (int a = 0; a < d; ++a) {
      if (ijk) ijk[i * d + a] = own[a];
      if (base) base[i * d + a] = own[a] + off[a];
    }
  }
}

cpm_status cpm_band_export(cpm_band band, int32_t* ijk, double* cp, int32_t* stencil_base) {
  CPM_API_BEGIN
  CPM_CHECK(band != nullptr, CPM_ERR_ARG, "band is NULL");
  export_level(band->lev, ijk, cp, stencil_base);
  CPM_API_END
}

cpm_status cpm_band_counts(cpm_band band, int64_t* counts, cpm_stream stream) {
  CPM_API_BEGIN
  CPM_CHECK(band != nullptr && counts != nullptr, CPM_ERR_ARG, "NULL argument");
  band_counts(band->lev, (cudaStream_t)stream, counts);
  CPM_API_END
}

cpm_status cpm_band_destroy(cpm_band band) {
  CPM_API_BEGIN
  delete band;
  CPM_API_END
}

// Copy a level (device to device) so the hierarchy owns its finest band.
static void copy_level(const Level& a, Level& b, cudaStream_t st) {
  b.dim = a.dim; b.lo = a.lo; b.dx = a.dx; b.lambda2 = a.lambda2; b.n = a.n;
  b.nbx = a.nbx; b.nby = a.nby; b.nbz = a.nbz; b.nbricks = a.nbricks; b.nB = a.nB; b.nG = a.nG;
  auto cp = [&](auto& dst, const auto& src) {
    dst.alloc(src.n);
    if (src.n)
      CPM_CUDA_TRY(cudaMemcpyAsync(dst.get(), src.get(), src.n * sizeof(*src.get()),
                                   cudaMemcpyDeviceToDevice, st));
  };
  cp(b.map, a.map); cp(b.bmask, a.bmask); cp(b.gmask, a.gmask); cp(b.bstart, a.bstart);
  cp(b.gstart, a.gstart); cp(b.bcoord, a.bcoord); cp(b.brec, a.brec); cp(b.key, a.key); cp(b.cp, a.cp);
  cp(b.fr64, a.fr64); cp(b.fr32, a.fr32);
  b.ntiles = a.ntiles;
  cp(b.tile_brick, a.tile_brick); cp(b.tile_box, a.tile_box); cp(b.tile_mask, a.tile_mask); cp(b.tile_bstart, a.tile_bstart); cp(b.tile_start, a.tile_start); cp(b.tile_mid, a.tile_mid); cp(b.erec, a.erec);
  cp(b.efr32, a.efr32); cp(b.ew64, a.ew64); cp(b.nbr, a.nbr);
  b.nchunks = a.nchunks;
  cp(b.echunk, a.echunk); cp(b.tile_cstart, a.tile_cstart); cp(b.tile_cmid, a.tile_cmid);
}

static void build_transfer(const Level& target, const Level& src, Transfer& t, int deg,
                           cudaStream_t st, int32_t* err) {
  t.n = target.nB;
  t.src = src.view();
  t.deg = deg;
  t.base.alloc((size_t)t.n);
  t.fr64.alloc((size_t)target.dim * t.n);
  t.fr32.alloc((size_t)target.dim * t.n);
  k_transfer_records<<<nblk(t.n, 256), 256, 0, st>>>(target.cp.get(), target.nplus(), t.n, target.dim, deg,
                                                     src.lo, src.dx, src.view(), t.base.get(),
                                                     t.fr64.get(), t.fr32.get(), err);
  CPM_CUDA_TRY(cudaGetLastError());
  if (CPM_TRANSFER_INDEXED && deg == 1 && t.n > 0) {
    t.idx.alloc((size_t)(target.dim == 3 ? 8 : 4) * t.n);
    k_transfer_index<<<nblk(t.n, 256), 256, 0, st>>>(t.base.get(), t.n, target.dim, src.view(),
                                                     t.idx.get());
    CPM_CUDA_TRY(cudaGetLastError());
  }
}

cpm_status cpm_build_hierarchy(cpm_band finest, const cpm_mg_opts* opts_in, cpm_stream stream,
                               cpm_hier* out) {
  CPM_API_BEGIN
  CPM_CHECK(finest != nullptr && out != nullptr, CPM_ERR_ARG, "NULL argument");
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  cpm_mg_opts o{};
  if (opts_in) o = *opts_in;
  if (o.nu1 <= 0 && o.nu2 <= 0) { o.nu1 = 3; o.nu2 = 3; }
  if (o.omega <= 0) o.omega = 0.8;
  if (o.transfer_deg == 0) o.transfer_deg = 1;
  CPM_CHECK(o.transfer_deg == 1 || o.transfer_deg == 3, CPM_ERR_ARG,
            "transfer_deg must be 1 (linear) or 3 (cubic)");
  CPM_CHECK(o.smoother == CPM_SMOOTH_JACOBI || o.smoother == CPM_SMOOTH_RM ||
                o.smoother == CPM_SMOOTH_RBGS,
            CPM_ERR_ARG, "unknown smoother");
  if (o.cycle == 0) o.cycle = 1;
  CPM_CHECK(o.cycle == 1 || o.cycle == 2, CPM_ERR_ARG, "cycle must be 1 (V) or 2 (W)");
  CPM_CHECK(o.nu1 >= 0 && o.nu2 >= 0 && o.nu1 + o.nu2 <= 64, CPM_ERR_ARG, "bad sweep counts");
  CPM_CHECK(o.op_form == CPM_OP_MBR || o.op_form == CPM_OP_PAPER || o.op_form == CPM_OP_VARDIFF,
            CPM_ERR_ARG, "unknown op_form");
  CPM_CHECK((o.op_form == CPM_OP_VARDIFF) == (o.a_device != nullptr), CPM_ERR_ARG,
            "a_device is given exactly with op_form CPM_OP_VARDIFF");
  CPM_CHECK(o.relative == 0 || (o.relative == 1 && o.op_form == CPM_OP_MBR), CPM_ERR_ARG,
            "relative = 1 is for the CPM_OP_MBR operator");
  CPM_CHECK(o.ext_variant >= 0 && o.ext_variant <= 3, CPM_ERR_ARG, "ext_variant must be 0 .. 3");
  CPM_CHECK(o.outer_f64 == 0 || o.outer_f64 == 1, CPM_ERR_ARG, "outer_f64 must be 0 or 1");
  CPM_CHECK(o.op_form == CPM_OP_MBR || o.smoother != CPM_SMOOTH_RM, CPM_ERR_ARG,
            "the paper-form operator is smoothed on A (Jacobi or red-black Gauss-Seidel)");
  if (!(o.c > 0)) o.c = 1.0;
  CPM_CHECK(std::isfinite(o.c), CPM_ERR_ARG, "c must be finite");
  std::unique_ptr<cpm_hier_s> H(new cpm_hier_s);
  H->surface = finest->surface;
  H->opts = o;
  H->c = o.c;
  const Level& f0 = finest->lev;
  const double reach = surface_reach(finest->surface);
  const double lam = std::sqrt(f0.lambda2);
  CPM_CHECK(o.coarse_f64_max >= 0 && o.coarse_dense_max >= 0 && o.coarse_dense_max <= 65536,
            CPM_ERR_ARG, "bad coarse_f64_max / coarse_dense_max");
  const int64_t dense_max = o.coarse_dense_max > 0 ? o.coarse_dense_max : 40000;
  const int64_t f64_max = std::min<int64_t>(o.coarse_f64_max > 0 ? o.coarse_f64_max : 16384, dense_max);

  // levels
  H->L.emplace_back();
  H->L[0].lev.reset(new Level);
  copy_level(f0, *H->L[0].lev, st);
  H->pair_resid = o.op_form == CPM_OP_MBR && o.outer_f64 == 0;
  if (H->pair_resid) build_pair_weights(*H->L[0].lev, st);
  double dx = f0.dx;
  for (;;) {
    const double next = 2.0 * dx;
    const Level& cur = *H->L.back().lev;
    bool more;
    if (o.coarsest_dx > 0) {
      more = next <= o.coarsest_dx * (1 + 1e-12);
      CPM_CHECK(!more || lam * next < reach, CPM_ERR_REACH,
                "coarsest_dx too coarse for the surface reach");
    } else {
      more = (lam + 1.0) * next < reach && cur.nB > 64;
    }
    if (!more) break;
    const int n_next = (int)std::llround(-2.0 * f0.lo / next) + 1;
    CPM_CHECK(std::fabs((n_next - 1) * next + 2.0 * f0.lo) < 1e-9 * next, CPM_ERR_ARG,
              "coarse grid does not nest (lo must be a multiple of the coarse spacing)");
    H->L.emplace_back();
    H->L.back().lev.reset(new Level);
    build_level(finest->surface, f0.lo, next, n_next, f0.lambda2, st, *H->L.back().lev);
    dx = next;
  }
  if (!(o.coarsest_dx > 0)) {
    // a coarsest level too large for the dense solve: coarser levels whose
    // band stays within the reach, as long as their band builds
    while (H->L.back().lev->nB > dense_max && lam * 2.0 * dx < reach) {
      const double next = 2.0 * dx;
      const int n_next = (int)std::llround(-2.0 * f0.lo / next) + 1;
      if (std::fabs((n_next - 1) * next + 2.0 * f0.lo) >= 1e-9 * next) break;
      std::unique_ptr<Level> lv(new Level);
      try {
        build_level(finest->surface, f0.lo, next, n_next, f0.lambda2, st, *lv);
      } catch (const Error& e) {
        if (e.status != CPM_ERR_REACH) throw;
        break;
      }
      H->L.emplace_back();
      H->L.back().lev = std::move(lv);
      dx = next;
    }
  }
  const int nl = (int)H->L.size();
  const Level& cl = *H->L[nl - 1].lev;
  CPM_CHECK(o.coarse_sweeps >= 0 && o.coarse_sweeps <= 10000, CPM_ERR_ARG, "bad coarse_sweeps");
  if (o.coarse_sweeps > 0) {
    H->coarse_mode = 2;
    H->coarse_sweeps = o.coarse_sweeps;
  } else if (cl.nB <= f64_max) {
    H->coarse_mode = 0;
  } else if (cl.nB <= dense_max) {
    H->coarse_mode = 1;
  } else {
    H->coarse_mode = 3;
    H->coarse_restarts = o.coarse_gmres > 0 ? o.coarse_gmres : 3;
  }
  CPM_CHECK(o.coarse_gmres >= 0 && o.coarse_gmres <= 1000, CPM_ERR_ARG, "bad coarse_gmres");
  CPM_CHECK(o.residual_mode == 0 || o.residual_mode == 1, CPM_ERR_ARG, "bad residual_mode");

  DBuf<int32_t> err(1);
  CPM_CUDA_TRY(cudaMemsetAsync(err.get(), 0, sizeof(int32_t), st));
  for (int l = 0; l + 1 < nl; ++l) {
    build_transfer(*H->L[l + 1].lev, *H->L[l].lev, H->L[l].R, o.transfer_deg, st, err.get());
    build_transfer(*H->L[l].lev, *H->L[l + 1].lev, H->L[l].P, o.transfer_deg, st, err.get());
  }
  // per-point c on every level (restricted from the finest band)
  if (o.c_device) {
    H->L[0].c64.alloc(f0.nB);
    CPM_CUDA_TRY(cudaMemcpyAsync(H->L[0].c64.get(), o.c_device, sizeof(double) * f0.nB,
                                 cudaMemcpyDeviceToDevice, st));
    for (int l = 0; l + 1 < nl; ++l) {
      HLevel& a = H->L[l];
      HLevel& b = H->L[l + 1];
      b.c64.alloc(b.lev->nB);
      launch_transfer<double>(tview<double>(a.R, a.lev->dim), a.c64.get(), b.c64.get(), false, st);
    }
    for (auto& lv : H->L) {
      lv.c32.alloc(lv.lev->nB);
      launch_cast_from_f64<float>(lv.c64.get(), lv.c32.get(), lv.lev->nB, st);
    }
  }
  // diffusion coefficient on every level (restricted from the finest band)
  if (o.a_device) {
    H->L[0].a64.alloc(f0.nB);
    CPM_CUDA_TRY(cudaMemcpyAsync(H->L[0].a64.get(), o.a_device, sizeof(double) * f0.nB,
                                 cudaMemcpyDeviceToDevice, st));
    for (int l = 0; l + 1 < nl; ++l) {
      HLevel& a = H->L[l];
      HLevel& b = H->L[l + 1];
      b.a64.alloc(b.lev->nB);
      launch_transfer<double>(tview<double>(a.R, a.lev->dim), a.a64.get(), b.a64.get(), false, st);
    }
    for (auto& lv : H->L) {
      lv.a32.alloc(lv.lev->nB);
      launch_cast_from_f64<float>(lv.a64.get(), lv.a32.get(), lv.lev->nB, st);
    }
  }
  // diag(A) = c - diag(M), work buffers
  for (auto& lv : H->L) {
    const int64_t nB = lv.lev->nB, np = lv.lev->nplus();
    DBuf<double> dM(nB);
    if (o.op_form != CPM_OP_MBR)
      launch_diag_Mp(lv.view<double>(), dM.get(), lv.a64.get(), st);
    else
      launch_diag_M(lv.view<double>(), dM.get(), st);
    lv.dA64.alloc(nB);
    lv.dA32.alloc(nB);
    k_diag_A<<<nblk(nB, 256), 256, 0, st>>>(dM.get(), lv.c64.get(), H->c, o.omega, lv.dA64.get(),
                                            lv.dA32.get(), nB);
    CPM_CUDA_TRY(cudaGetLastError());
    CPM_CUDA_TRY(cudaStreamSynchronize(st));
    lv.dM64 = std::move(dM);
  }
  // coarsest: dense A = diag(c) - M, inverted in place (FP64)
  H->nc = cl.nB;
  const size_t nn = (size_t)H->nc * H->nc;
  if (H->coarse_mode == 0) {
    H->Ainv.alloc(nn);
    CPM_CUDA_TRY(cudaMemsetAsync(H->Ainv.get(), 0, sizeof(double) * nn, st));
    if (o.op_form != CPM_OP_MBR)
      launch_assemble_Ap<double>(H->L[nl - 1].view<double>(), H->L[nl - 1].c64.get(), H->c,
                                 H->Ainv.get(), H->L[nl - 1].a64.get(), st);
    else
      launch_assemble_A<double>(H->L[nl - 1].view<double>(), H->L[nl - 1].c64.get(), H->c,
                                H->Ainv.get(), st);
    CPM_CUDA_TRY(cudaGetLastError());
    invert_dense(H->Ainv.get(), H->nc, st, err.get());
    if (H->nc <= kCoarseF32CopyMax) {
      H->ld_f32 = (H->nc + 3) / 4 * 4;
      const int64_t np = (int64_t)H->nc * H->ld_f32;
      H->Ainv_f32.alloc((size_t)np);
      k_round_f32<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(H->Ainv.get(), H->nc, H->ld_f32,
                                                               H->Ainv_f32.get());
      CPM_CUDA_TRY(cudaGetLastError());
    }
  } else if (H->coarse_mode == 1) {
    DBuf<float> A32(nn);
    CPM_CUDA_TRY(cudaMemsetAsync(A32.get(), 0, sizeof(float) * nn, st));
    if (o.op_form != CPM_OP_MBR)
      launch_assemble_Ap<float>(H->L[nl - 1].view<double>(), H->L[nl - 1].c64.get(), H->c,
                                A32.get(), H->L[nl - 1].a64.get(), st);
    else
      launch_assemble_A<float>(H->L[nl - 1].view<double>(), H->L[nl - 1].c64.get(), H->c,
                               A32.get(), st);
    CPM_CUDA_TRY(cudaGetLastError());
    H->Ainv32.alloc(nn);
    invert_dense_f32(A32.get(), H->Ainv32.get(), H->nc, st, err.get());
  }
  int32_t herr = 0;
  CPM_CUDA_TRY(cudaMemcpyAsync(&herr, err.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  CPM_CHECK(!(herr & 4), CPM_ERR_REACH, "a transfer stencil leaves the source band");
  CPM_CHECK(!(herr & 1), CPM_ERR_SINGULAR, "coarsest-level matrix is singular");

  // solve buffers
  alloc_workspace(*H, H->ws);
  // the FP32 extension variant of every level, by timing (its "tile": one
  // thread per point, persistent pipelined tiles, or chunks of one base)
  for (int l = 0; l < nl; ++l) {
    Level& lev = *H->L[l].lev;
    if (o.ext_variant > 0) {
      lev.ext_variant = o.ext_variant - 1;
      continue;
    }
    CPM_CUDA_TRY(cudaMemsetAsync(H->ws.w32[l].u.get(), 0, sizeof(float) * lev.nB, st));
    lev.ext_variant = tune_extension(H->L[l].view<float>(), H->ws.w32[l].u.get(), H->ws.w32[l].w.get(),
                                     st, lev.ext_ms);
  }
  *out = H.release();
  CPM_API_END
}

cpm_status cpm_hier_ext_tuning(cpm_hier h, int32_t level, int32_t* variant, double* ms) {
  CPM_API_BEGIN
  CPM_CHECK(h != nullptr, CPM_ERR_ARG, "hierarchy is NULL");
  CPM_CHECK(level >= 0 && level < (int)h->L.size(), CPM_ERR_ARG, "level out of range");
  const Level& lev = *h->L[level].lev;
  if (variant) *variant = lev.ext_variant;
  if (ms)
    for (int v = 0; v < 3; ++v) ms[v] = lev.ext_ms[v];
  CPM_API_END
}

cpm_status cpm_hier_info(cpm_hier h, int32_t* n_levels, int32_t level, int64_t* n_band) {
  CPM_API_BEGIN
  CPM_CHECK(h != nullptr, CPM_ERR_ARG, "hierarchy is NULL");
  if (n_levels) *n_levels = (int32_t)h->L.size();
  if (n_band) {
    CPM_CHECK(level >= 0 && level < (int)h->L.size(), CPM_ERR_ARG, "level out of range");
    *n_band = h->L[level].lev->nB;
  }
  CPM_API_END
}

cpm_status cpm_apply(cpm_hier h, int32_t level, int32_t prec, const void* u, void* Mu,
                     cpm_stream stream) {
  CPM_API_BEGIN
  CPM_CHECK(h != nullptr && u != nullptr && Mu != nullptr, CPM_ERR_ARG, "NULL argument");
  CPM_CHECK(level >= 0 && level < (int)h->L.size(), CPM_ERR_ARG, "level out of range");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == CPM_F64) {
    level_op<double>(h, h->ws, level, LAP_APPLY, nullptr, (const double*)u, (double*)Mu, nullptr, st);
  } else {
    CPM_CHECK(prec == CPM_F32, CPM_ERR_ARG, "unknown precision");
    level_op<float>(h, h->ws, level, LAP_APPLY, nullptr, (const float*)u, (float*)Mu, nullptr, st);
  }
  CPM_CUDA_TRY(cudaGetLastError());
  CPM_API_END
}

cpm_status cpm_extend(cpm_hier h, int32_t level, int32_t prec, const void* u, void* w,
                      int32_t with_ghost, cpm_stream stream) {
  CPM_API_BEGIN
  CPM_CHECK(h != nullptr && u != nullptr && w != nullptr, CPM_ERR_ARG, "NULL argument");
  CPM_CHECK(level >= 0 && level < (int)h->L.size(), CPM_ERR_ARG, "level out of range");
  cudaStream_t st = (cudaStream_t)stream;
  HLevel& lv = h->L[level];
  const int32_t np = with_ghost ? (int32_t)lv.lev->nplus() : lv.lev->nB;
  if (prec == CPM_F64) {
    launch_extend<double>(lv.view<double>(), (const double*)u, (double*)w, np, st);
  } else {
    CPM_CHECK(prec == CPM_F32, CPM_ERR_ARG, "unknown precision");
    launch_extend<float>(lv.view<float>(), (const float*)u, (float*)w, np, st);
  }
  CPM_CUDA_TRY(cudaGetLastError());
  CPM_API_END
}

int64_t cpm_kernel_launches(void) { return cpm::launches_total(); }

cpm_status cpm_smooth(cpm_hier h, int32_t level, int32_t prec, const void* f, void* u,
                      int32_t sweeps, cpm_stream stream) {
  CPM_API_BEGIN
  CPM_CHECK(h != nullptr && u != nullptr && f != nullptr, CPM_ERR_ARG, "NULL argument");
  CPM_CHECK(level >= 0 && level < (int)h->L.size(), CPM_ERR_ARG, "level out of range");
  CPM_CHECK(sweeps >= 0, CPM_ERR_ARG, "sweeps must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == CPM_F64)
    smooth<double>(h, h->ws, level, (const double*)f, (double*)u, sweeps, st);
  else {
    CPM_CHECK(prec == CPM_F32, CPM_ERR_ARG, "unknown precision");
    smooth<float>(h, h->ws, level, (const float*)f, (float*)u, sweeps, st);
  }
  CPM_CUDA_TRY(cudaGetLastError());
  CPM_API_END
}

cpm_status cpm_vcycle(cpm_hier h, int32_t prec, const void* f, void* u, cpm_stream stream) {
  CPM_API_BEGIN
  CPM_CHECK(h != nullptr && u != nullptr && f != nullptr, CPM_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == CPM_F64)
    vcycle_level<double>(h, h->ws, 0, (const double*)f, (double*)u, st);
  else {
    CPM_CHECK(prec == CPM_F32, CPM_ERR_ARG, "unknown precision");
    vcycle_level<float>(h, h->ws, 0, (const float*)f, (float*)u, st);
  }
  CPM_CUDA_TRY(cudaGetLastError());
  CPM_API_END
}

cpm_status cpm_residual(cpm_hier h, const double* f, const double* u, double* r, cpm_stream stream) {
  CPM_API_BEGIN
  CPM_CHECK(h != nullptr && u != nullptr && f != nullptr && r != nullptr, CPM_ERR_ARG, "NULL argument");
  outer_residual(h, h->ws, f, u, r, (cudaStream_t)stream, h->pair_resid);
  CPM_CUDA_TRY(cudaGetLastError());
  CPM_API_END
}

cpm_status cpm_residual_norms(cpm_hier h, const double* f, const double* u, double* rel_inf,
                              double* abs_l2, cpm_stream stream) {
  CPM_API_BEGIN
  CPM_CHECK(h != nullptr && u != nullptr && f != nullptr, CPM_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nB = h->L[0].lev->nB;
  Workspace& W = h->ws;
  launch_norm_partials<double>(f, nB, W.part.get(), st);
  launch_norm_final(W.part.get(), kNormBlocks, W.normf.get(), st);
  outer_residual(h, W, f, u, W.r64.get(), st, h->pair_resid);
  double hn[3], hf[3];
  CPM_CUDA_TRY(cudaMemcpyAsync(hn, W.norms, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaMemcpyAsync(hf, W.normf.get(), 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  if (rel_inf) *rel_inf = hf[0] > 0 ? hn[0] / hf[0] : hn[0];
  if (abs_l2) *abs_l2 = std::sqrt(hn[1]);
  CPM_API_END
}

cpm_status cpm_residual_norms_noalloc(cpm_hier h, const double* f, const double* u, double* norms,
                                      cpm_stream stream) {
  CPM_API_BEGIN
  CPM_CHECK(h != nullptr && u != nullptr && f != nullptr && norms != nullptr, CPM_ERR_ARG,
            "NULL argument");
  CPM_CHECK(h->opts.op_form == CPM_OP_MBR, CPM_ERR_ARG,
            "cpm_residual_norms_noalloc evaluates the CPM_OP_MBR operator only");
  const HLevel& lv = h->L[0];
  residual_norms_noalloc(lv.view<double>(), f, u, lv.c64.get(), h->c, norms, (cudaStream_t)stream);
  CPM_API_END
}

// Size of the rounding error of an outer residual in FP32 pairs, from the
// largest staged difference dmax = max |u - ref| (norms[3]): each extended
// value carries about 2^-48 dmax, and the stencil adds 2d + 1 of them with
// weights of total size (2d + 2d) / dx^2 + gamma = 6d / dx^2.  Measured errors
// are about 0.4 of 2^-48 dmax 6d / dx^2 (unit circle and sphere, dx = 1/32 ..
// 1/256, emulated; the GPU agrees at dx = 1/256); the estimate takes four times
// 2^-48 dmax 6d / dx^2, about ten times the error.
static double pair_error_estimate(const cpm_hier_s* h, double dmax) {
  const Level& l0 = *h->L[0].lev;
  return 4.0 * std::ldexp(dmax, -48) * 6.0 * l0.dim / (l0.dx * l0.dx);
}

// Whether an outer residual in FP32 pairs (relative size rel, the previous
// one prev, estimated rounding error est) is checked in FP64 on the same
// iterate: when it meets the tolerance only within the estimate, when it has
// reached the estimate, or when it has stopped falling (at most halved).
static bool pair_needs_check(double rel, double prev, double est, double tol, int it) {
  if (rel <= tol) return rel + est > tol;
  return rel <= est || (it > 0 && rel > 0.5 * prev);
}

// Pointwise FP64 check of the pair residual in W.r64 (iterate W.u_own): the
// points with |r_i| > thr (absolute) evaluated in FP64.  Returns the largest
// such |r_i|, or -1 if there were more than kCheckCap candidates.  Synchronous.
static double pointwise_check(cpm_hier_s* h, Workspace& W, double thr, cudaStream_t st) {
  const HLevel& lv = h->L[0];
  launch_pointwise_check(lv.view<double>(), W.u_own.get(), W.f_own.get(), lv.c64.get(), h->c,
                         W.r64.get(), thr, W.chk_list.get(), kCheckCap, W.chk_count.get(),
                         W.chk_max.get(), st);
  int32_t cnt = 0;
  unsigned long long mb = 0;
  CPM_CUDA_TRY(cudaMemcpyAsync(W.pinned + 5, W.chk_count.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaMemcpyAsync(W.pinned + 6, W.chk_max.get(), sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  std::memcpy(&cnt, W.pinned + 5, sizeof(cnt));
  std::memcpy(&mb, W.pinned + 6, sizeof(mb));
  if (cnt > kCheckCap) return -1.0;
  double m;
  std::memcpy(&m, &mb, sizeof(m));
  return m;
}

// Options with defaults filled in and checked.
static cpm_solve_opts solve_opts(const cpm_solve_opts* opts_in) {
  cpm_solve_opts o{};
  o.use_graph = 1;
  if (opts_in) o = *opts_in;
  if (!(o.tol > 0)) o.tol = 1e-10;
  if (o.inner_cycles <= 0) o.inner_cycles = 1;
  CPM_CHECK(o.inner_cycles <= 16, CPM_ERR_ARG, "inner_cycles must be <= 16");
  if (o.max_iter <= 0) o.max_iter = 100;
  CPM_CHECK(o.mode == CPM_SOLVE_F64 || o.mode == CPM_SOLVE_MIXED, CPM_ERR_ARG, "unknown mode");
  return o;
}

// Graph of one outer step of workspace W (captured on first use).
static void capture_outer_step(cpm_hier_s* h, Workspace& W, int idx, int mode, int inner,
                               cudaStream_t st) {
  cudaGraphExec_t& gx = W.graph[idx];
  if (gx && W.graph_inner[idx] != inner) {
    cudaGraphExecDestroy(gx);
    gx = nullptr;
  }
  if (gx) return;
  W.graph_inner[idx] = inner;
  cudaGraph_t g;
  CPM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  set_capturing(true);
  try {
    outer_step(h, W, mode, inner, st);
  } catch (...) {
    set_capturing(false);
    cudaStreamEndCapture(st, &g);
    throw;
  }
  set_capturing(false);
  CPM_CUDA_TRY(cudaStreamEndCapture(st, &g));
  size_t nn = 0;
  CPM_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  CPM_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &nn));
  int64_t nk = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    CPM_CUDA_TRY(cudaGraphNodeGetType(nd, &t));
    nk += t == cudaGraphNodeTypeKernel;
  }
  W.graph_kernels[idx] = nk;
  CPM_CUDA_TRY(cudaGraphInstantiate(&gx, g, 0));
  CPM_CUDA_TRY(cudaGraphDestroy(g));
}

// One complete solve with workspace W (synchronous); returns the status.
static cpm_status solve_ws(cpm_hier h, Workspace& W, const double* f, double* u,
                           const cpm_solve_opts* opts_in, cpm_solve_report* report, cpm_stream stream) {
  CPM_CHECK(h != nullptr && u != nullptr && f != nullptr, CPM_ERR_ARG, "NULL argument");
  const cpm_solve_opts o = solve_opts(opts_in);
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t us = (cudaStream_t)stream;
  cudaStream_t st = W.hs;
  const int64_t nB = h->L[0].lev->nB;
  CPM_CUDA_TRY(cudaEventRecord(W.ev, us));
  CPM_CUDA_TRY(cudaStreamWaitEvent(st, W.ev, 0));
  CPM_CUDA_TRY(cudaMemcpyAsync(W.f_own.get(), f, nB * sizeof(double), cudaMemcpyDeviceToDevice, st));
  W.pair = h->pair_resid;
  if (o.zero_init)
    CPM_CUDA_TRY(cudaMemsetAsync(W.u_own.get(), 0, nB * sizeof(double), st));
  else
    CPM_CUDA_TRY(cudaMemcpyAsync(W.u_own.get(), u, nB * sizeof(double), cudaMemcpyDeviceToDevice, st));
  launch_norm_partials<double>(W.f_own.get(), nB, W.part.get(), st);
  launch_norm_final(W.part.get(), kNormBlocks, W.normf.get(), st);
  CPM_CUDA_TRY(cudaMemcpyAsync(W.pinned + 4, W.normf.get(), 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (o.zero_init) {  // u = 0: the residual is f itself, and so are its norms
    CPM_CUDA_TRY(cudaMemcpyAsync(W.r64.get(), W.f_own.get(), nB * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st));
    CPM_CUDA_TRY(cudaMemcpyAsync(W.norms, W.normf.get(), 4 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  } else {
    outer_residual(h, W, W.f_own.get(), W.u_own.get(), W.r64.get(), st, W.pair);
  }
  CPM_CUDA_TRY(cudaMemcpyAsync(W.pinned, W.norms, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  const double fmax = W.pinned[4];
  // the maximum skips NaN (fmax), the sum of squares does not (it may still
  // overflow to infinity for a finite f, so only NaN is tested there)
  CPM_CHECK(std::isfinite(fmax) && !std::isnan(W.pinned[5]), CPM_ERR_ARG, "f is not finite");
  const double fn = fmax > 0 ? fmax : 1.0;
  CPM_CHECK(!o.learned || (o.mode == CPM_SOLVE_MIXED && h->mlp), CPM_ERR_ARG,
            "learned smoothing needs mode MIXED and cpm_hier_set_smoother");
  h->learned_active = false;
  int gi = o.mode;
  cpm_solve_report rep{};
  double rel = W.pinned[0] / fn, best = rel, prev = rel;
  cpm_status result = CPM_ERR_NOT_CONVERGED;
  int it = 0;
  // learned smoothing: iteration 0 runs plain Jacobi V-cycles and sets the
  // reference reduction factor; later iterations use the network until one
  // of them reduces the residual by a factor worse than 1.25 x that reference
  // (then plain Jacobi for the rest of the solve).
  bool learned_on = false;
  double ref_factor = 0.0, learned_log = 0.0;
  for (;; ++it) {
    if (W.pair) {
      rep.pair_floor = pair_error_estimate(h, W.pinned[3]) / fn;
      if (pair_needs_check(rel, prev, rep.pair_floor, o.tol, it)) {
        ++rep.f64_checks;
        // meets the tolerance within the estimate: only the points whose pair
        // residual lies within the estimate of the tolerance can violate it
        const double m = rel <= o.tol ? pointwise_check(h, W, (o.tol - rep.pair_floor) * fn, st) : -1.0;
        if (m >= 0.0 && m <= o.tol * fn) {
          rel = m / fn;
        } else {
          outer_residual(h, W, W.f_own.get(), W.u_own.get(), W.r64.get(), st, false);
          CPM_CUDA_TRY(cudaMemcpyAsync(W.pinned, W.norms, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
          CPM_CUDA_TRY(cudaStreamSynchronize(st));
          rel = W.pinned[0] / fn;
          if (!(rel <= o.tol)) W.pair = false;
        }
      }
    }
    if (it < CPM_MAX_HISTORY) rep.history[it] = rel;
    if (rel <= o.tol) { result = CPM_OK; break; }
    if (!std::isfinite(rel) || rel > 1e3 * best) { result = CPM_ERR_DIVERGED; break; }
    if (it >= o.max_iter) break;
    best = std::min(best, rel);
    if (o.learned && it == 1 && !rep.fallback) learned_on = true;
    h->learned_active = learned_on;
    gi = (learned_on ? 2 : o.mode) + (W.pair ? 3 : 0);
    if (o.fmg && it == 0) {
      outer_step(h, W, o.mode, o.inner_cycles, st, true);
    } else if (o.use_graph) {
      capture_outer_step(h, W, gi, o.mode, o.inner_cycles, st);
      CPM_CUDA_TRY(cudaGraphLaunch(W.graph[gi], st));
      count_launch(W.graph_kernels[gi]);
    } else {
      outer_step(h, W, o.mode, o.inner_cycles, st);
    }
    CPM_CUDA_TRY(cudaMemcpyAsync(W.pinned, W.norms, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CPM_CUDA_TRY(cudaStreamSynchronize(st));
    prev = rel;
    rel = W.pinned[0] / fn;
    // a reduction factor is judged only where the residual is well above the
    // pair rounding error (near it the factor says more about the rounding)
    const bool judged = !W.pair || rel > 2.0 * pair_error_estimate(h, W.pinned[3]) / fn;
    if (o.learned && judged) {
      const double fac = prev > 0 ? rel / prev : 0.0;
      if (it == 0) {
        ref_factor = fac;
      } else if (learned_on) {
        ++rep.learned_iters;
        learned_log += std::log(std::max(fac, 1e-300));
        rep.learned_worst = std::max(rep.learned_worst, fac);
        if (fac > 1.25 * ref_factor) {
          learned_on = false;
          rep.fallback = 1;
        }
      }
    }
  }
  h->learned_active = false;
  rep.jacobi_factor = ref_factor;
  rep.learned_factor = rep.learned_iters ? std::exp(learned_log / rep.learned_iters) : 0.0;
  CPM_CUDA_TRY(cudaMemcpyAsync(u, W.u_own.get(), nB * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CPM_CUDA_TRY(cudaEventRecord(W.ev, st));
  CPM_CUDA_TRY(cudaStreamWaitEvent(us, W.ev, 0));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  rep.iters = it;
  rep.converged = result == CPM_OK;
  rep.rel_residual = rel;
  rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (report) *report = rep;
  if (result != CPM_OK)
    cpm::set_last_error(result == CPM_ERR_DIVERGED ? "residual diverged" : "max_iter reached");
  return result;
}

cpm_status cpm_solve(cpm_hier h, const double* f, double* u, const cpm_solve_opts* opts_in,
                     cpm_solve_report* report, cpm_stream stream) {
  CPM_API_BEGIN
  CPM_CHECK(h != nullptr, CPM_ERR_ARG, "NULL argument");
  return solve_ws(h, h->ws, f, u, opts_in, report, stream);
  CPM_API_END
}

// ----------------------------------------------------------------- learned smoother
static double splitmix_normal(uint64_t& state) {
  auto next = [&]() {
    uint64_t z = (state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
  };
  const double u1 = ((next() >> 11) + 1.0) * (1.0 / 9007199254740993.0);
  const double u2 = (next() >> 11) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

cpm_status cpm_mlp_create(uint64_t seed, cpm_mlp* out) {
  CPM_API_BEGIN
  CPM_CHECK(out != nullptr, CPM_ERR_ARG, "NULL argument");
  *out = nullptr;
  std::unique_ptr<cpm_mlp_s> m(new cpm_mlp_s);
  std::vector<float> p(kNParams, 0.f);
  uint64_t st = seed;
  for (int k = 0; k < 31; ++k)
    for (int n = 0; n < 64; ++n) p[kOffW1 + k * 64 + n] = (float)(splitmix_normal(st) * std::sqrt(2.0 / 31));
  for (int q = 0; q < 64 * 64; ++q) p[kOffW2 + q] = (float)(splitmix_normal(st) * std::sqrt(2.0 / 64));
  for (int q = 0; q < 64; ++q) p[kOffW3 + q] = (float)(splitmix_normal(st) * std::sqrt(1.0 / 64));
  m->params.alloc(kNParams);
  m->m.alloc(kNParams);
  m->v.alloc(kNParams);
  CPM_CUDA_TRY(cudaMemcpy(m->params.get(), p.data(), kNParams * sizeof(float), cudaMemcpyHostToDevice));
  CPM_CUDA_TRY(cudaMemset(m->m.get(), 0, kNParams * sizeof(float)));
  CPM_CUDA_TRY(cudaMemset(m->v.get(), 0, kNParams * sizeof(float)));
  *out = m.release();
  CPM_API_END
}

cpm_status cpm_mlp_set_params(cpm_mlp m, const float* params, int32_t n) {
  CPM_API_BEGIN
  CPM_CHECK(m != nullptr && params != nullptr && n == kNParams, CPM_ERR_ARG, "bad arguments");
  CPM_CUDA_TRY(cudaMemcpy(m->params.get(), params, kNParams * sizeof(float), cudaMemcpyHostToDevice));
  CPM_CUDA_TRY(cudaMemset(m->m.get(), 0, kNParams * sizeof(float)));
  CPM_CUDA_TRY(cudaMemset(m->v.get(), 0, kNParams * sizeof(float)));
  m->step = 0;
  CPM_API_END
}

cpm_status cpm_mlp_get_params(cpm_mlp m, float* params, int32_t n) {
  CPM_API_BEGIN
  CPM_CHECK(m != nullptr && params != nullptr && n == kNParams, CPM_ERR_ARG, "bad arguments");
  CPM_CUDA_TRY(cudaDeviceSynchronize());
  CPM_CUDA_TRY(cudaMemcpy(params, m->params.get(), kNParams * sizeof(float), cudaMemcpyDeviceToHost));
  CPM_API_END
}

cpm_status cpm_mlp_destroy(cpm_mlp m) {
  CPM_API_BEGIN
  delete m;
  CPM_API_END
}

cpm_status cpm_hier_set_smoother(cpm_hier h, cpm_mlp m) {
  CPM_API_BEGIN
  CPM_CHECK(h != nullptr, CPM_ERR_ARG, "hierarchy is NULL");
  for (int g : {2, 5}) {  // the graphs with the learned smoother
    if (h->ws.graph[g]) {
      cudaGraphExecDestroy(h->ws.graph[g]);
      h->ws.graph[g] = nullptr;
    }
  }
  h->mlp = m;
  if (m && !h->mlpd) {
    CPM_CHECK(h->L[0].lev->dim == 3, CPM_ERR_ARG, "the learned smoother is for surfaces in 3-D");
    CPM_CHECK(h->opts.op_form == CPM_OP_MBR, CPM_ERR_ARG,
              "the learned smoother is trained on the CPM_OP_MBR operator");
    h->mlpd.reset(new MlpLevelData);
    h->mlpd->build(*h->L[0].lev, h->L[0].dM64.get(), h->ws.hs);
    CPM_CUDA_TRY(cudaStreamSynchronize(h->ws.hs));
  }
  CPM_API_END
}

cpm_status cpm_mlp_correction(cpm_hier h, const float* r, float* du, cpm_stream stream) {
  CPM_API_BEGIN
  CPM_CHECK(h != nullptr && r != nullptr && du != nullptr, CPM_ERR_ARG, "NULL argument");
  CPM_CHECK(h->mlp && h->mlpd, CPM_ERR_ARG, "no learned smoother set (cpm_hier_set_smoother)");
  const double dx = h->L[0].lev->dx;
  mlp_forward(h->mlp->params.get(), *h->mlpd, r, (float)(dx * dx), du, nullptr, nullptr,
              (cudaStream_t)stream);
  CPM_CUDA_TRY(cudaGetLastError());
  CPM_API_END
}

static void mlp_loss_grad_host(cpm_hier h, const float* r, cudaStream_t st) {
  CPM_CHECK(h != nullptr && r != nullptr, CPM_ERR_ARG, "NULL argument");
  CPM_CHECK(h->mlp && h->mlpd, CPM_ERR_ARG, "no learned smoother set (cpm_hier_set_smoother)");
  HLevel& lv = h->L[0];
  mlp_loss_grad(h->mlp->params.get(), *h->mlpd, lv.view<float>(), lv.c32.get(), (float)h->c, r,
                h->mlp->tb, st);
}

cpm_status cpm_mlp_loss_grad(cpm_hier h, const float* r, double* loss, float* grad, cpm_stream stream) {
  CPM_API_BEGIN
  cudaStream_t st = (cudaStream_t)stream;
  mlp_loss_grad_host(h, r, st);
  double l2[2];
  CPM_CUDA_TRY(cudaMemcpyAsync(l2, h->mlp->tb.loss.get(), sizeof(l2), cudaMemcpyDeviceToHost, st));
  if (grad)
    CPM_CUDA_TRY(cudaMemcpyAsync(grad, h->mlp->tb.grad.get(), kNParams * sizeof(float),
                                 cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  if (loss) *loss = l2[1] > 0 ? l2[0] / l2[1] : 0.0;
  CPM_API_END
}

cpm_status cpm_mlp_train_step(cpm_hier h, const float* r, float lr, double* loss, cpm_stream stream) {
  CPM_API_BEGIN
  CPM_CHECK(lr > 0 && std::isfinite(lr), CPM_ERR_ARG, "lr must be positive");
  cudaStream_t st = (cudaStream_t)stream;
  mlp_loss_grad_host(h, r, st);
  cpm_mlp m = h->mlp;
  ++m->step;
  mlp_adam(m->params.get(), m->tb.grad.get(), m->m.get(), m->v.get(), m->step, lr, st);
  CPM_CUDA_TRY(cudaGetLastError());
  if (loss) {
    double l2[2];
    CPM_CUDA_TRY(cudaMemcpyAsync(l2, m->tb.loss.get(), sizeof(l2), cudaMemcpyDeviceToHost, st));
    CPM_CUDA_TRY(cudaStreamSynchronize(st));
    *loss = l2[1] > 0 ? l2[0] / l2[1] : 0.0;
  }
  CPM_API_END
}

cpm_status cpm_mlp_train(cpm_mlp m, const cpm_train_set* set, const cpm_train_opts* opts_in,
                         cpm_train_report* report, cpm_stream stream) {
  CPM_API_BEGIN
  CPM_CHECK(m != nullptr && set != nullptr && set->n_fields > 0 && set->hier != nullptr &&
                set->r != nullptr,
            CPM_ERR_ARG, "cpm_mlp_train: NULL or empty training set");
  cpm_train_opts o{};
  if (opts_in) o = *opts_in;
  if (o.steps <= 0) o.steps = 400;
  if (!(o.lr > 0)) o.lr = 2e-3f;
  if (!(o.lr_final > 0)) o.lr_final = o.lr;
  CPM_CHECK(std::isfinite(o.lr) && std::isfinite(o.lr_final), CPM_ERR_ARG, "learning rate not finite");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)stream;
  const int nf = set->n_fields;
  int32_t maxB = 0;
  int64_t maxP = 0;
  for (int k = 0; k < nf; ++k) {
    cpm_hier h = set->hier[k];
    CPM_CHECK(h != nullptr && set->r[k] != nullptr, CPM_ERR_ARG, "cpm_mlp_train: NULL field");
    CPM_CHECK(h->L[0].lev->dim == 3, CPM_ERR_ARG, "the learned smoother is for surfaces in 3-D");
    if (h->mlp != m || !h->mlpd) {
      const cpm_status sm = cpm_hier_set_smoother(h, m);
      if (sm != CPM_OK) return sm;
    }
    maxB = std::max(maxB, h->L[0].lev->nB);
    maxP = std::max(maxP, h->L[0].lev->nplus());
  }
  if (o.reset) {
    CPM_CUDA_TRY(cudaMemsetAsync(m->m.get(), 0, kNParams * sizeof(float), st));
    CPM_CUDA_TRY(cudaMemsetAsync(m->v.get(), 0, kNParams * sizeof(float), st));
    m->step = 0;
  }
  m->tb.ensure(maxB, maxP);
  // the fields scaled by 1 / max|r| into FP32
  std::vector<DBuf<float>> f32(nf);
  DBuf<double> norms(4 * (size_t)nf), part(2 * (size_t)kNormBlocks);
  for (int k = 0; k < nf; ++k) {
    const int32_t nB = set->hier[k]->L[0].lev->nB;
    f32[k].alloc(nB);
    launch_norm_partials<double>(set->r[k], nB, part.get(), st);
    launch_norm_final(part.get(), kNormBlocks, norms.get() + 4 * (size_t)k, st);
    launch_scale_to_f32(set->r[k], norms.get() + 4 * (size_t)k, f32[k].get(), nB, st);
  }
  std::vector<double> hn(4 * (size_t)nf);
  CPM_CUDA_TRY(cudaMemcpyAsync(hn.data(), norms.get(), hn.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  for (int k = 0; k < nf; ++k)
    CPM_CHECK(std::isfinite(hn[4 * (size_t)k]) && hn[4 * (size_t)k] > 0, CPM_ERR_ARG,
              "cpm_mlp_train: a field is zero or not finite");
  auto mean_loss = [&]() {
    double acc = 0.0;
    for (int k = 0; k < nf; ++k) {
      mlp_loss_grad_host(set->hier[k], f32[k].get(), st);
      double l2[2];
      CPM_CUDA_TRY(cudaMemcpyAsync(l2, m->tb.loss.get(), sizeof(l2), cudaMemcpyDeviceToHost, st));
      CPM_CUDA_TRY(cudaStreamSynchronize(st));
      acc += l2[1] > 0 ? l2[0] / l2[1] : 0.0;
    }
    return acc / nf;
  };
  const double loss_first = mean_loss();
  const int per = std::max(1, o.steps / nf);
  int step = 0, k = 0;
  while (step < o.steps) {
    for (int j = 0; j < per && step < o.steps; ++j, ++step) {
      const float frac = o.steps > 1 ? (float)step / (float)(o.steps - 1) : 0.f;
      const float lr = o.lr + (o.lr_final - o.lr) * frac;
      mlp_loss_grad_host(set->hier[k], f32[k].get(), st);
      ++m->step;
      mlp_adam(m->params.get(), m->tb.grad.get(), m->m.get(), m->v.get(), m->step, lr, st);
    }
    k = (k + 1) % nf;
  }
  CPM_CUDA_TRY(cudaGetLastError());
  const double loss_last = mean_loss();
  if (report) {
    report->steps = o.steps;
    report->n_fields = nf;
    report->loss_first = loss_first;
    report->loss_last = loss_last;
    report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  CPM_API_END
}

static const char kMlpMagic[8] = {'C', 'P', 'M', 'M', 'L', 'P', '0', '1'};

cpm_status cpm_mlp_save(cpm_mlp m, const char* path) {
  CPM_API_BEGIN
  CPM_CHECK(m != nullptr && path != nullptr, CPM_ERR_ARG, "NULL argument");
  std::vector<float> buf(3 * (size_t)kNParams);
  CPM_CUDA_TRY(cudaDeviceSynchronize());
  CPM_CUDA_TRY(cudaMemcpy(buf.data(), m->params.get(), kNParams * sizeof(float), cudaMemcpyDeviceToHost));
  CPM_CUDA_TRY(cudaMemcpy(buf.data() + kNParams, m->m.get(), kNParams * sizeof(float),
                          cudaMemcpyDeviceToHost));
  CPM_CUDA_TRY(cudaMemcpy(buf.data() + 2 * kNParams, m->v.get(), kNParams * sizeof(float),
                          cudaMemcpyDeviceToHost));
  FILE* fp = std::fopen(path, "wb");
  CPM_CHECK(fp != nullptr, CPM_ERR_ARG, std::string("cannot open ") + path + " for writing");
  const int32_t n = kNParams;
  const int64_t step = m->step;
  bool ok = std::fwrite(kMlpMagic, 1, 8, fp) == 8 && std::fwrite(&n, sizeof(n), 1, fp) == 1 &&
            std::fwrite(&step, sizeof(step), 1, fp) == 1 &&
            std::fwrite(buf.data(), sizeof(float), buf.size(), fp) == buf.size();
  ok = (std::fclose(fp) == 0) && ok;
  CPM_CHECK(ok, CPM_ERR_ARG, std::string("short write to ") + path);
  CPM_API_END
}

cpm_status cpm_mlp_load(const char* path, cpm_mlp* out) {
  CPM_API_BEGIN
  CPM_CHECK(path != nullptr && out != nullptr, CPM_ERR_ARG, "NULL argument");
  *out = nullptr;
  FILE* fp = std::fopen(path, "rb");
  CPM_CHECK(fp != nullptr, CPM_ERR_ARG, std::string("cannot open ") + path);
  char magic[8];
  int32_t n = 0;
  int64_t step = 0;
  std::vector<float> buf(3 * (size_t)kNParams);
  bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, kMlpMagic, 8) == 0 &&
            std::fread(&n, sizeof(n), 1, fp) == 1 && n == kNParams &&
            std::fread(&step, sizeof(step), 1, fp) == 1 && step >= 0 &&
            std::fread(buf.data(), sizeof(float), buf.size(), fp) == buf.size();
  std::fclose(fp);
  CPM_CHECK(ok, CPM_ERR_ARG, std::string(path) + " is not a network written by cpm_mlp_save");
  cpm_mlp m = nullptr;
  const cpm_status cs = cpm_mlp_create(0, &m);
  if (cs != CPM_OK) return cs;
  std::unique_ptr<cpm_mlp_s> guard(m);
  CPM_CUDA_TRY(cudaMemcpy(m->params.get(), buf.data(), kNParams * sizeof(float), cudaMemcpyHostToDevice));
  CPM_CUDA_TRY(cudaMemcpy(m->m.get(), buf.data() + kNParams, kNParams * sizeof(float),
                          cudaMemcpyHostToDevice));
  CPM_CUDA_TRY(cudaMemcpy(m->v.get(), buf.data() + 2 * kNParams, kNParams * sizeof(float),
                          cudaMemcpyHostToDevice));
  m->step = step;
  *out = guard.release();
  CPM_API_END
}

cpm_status cpm_hier_destroy(cpm_hier h) {
  CPM_API_BEGIN
  delete h;
  CPM_API_END
}

}  // extern "C"

// ----------------------------------------------------------------- batches
struct cpm_batch_s {
  std::vector<cpm_hier> H;       // per system
  std::vector<std::unique_ptr<Workspace>> W;
  int32_t n_rhs = 1;
  std::string cache;
  cpm::DBuf<double> norms_all;   // 4 per system
  double* host_norms = nullptr;  // pinned, 4 per system
  cudaStream_t ms = nullptr;
  std::vector<cudaStream_t> fs;  // branch streams
  cudaEvent_t ev_fork = nullptr, t0 = nullptr, t1 = nullptr;
  std::vector<cudaEvent_t> ev_join;
  cudaGraphExec_t graph = nullptr;
  int graph_k = 0, graph_mode = -1, graph_inner = -1;
  std::vector<int> graph_sys;    // systems in the current graph
  int64_t pair_epoch = 0;        // bumped when a system's outer residual leaves FP32 pairs
  int64_t graph_epoch = -1;      // pair_epoch when the graph was captured
  int64_t graph_kernels = 0;
  int32_t chosen = 0;
  double tune_ms[8] = {0};
  ~cpm_batch_s() {
    if (graph) cudaGraphExecDestroy(graph);
    for (auto e : ev_join) cudaEventDestroy(e);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    for (auto s : fs) cudaStreamDestroy(s);
    if (ms) cudaStreamDestroy(ms);
    if (host_norms) cudaFreeHost(host_norms);
  }
};

namespace cpm {

static constexpr int kMaxBranches = 32;

// Tune-cache key: the batch shape (number of systems and the finest band
// sizes), so a cached concurrency is reused only for the same workload.
static std::string batch_key(const cpm_batch_s& b) {
  uint64_t h = 1469598103934665603ull;
  for (auto* hh : b.H) {
    h ^= (uint64_t)hh->L[0].lev->nB;
    h *= 1099511628211ull;
  }
  return "n" + std::to_string(b.H.size()) + "_" + std::to_string(h);
}

static int cache_lookup(const cpm_batch_s& b) {
  if (b.cache.empty()) return 0;
  FILE* fp = std::fopen(b.cache.c_str(), "r");
  if (!fp) return 0;
  char key[256];
  int k = 0, found = 0;
  const std::string want = batch_key(b);
  while (std::fscanf(fp, "%255s %d", key, &k) == 2)
    if (want == key && k >= 1 && k <= kMaxBranches) found = k;
  std::fclose(fp);
  return found;
}

static void cache_store(const cpm_batch_s& b, int k) {
  if (b.cache.empty()) return;
  FILE* fp = std::fopen(b.cache.c_str(), "a");
  if (!fp) return;
  std::fprintf(fp, "%s %d\n", batch_key(b).c_str(), k);
  std::fclose(fp);
}

// Lockstep groups among the systems in sys: systems of one hierarchy, at
// most kMaxGroup per group.
static std::vector<std::vector<int>> make_groups(const cpm_batch_s& b, const std::vector<int>& sys) {
  std::vector<std::vector<int>> groups;
  std::vector<int> rest(sys);
  while (!rest.empty()) {
    std::vector<int> grp, other;
    for (int s : rest)
      (b.H[s] == b.H[rest[0]] && (int)grp.size() < kMaxGroup ? grp : other).push_back(s);
    groups.push_back(grp);
    rest.swap(other);
  }
  return groups;
}

static int count_groups(const cpm_batch_s& b, const std::vector<int>& sys) {
  return (int)make_groups(b, sys).size();
}

// Graph of one outer iteration of the systems in sys on K concurrent
// branches.  Systems of the same hierarchy form lockstep groups (up to
// kMaxGroup, one coarse-inverse pass for all of them); groups go to branches
// largest first, each to the branch with the least work so far.
static void capture_batch(cpm_batch_s& b, const std::vector<int>& sys, int K, int mode, int inner) {
  if (b.graph && b.graph_k == K && b.graph_mode == mode && b.graph_inner == inner && b.graph_sys == sys &&
      b.graph_epoch == b.pair_epoch)
    return;
  if (b.graph) {
    cudaGraphExecDestroy(b.graph);
    b.graph = nullptr;
  }
  std::vector<std::vector<int>> groups = make_groups(b, sys);
  auto work = [&](const std::vector<int>& g) { return (double)b.H[g[0]]->L[0].lev->nB * g.size(); };
  std::stable_sort(groups.begin(), groups.end(),
                   [&](const std::vector<int>& x, const std::vector<int>& y) { return work(x) > work(y); });
  std::vector<std::vector<int>> branch(K);  // group indices per branch
  std::vector<double> load(K, 0.0);
  for (size_t j = 0; j < groups.size(); ++j) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    branch[k].push_back((int)j);
    load[k] += work(groups[j]);
  }
  cudaGraph_t g;
  CPM_CUDA_TRY(cudaStreamBeginCapture(b.ms, cudaStreamCaptureModeThreadLocal));
  set_capturing(true);
  try {
    CPM_CUDA_TRY(cudaEventRecord(b.ev_fork, b.ms));
    for (int k = 0; k < K; ++k) CPM_CUDA_TRY(cudaStreamWaitEvent(b.fs[k], b.ev_fork, 0));
    for (int k = 0; k < K; ++k)
      for (int j : branch[k]) {
        Workspace* ws[kMaxGroup];
        const std::vector<int>& g = groups[j];
        for (size_t q = 0; q < g.size(); ++q) ws[q] = b.W[g[q]].get();
        outer_step(b.H[g[0]], ws, (int)g.size(), mode, inner, b.fs[k]);
      }
    for (int k = 0; k < K; ++k) {
      CPM_CUDA_TRY(cudaEventRecord(b.ev_join[k], b.fs[k]));
      CPM_CUDA_TRY(cudaStreamWaitEvent(b.ms, b.ev_join[k], 0));
    }
  } catch (...) {
    set_capturing(false);
    cudaStreamEndCapture(b.ms, &g);
    throw;
  }
  set_capturing(false);
  CPM_CUDA_TRY(cudaStreamEndCapture(b.ms, &g));
  size_t nn = 0;
  CPM_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  CPM_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &nn));
  int64_t nk = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    CPM_CUDA_TRY(cudaGraphNodeGetType(nd, &t));
    nk += t == cudaGraphNodeTypeKernel;
  }
  b.graph_kernels = nk;
  CPM_CUDA_TRY(cudaGraphInstantiate(&b.graph, g, 0));
  CPM_CUDA_TRY(cudaGraphDestroy(g));
  b.graph_k = K;
  b.graph_epoch = b.pair_epoch;
  b.graph_mode = mode;
  b.graph_inner = inner;
  b.graph_sys = sys;
}

}  // namespace cpm

extern "C" {

cpm_status cpm_build_batch(const cpm_hier* hiers, int32_t n_hier, int32_t n_rhs,
                           const char* tune_cache, cpm_batch* out) {
  CPM_API_BEGIN
  CPM_CHECK(hiers != nullptr && out != nullptr && n_hier > 0 && n_rhs > 0 &&
                (int64_t)n_hier * n_rhs <= CPM_BATCH_MAX_SYSTEMS,
            CPM_ERR_ARG, "bad batch arguments");
  *out = nullptr;
  std::unique_ptr<cpm_batch_s> b(new cpm_batch_s);
  b->n_rhs = n_rhs;
  if (tune_cache) b->cache = tune_cache;
  const int ns = n_hier * n_rhs;
  b->norms_all.alloc(4 * (size_t)ns);
  CPM_CUDA_TRY(cudaMallocHost(&b->host_norms, 4 * sizeof(double) * ns));
  for (int i = 0; i < n_hier; ++i) {
    CPM_CHECK(hiers[i] != nullptr, CPM_ERR_ARG, "NULL hierarchy");
    for (int k = 0; k < n_rhs; ++k) {
      const int s = i * n_rhs + k;
      b->H.push_back(hiers[i]);
      b->W.emplace_back(new Workspace);
      alloc_workspace(*hiers[i], *b->W.back(), b->norms_all.get() + 4 * (size_t)s);
    }
  }
  CPM_CUDA_TRY(cudaStreamCreateWithFlags(&b->ms, cudaStreamNonBlocking));
  b->fs.resize(kMaxBranches);
  b->ev_join.resize(kMaxBranches);
  for (int k = 0; k < kMaxBranches; ++k) {
    CPM_CUDA_TRY(cudaStreamCreateWithFlags(&b->fs[k], cudaStreamNonBlocking));
    CPM_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming));
  }
  CPM_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
  CPM_CUDA_TRY(cudaEventCreate(&b->t0));
  CPM_CUDA_TRY(cudaEventCreate(&b->t1));
  *out = b.release();
  CPM_API_END
}

cpm_status cpm_solve_batch(cpm_batch b, const double* const* f, double* const* u,
                           const cpm_solve_opts* opts_in, cpm_solve_report* reports,
                           cpm_stream stream) {
  CPM_API_BEGIN
  CPM_CHECK(b != nullptr && f != nullptr && u != nullptr, CPM_ERR_ARG, "NULL argument");
  const cpm_solve_opts o = solve_opts(opts_in);
  CPM_CHECK(!o.learned, CPM_ERR_ARG, "learned smoothing is not available in batches");
  CPM_CHECK(!o.fmg, CPM_ERR_ARG, "full multigrid is not available in batches");
  const int ns = (int)b->H.size();
  for (int s = 0; s < ns; ++s)
    CPM_CHECK(f[s] != nullptr && u[s] != nullptr, CPM_ERR_ARG, "NULL vector in batch");
  const auto tstart = std::chrono::steady_clock::now();
  cudaStream_t us = (cudaStream_t)stream;
  CPM_CUDA_TRY(cudaEventRecord(b->ev_fork, us));
  CPM_CUDA_TRY(cudaStreamWaitEvent(b->ms, b->ev_fork, 0));
  for (int k = 0; k < kMaxBranches; ++k) CPM_CUDA_TRY(cudaStreamWaitEvent(b->fs[k], b->ev_fork, 0));
  // copies in, norms of f and the initial residuals, spread over the branch streams
  DBuf<double> fn_all(4 * (size_t)ns);
  for (int s = 0; s < ns; ++s) {
    Workspace& W = *b->W[s];
    cudaStream_t st = b->fs[s % kMaxBranches];
    const int64_t nB = b->H[s]->L[0].lev->nB;
    CPM_CUDA_TRY(cudaMemcpyAsync(W.f_own.get(), f[s], nB * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (W.pair != b->H[s]->pair_resid) ++b->pair_epoch;
    W.pair = b->H[s]->pair_resid;
    if (o.zero_init)
      CPM_CUDA_TRY(cudaMemsetAsync(W.u_own.get(), 0, nB * sizeof(double), st));
    else
      CPM_CUDA_TRY(cudaMemcpyAsync(W.u_own.get(), u[s], nB * sizeof(double), cudaMemcpyDeviceToDevice, st));
    launch_norm_partials<double>(W.f_own.get(), nB, W.part.get(), st);
    launch_norm_final(W.part.get(), kNormBlocks, fn_all.get() + 4 * (size_t)s, st);
    if (o.zero_init) {  // u = 0: the residual is f itself, and so are its norms
      CPM_CUDA_TRY(cudaMemcpyAsync(W.r64.get(), W.f_own.get(), nB * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
      CPM_CUDA_TRY(cudaMemcpyAsync(W.norms, fn_all.get() + 4 * (size_t)s, 4 * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
    } else {
      outer_residual(b->H[s], W, W.f_own.get(), W.u_own.get(), W.r64.get(), st, W.pair);
    }
  }
  for (int k = 0; k < kMaxBranches; ++k) {
    CPM_CUDA_TRY(cudaEventRecord(b->ev_join[k], b->fs[k]));
    CPM_CUDA_TRY(cudaStreamWaitEvent(b->ms, b->ev_join[k], 0));
  }
  std::vector<double> hf(4 * (size_t)ns);
  CPM_CUDA_TRY(cudaMemcpyAsync(hf.data(), fn_all.get(), hf.size() * sizeof(double), cudaMemcpyDeviceToHost,
                               b->ms));
  CPM_CUDA_TRY(cudaMemcpyAsync(b->host_norms, b->norms_all.get(), 4 * sizeof(double) * ns,
                               cudaMemcpyDeviceToHost, b->ms));
  CPM_CUDA_TRY(cudaStreamSynchronize(b->ms));
  std::vector<cpm_solve_report> rep(ns);
  std::vector<double> fmax(ns), rel(ns), best(ns), prev(ns);
  std::vector<int> done(ns, 0);
  for (int s = 0; s < ns; ++s) {
    CPM_CHECK(std::isfinite(hf[4 * (size_t)s]) && !std::isnan(hf[4 * (size_t)s + 1]), CPM_ERR_ARG,
              "f is not finite");
    fmax[s] = hf[4 * (size_t)s] > 0 ? hf[4 * (size_t)s] : 1.0;
    rel[s] = best[s] = prev[s] = b->host_norms[4 * (size_t)s] / fmax[s];
  }
  // autotuner: the first outer iterations try K = 1, 2, 4, ... concurrent
  // branches (each a real iteration of every active system)
  std::vector<int> cand, all_systems(ns);
  for (int s = 0; s < ns; ++s) all_systems[s] = s;
  if (b->chosen == 0) b->chosen = cache_lookup(*b);
  if (b->chosen == 0)
    for (int k = 1; k <= std::min(count_groups(*b, all_systems), kMaxBranches); k *= 2) cand.push_back(k);
  size_t ci = 0;
  double best_ms = 1e300;
  int best_k = b->chosen;
  cpm_status result = CPM_OK;
  std::vector<int> active, in_graph;
  int it = 0;
  std::vector<int> check;
  for (;; ++it) {
    // FP64 check of residuals in FP32 pairs that meet the tolerance or have
    // stopped falling (as in cpm_solve); a system whose check misses the
    // tolerance continues with FP64 residuals
    check.clear();
    for (int s = 0; s < ns; ++s) {
      if (done[s] || !b->W[s]->pair) continue;
      rep[s].pair_floor = pair_error_estimate(b->H[s], b->host_norms[4 * (size_t)s + 3]) / fmax[s];
      if (pair_needs_check(rel[s], prev[s], rep[s].pair_floor, o.tol, it)) check.push_back(s);
    }
    if (!check.empty()) {
      // a residual that meets the tolerance within the estimate: pointwise
      // check first (as in cpm_solve); the others get the full FP64 residual
      std::vector<int> full;
      for (int s : check) {
        Workspace& W = *b->W[s];
        if (rel[s] <= o.tol) {
          const double m = pointwise_check(b->H[s], W, (o.tol - rep[s].pair_floor) * fmax[s], b->ms);
          if (m >= 0.0 && m <= o.tol * fmax[s]) {
            ++rep[s].f64_checks;
            rel[s] = m / fmax[s];
            continue;
          }
        }
        full.push_back(s);
      }
      check.swap(full);
    }
    if (!check.empty()) {
      for (int s : check) {
        Workspace& W = *b->W[s];
        outer_residual(b->H[s], W, W.f_own.get(), W.u_own.get(), W.r64.get(), b->ms, false);
      }
      CPM_CUDA_TRY(cudaMemcpyAsync(b->host_norms, b->norms_all.get(), 4 * sizeof(double) * ns,
                                   cudaMemcpyDeviceToHost, b->ms));
      CPM_CUDA_TRY(cudaStreamSynchronize(b->ms));
      for (int s : check) {
        rel[s] = b->host_norms[4 * (size_t)s] / fmax[s];
        ++rep[s].f64_checks;
        if (!(rel[s] <= o.tol)) {
          b->W[s]->pair = false;
          ++b->pair_epoch;
        }
      }
    }
    bool diverged = false;
    active.clear();
    for (int s = 0; s < ns; ++s) {
      if (done[s]) continue;
      if (it < CPM_MAX_HISTORY) rep[s].history[it] = rel[s];
      rep[s].iters = it;
      rep[s].rel_residual = rel[s];
      if (rel[s] <= o.tol) {
        // the converged iterate is the result, whatever later iterations of
        // the other systems do to this workspace
        done[s] = 1;
        rep[s].converged = 1;
        CPM_CUDA_TRY(cudaMemcpyAsync(u[s], b->W[s]->u_own.get(), b->H[s]->L[0].lev->nB * sizeof(double),
                                     cudaMemcpyDeviceToDevice, b->ms));
        continue;
      }
      if (!std::isfinite(rel[s]) || rel[s] > 1e3 * best[s]) diverged = true;
      best[s] = std::min(best[s], rel[s]);
      active.push_back(s);
    }
    if (active.empty()) break;
    if (diverged) { result = CPM_ERR_DIVERGED; break; }
    if (it >= o.max_iter) { result = CPM_ERR_NOT_CONVERGED; break; }
    // the graph covers a superset of the active systems; it is re-captured
    // over the active ones once they are at most half of it
    if (in_graph.empty() || 2 * active.size() <= in_graph.size()) in_graph = active;
    const int K = ci < cand.size() ? cand[ci] : (best_k > 0 ? best_k : 1);
    capture_batch(*b, in_graph, std::min<int>(K, count_groups(*b, in_graph)), o.mode, o.inner_cycles);
    CPM_CUDA_TRY(cudaEventRecord(b->t0, b->ms));
    CPM_CUDA_TRY(cudaGraphLaunch(b->graph, b->ms));
    CPM_CUDA_TRY(cudaEventRecord(b->t1, b->ms));
    count_launch(b->graph_kernels);
    CPM_CUDA_TRY(cudaMemcpyAsync(b->host_norms, b->norms_all.get(), 4 * sizeof(double) * ns,
                                 cudaMemcpyDeviceToHost, b->ms));
    CPM_CUDA_TRY(cudaStreamSynchronize(b->ms));
    if (ci < cand.size()) {
      // systems converge during the tuning iterations, so each candidate's
      // time is scaled to the whole batch by the band points its graph covered
      float ms = 0.f;
      CPM_CUDA_TRY(cudaEventElapsedTime(&ms, b->t0, b->t1));
      double all = 0.0, covered = 0.0;
      for (int s = 0; s < ns; ++s) all += (double)b->H[s]->L[0].lev->nB;
      for (int s : in_graph) covered += (double)b->H[s]->L[0].lev->nB;
      const double scaled = covered > 0.0 ? ms * all / covered : ms;
      int slot = 0;
      while ((1 << slot) < K && slot < 7) ++slot;
      b->tune_ms[slot] = scaled;
      if (scaled < best_ms) { best_ms = scaled; best_k = K; }
      if (++ci == cand.size()) {
        b->chosen = best_k;
        cache_store(*b, best_k);
      }
    }
    for (int s : in_graph) {
      prev[s] = rel[s];
      rel[s] = b->host_norms[4 * (size_t)s] / fmax[s];
    }
  }
  if (result != CPM_OK)
    for (int s = 0; s < ns; ++s)
      if (!done[s])
        CPM_CUDA_TRY(cudaMemcpyAsync(u[s], b->W[s]->u_own.get(), b->H[s]->L[0].lev->nB * sizeof(double),
                                     cudaMemcpyDeviceToDevice, b->ms));
  if (b->chosen == 0 && best_k > 0) b->chosen = best_k;
  CPM_CUDA_TRY(cudaEventRecord(b->ev_fork, b->ms));
  CPM_CUDA_TRY(cudaStreamWaitEvent(us, b->ev_fork, 0));
  CPM_CUDA_TRY(cudaStreamSynchronize(b->ms));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - tstart).count();
  if (reports)
    for (int s = 0; s < ns; ++s) {
      rep[s].seconds = secs;
      reports[s] = rep[s];
    }
  if (result != CPM_OK) {
    cpm::set_last_error(result == CPM_ERR_DIVERGED ? "a system of the batch diverged"
                                                   : "max_iter reached before every system converged");
    return result;
  }
  CPM_API_END
}

cpm_status cpm_batch_info(cpm_batch b, int32_t* concurrency, double* tune_ms) {
  CPM_API_BEGIN
  CPM_CHECK(b != nullptr, CPM_ERR_ARG, "NULL argument");
  if (concurrency) *concurrency = b->chosen;
  if (tune_ms)
    for (int q = 0; q < 8; ++q) tune_ms[q] = b->tune_ms[q];
  CPM_API_END
}

cpm_status cpm_batch_destroy(cpm_batch b) {
  CPM_API_BEGIN
  delete b;
  CPM_API_END
}

}  // extern "C"
