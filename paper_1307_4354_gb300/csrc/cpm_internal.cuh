// Internal declarations of the closest-point multigrid library (sm_103a).
//
// Data layout in HBM (one "level" = one grid spacing dx):
//   * Bricks of 4x4x4 grid nodes (4x4 in 2-D).  Bricks that hold band or
//     ghost nodes are stored in Morton order of their brick coordinates.
//   * Band points B (|x - cp(x)|^2 <= lambda^2 dx^2) come first, brick by
//     brick, nodes inside a brick in x-fastest order; the ghost ring G (the
//     Laplacian neighbours of B outside B) follows in the same brick order.
//     Unknowns u, f, r live on B (length nB); the extension w = E u lives on
//     B+ = B then G (length nB + nG) so that w[i] and u[i] share an index.
//   * A node (x, y, z) is located through a dense brick map
//     (brick coordinates -> brick index) and per-brick 64-bit occupancy
//     masks: index = start + popcount(mask & (bit - 1)).
//   * Per point of B+: one 64-bit key (grid coordinates, 16 bits each, and
//     the offset of the cubic stencil base from the node, 4 bits each) and
//     the fractional position of cp inside the stencil cell (SoA, FP64 and
//     an FP32 copy).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/cpm.h"

namespace cpm {

// ----------------------------------------------------------------- errors
struct Error {
  cpm_status status;
  std::string msg;
};
void set_last_error(const std::string& msg);

#define CPM_CUDA_TRY(expr)                                                            \
  do {                                                                                \
    cudaError_t e_ = (expr);                                                          \
    if (e_ != cudaSuccess)                                                            \
      throw ::cpm::Error{CPM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define CPM_CHECK(cond, status, msg)                 \
  do {                                               \
    if (!(cond)) throw ::cpm::Error{(status), (msg)}; \
  } while (0)

// ----------------------------------------------------------------- device buffer
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  explicit DBuf(size_t count) { alloc(count); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    release();
    n = count;
    if (count) {
      cudaError_t e = cudaMalloc(&p, count * sizeof(T));
      if (e != cudaSuccess) {
        p = nullptr;
        n = 0;
        throw Error{CPM_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
      }
    }
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  T* get() const { return p; }
};

// ----------------------------------------------------------------- key packing
// key = x | y << 16 | z << 32 | (ox + 8) << 48 | (oy + 8) << 52 | (oz + 8) << 56
// (o = cubic stencil base - node coordinate, in [-8, 7]).
__host__ __device__ inline int key_x(uint64_t k) { return (int)(k & 0xffffu); }
__host__ __device__ inline int key_y(uint64_t k) { return (int)((k >> 16) & 0xffffu); }
__host__ __device__ inline int key_z(uint64_t k) { return (int)((k >> 32) & 0xffffu); }
__host__ __device__ inline int key_ox(uint64_t k) { return (int)((k >> 48) & 15u) - 8; }
__host__ __device__ inline int key_oy(uint64_t k) { return (int)((k >> 52) & 15u) - 8; }
__host__ __device__ inline int key_oz(uint64_t k) { return (int)((k >> 56) & 15u) - 8; }

// ----------------------------------------------------------------- brick records
// Per brick, the occupancy masks and starts of the brick itself (slot 0) and
// of its face neighbours (slots 1..6: -x, +x, -y, +y, -z, +z; zero masks where
// there is none), so that a stencil pass finds every Laplacian neighbour with
// loads addressed by the brick number alone.
struct BrickRec {
  uint64_t bm[7], gm[7];
  int32_t bs[7], gs[7];
};

// ----------------------------------------------------------------- brick view
// Plain-pointer view of a level's brick tables, passed by value to kernels.
struct BrickView {
  const int32_t* map;     // nbx*nby*nbz -> brick index or -1
  const uint64_t* bmask;  // band occupancy
  const uint64_t* gmask;  // ghost occupancy
  const int32_t* bstart;  // first band index of the brick
  const int32_t* gstart;  // first ghost index of the brick (relative to nB)
  const BrickRec* brec;   // nbricks brick records
  int nbx, nby, nbz;
  int n;                  // nodes per axis
  int32_t nB;
  int32_t nbricks;
};

// Index in B+ of grid node (x, y, z) (B: [0, nB), G: [nB, nB+nG)), or -1.
__device__ inline int32_t node_index(const BrickView& v, int x, int y, int z) {
  if ((unsigned)x >= (unsigned)v.n || (unsigned)y >= (unsigned)v.n || (unsigned)z >= (unsigned)v.n)
    return -1;
  const int bx = x >> 2, by = y >> 2, bz = z >> 2;
  const int32_t b = __ldg(v.map + ((size_t)bz * v.nby + by) * v.nbx + bx);
  if (b < 0) return -1;
  const int l = (x & 3) | ((y & 3) << 2) | ((z & 3) << 4);
  const uint64_t bit = 1ull << l;
  const uint64_t bm = __ldg(v.bmask + b);
  if (bm & bit) return __ldg(v.bstart + b) + __popcll(bm & (bit - 1));
  const uint64_t gm = __ldg(v.gmask + b);
  if (gm & bit) return v.nB + __ldg(v.gstart + b) + __popcll(gm & (bit - 1));
  return -1;
}

// Index in B of a node known to be a band node (stencil nodes are).  Returns
// -1 if it is not (the caller raises a checked error).
__device__ inline int32_t band_index(const BrickView& v, int x, int y, int z) {
  if ((unsigned)x >= (unsigned)v.n || (unsigned)y >= (unsigned)v.n || (unsigned)z >= (unsigned)v.n)
    return -1;
  const int32_t b = __ldg(v.map + ((size_t)(z >> 2) * v.nby + (y >> 2)) * v.nbx + (x >> 2));
  if (b < 0) return -1;
  const int l = (x & 3) | ((y & 3) << 2) | ((z & 3) << 4);
  const uint64_t bit = 1ull << l;
  const uint64_t bm = __ldg(v.bmask + b);
  if (!(bm & bit)) return -1;
  return __ldg(v.bstart + b) + __popcll(bm & (bit - 1));
}

// ----------------------------------------------------------------- level
struct Level {
  int dim = 3;
  double lo = -2.0, dx = 0.0, lambda2 = 17.0;
  int n = 0;
  int nbx = 0, nby = 0, nbz = 0;
  int32_t nbricks = 0;
  int32_t nB = 0, nG = 0;
  // brick tables
  DBuf<int32_t> map;
  DBuf<uint64_t> bmask, gmask;
  DBuf<int32_t> bstart, gstart;
  DBuf<uint32_t> bcoord;  // packed brick coordinates bx | by << 10 | bz << 20 (<= 1023 each)
  DBuf<BrickRec> brec;    // per brick: masks and starts of it and its face neighbours
  // per point of B+
  DBuf<uint64_t> key;
  DBuf<double> cp;    // d x (nB+nG), SoA
  DBuf<double> fr64;  // d x (nB+nG), SoA
  DBuf<float> fr32;   // d x (nB+nG), SoA
  // extension tiles: the points of B+ grouped by the brick that holds their
  // cubic stencil base, points of B first in each tile ("E order"); see ext.cu
  int32_t ntiles = 0;
  DBuf<uint32_t> tile_brick;  // packed brick coordinates of each tile
  DBuf<uint32_t> tile_box;    // per axis: lowest and highest base position in the brick
  DBuf<uint64_t> tile_mask;   // 8 per tile: band masks of the bricks the tile's box overlaps
  DBuf<int32_t> tile_bstart;  // 8 per tile: their band starts
  DBuf<int32_t> tile_start;   // ntiles + 1 offsets into the E-order arrays
  DBuf<int32_t> tile_mid;     // per tile: end of its points of B
  DBuf<uint32_t> erec;        // band index << 6 | stencil base inside the brick
  DBuf<float> efr32;          // d x (nB+nG) fractions in E order
  DBuf<double> ew64;          // 4d x (nB+nG) FP64 cubic weights in E order
  DBuf<float2> ewp;           // the same as FP32 pairs (built on demand: build_pair_weights)
  // chunks: runs of at most kChunkMax consecutive E-order points of one tile
  // that share one stencil base (and are all in B or all in G); one thread
  // loads the base's 4^d values once and evaluates every point of the chunk
  int ext_variant = 0;        // FP32 extension variant chosen by timing (ExtVariant)
  float ext_ms[3] = {0.f, 0.f, 0.f};
  int32_t nchunks = 0;
  DBuf<uint32_t> echunk;      // first E-order point | (count - 1) << 26
  DBuf<int32_t> tile_cstart;  // ntiles + 1 offsets into echunk
  DBuf<int32_t> tile_cmid;    // per tile: end of its chunks of points of B
  DBuf<int32_t> nbr;          // 2d x nB: B+ index of the Laplacian neighbours of B

  BrickView view() const {
    BrickView v;
    v.map = map.get(); v.bmask = bmask.get(); v.gmask = gmask.get();
    v.bstart = bstart.get(); v.gstart = gstart.get(); v.brec = brec.get();
    v.nbx = nbx; v.nby = nby; v.nbz = nbz; v.n = n; v.nB = nB; v.nbricks = nbricks;
    return v;
  }
  int64_t nplus() const { return (int64_t)nB + nG; }
};

// Build the band of one level (band.cu).  Throws cpm::Error.
void build_level(const cpm_surface& s, double lo, double dx, int n, double lambda2,
                 cudaStream_t st, Level& out);
// |B|, nnz(L_B), nnz(E_3), nnz(E_1 L_B - gamma (I - E_3)) of a level (band.cu).
void band_counts(const Level& L, cudaStream_t st, int64_t counts[4]);
// Group the points of a level into extension tiles (ext.cu).
void build_ext_tiles(Level& L, cudaStream_t st);
// L.ewp from L.ew64 (each weight split into a float pair, see pair.cuh).
void build_pair_weights(Level& L, cudaStream_t st);

// Host counter of solve-path kernel launches (cpm_kernel_launches).  While a
// stream capture is being recorded the launch helpers do not count; a graph
// adds its kernel-node count on every replay instead.
void count_launch(int64_t n = 1);
void set_capturing(bool on);

// Exclusive scan of int64 values in place; returns the total (band.cu).
int64_t scan_exclusive_i64(int64_t* d, int64_t n, cudaStream_t st);

// Surface descriptor as passed to kernels.
struct SurfaceDev {
  int kind;
  int dim;
  double p[8];
};
SurfaceDev make_surface(const cpm_surface& s);
double surface_reach(const cpm_surface& s);
int surface_dim(const cpm_surface& s);

}  // namespace cpm

// The public handle types.
struct cpm_band_s {
  cpm_surface surface;
  cpm::Level lev;
};
