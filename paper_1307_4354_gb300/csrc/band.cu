// Band construction on the device (Sec. 3.1 band; Table 4.1 sizes).
//
// Pipeline (all kernels below, one level at a time):
//   1. brick candidates: every 4^d brick of the grid, in Morton order of its
//      brick coordinates, is tested in FP32 against a conservative distance
//      bound (a superset of the bricks that can hold band or ghost nodes);
//      warp ballots give one flag bit per Morton code.
//   2. compaction of the flagged codes (scan of popcounts), brick map.
//   3. band mask: every node of a candidate brick is tested exactly,
//      |x - cp(x)|^2 <= lambda2 * (dx*dx), in FP64 with the operation order
//      fixed and no fused multiply-add (__dmul_rn / __dadd_rn / __dsqrt_rn),
//      so that membership is reproducible bit for bit.
//   4. ghost mask: nodes outside B with a Laplacian neighbour in B.
//   5. compaction to occupied bricks, per-brick starts (exclusive scans).
//   6. emission of keys, closest points and stencil fractions for B then G.
//   7. check that every cubic stencil node of every point of B+ is in B.
#include <math_constants.h>

#include <cmath>
#include <cstdio>

#include "cpm_internal.cuh"

namespace cpm {

// ----------------------------------------------------------------- surfaces
SurfaceDev make_surface(const cpm_surface& s) {
  SurfaceDev d;
  d.kind = s.kind;
  d.dim = surface_dim(s);
  for (int i = 0; i < 8; ++i) d.p[i] = s.param[i];
  return d;
}

int surface_dim(const cpm_surface& s) { return s.kind == CPM_CIRCLE ? 2 : 3; }

double surface_reach(const cpm_surface& s) {
  switch (s.kind) {
    case CPM_CIRCLE:
    case CPM_SPHERE: return s.param[0];
    case CPM_TORUS: return std::fmin(s.param[1], s.param[0] - s.param[1]);
    case CPM_ELLIPSOID: {
      double a = std::fmin(s.param[0], std::fmin(s.param[1], s.param[2]));
      double b = std::fmax(s.param[0], std::fmax(s.param[1], s.param[2]));
      return a * a / b;
    }
    // largest principal curvature of the Dziuk surface: 10.44 near x3 = +-0.92
    // (shape operator of the level set evaluated on a fine grid of the surface)
    case CPM_DZIUK: return 0.0957;
  }
  return 0.0;
}

// Closest point and squared distance in FP64, every operation rounded
// separately in the order stated in the oracle's geometry module:
//   sphere/circle: r = sqrt((x*x + y*y) + z*z); d = r - R; t = R / r; cp = x*t
//   torus:         rho = sqrt(x*x + y*y); a = rho - R; q = sqrt(a*a + z*z);
//                  d = q - r; s = r / q; m = R + a*s; k = m / rho;
//                  cp = (x*k, y*k, z*s)
//   ellipsoid:     bisection on sum a_i^2 x_i^2 / (a_i^2 + t)^2 = 1 to the last
//                  bit, cp_i = (a_i^2 x_i) / (a_i^2 + t); if the function is
//                  never positive the node is on the medial disk: dist2 = inf.
__device__ inline double dsub(double a, double b) { return __dadd_rn(a, -b); }
__device__ inline double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ inline double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ inline double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// Dziuk surface phi(y) = (y1 - y3^2)^2 + y2^2 + y3^2 - 1 (Sec. 4.5.5): closest
// point by Newton's method on  y - x + lam g(y) = 0, phi(y) = 0  with
// g = grad(phi)/2 = (a, y2, y3 (1 - 2a)), a = y1 - y3^2, from y = x, lam = 0;
// 30 steps, each solving [K, g; 2 g^T, 0][dy; dl] = -[F1; F2] with
// K = I + lam dg/dy (K13 = K31 = -2 lam y3 its only off-diagonal entry):
// dl = (F2 - 2 g.K^-1 F1) / (2 g.K^-1 g), dy = -K^-1 (F1 + g dl).
__device__ void dziuk_cp(double x1, double x2, double x3, double cp[3], double& dist2) {
  double y1 = x1, y2 = x2, y3 = x3, lam = 0.0;
  for (int it = 0; it < 30; ++it) {
    const double y3s = dmul(y3, y3);
    const double a = dsub(y1, y3s);
    const double g1 = a, g2 = y2, g3 = dmul(y3, dsub(1.0, dmul(2.0, a)));
    const double F11 = dadd(dsub(y1, x1), dmul(lam, g1));
    const double F12 = dadd(dsub(y2, x2), dmul(lam, g2));
    const double F13 = dadd(dsub(y3, x3), dmul(lam, g3));
    const double F2 = dsub(dadd(dadd(dmul(a, a), dmul(y2, y2)), y3s), 1.0);
    const double k11 = dadd(1.0, lam), k22 = dadd(1.0, lam);
    const double k13 = dmul(-2.0, dmul(lam, y3));
    const double k33 = dadd(1.0, dmul(lam, dadd(dsub(1.0, dmul(2.0, y1)), dmul(6.0, y3s))));
    const double det = dsub(dmul(k11, k33), dmul(k13, k13));
    const double p1 = ddiv(dsub(dmul(k33, F11), dmul(k13, F13)), det);
    const double p2 = ddiv(F12, k22);
    const double p3 = ddiv(dsub(dmul(k11, F13), dmul(k13, F11)), det);
    const double q1 = ddiv(dsub(dmul(k33, g1), dmul(k13, g3)), det);
    const double q2 = ddiv(g2, k22);
    const double q3 = ddiv(dsub(dmul(k11, g3), dmul(k13, g1)), det);
    const double gp = dadd(dadd(dmul(g1, p1), dmul(g2, p2)), dmul(g3, p3));
    const double gq = dadd(dadd(dmul(g1, q1), dmul(g2, q2)), dmul(g3, q3));
    const double dl = ddiv(dsub(F2, dmul(2.0, gp)), dmul(2.0, gq));
    y1 = dsub(y1, dadd(p1, dmul(q1, dl)));
    y2 = dsub(y2, dadd(p2, dmul(q2, dl)));
    y3 = dsub(y3, dadd(p3, dmul(q3, dl)));
    lam = dadd(lam, dl);
  }
  const double d1 = dsub(x1, y1), d2 = dsub(x2, y2), d3 = dsub(x3, y3);
  dist2 = dadd(dadd(dmul(d1, d1), dmul(d2, d2)), dmul(d3, d3));
  if (!isfinite(dist2)) {
    cp[0] = cp[1] = cp[2] = CUDART_NAN;
    dist2 = CUDART_INF;
    return;
  }
  cp[0] = y1;
  cp[1] = y2;
  cp[2] = y3;
}

__device__ void closest_point_f64(const SurfaceDev& s, double x, double y, double z, double cp[3],
                                  double& dist2) {
  if (s.kind == CPM_CIRCLE || s.kind == CPM_SPHERE) {
    const double R = s.p[0];
    double r2 = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
    if (s.dim == 3) r2 = __dadd_rn(r2, __dmul_rn(z, z));
    const double r = __dsqrt_rn(r2);
    const double d = dsub(r, R);
    dist2 = __dmul_rn(d, d);
    const double t = __ddiv_rn(R, r);
    cp[0] = __dmul_rn(x, t);
    cp[1] = __dmul_rn(y, t);
    cp[2] = s.dim == 3 ? __dmul_rn(z, t) : 0.0;
  } else if (s.kind == CPM_TORUS) {
    const double R = s.p[0], rr = s.p[1];
    const double rho = __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
    const double a = dsub(rho, R);
    const double q = __dsqrt_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(z, z)));
    const double d = dsub(q, rr);
    dist2 = __dmul_rn(d, d);
    const double sc = __ddiv_rn(rr, q);
    const double m = __dadd_rn(R, __dmul_rn(a, sc));
    const double k = __ddiv_rn(m, rho);
    cp[0] = __dmul_rn(x, k);
    cp[1] = __dmul_rn(y, k);
    cp[2] = __dmul_rn(z, sc);
  } else if (s.kind == CPM_DZIUK) {
    dziuk_cp(x, y, z, cp, dist2);
  } else {  // ellipsoid
    const double X[3] = {x, y, z};
    double a2[3], ax[3];
    for (int i = 0; i < 3; ++i) {
      a2[i] = __dmul_rn(s.p[i], s.p[i]);
      ax[i] = __dmul_rn(fabs(X[i]), s.p[i]);
    }
    const double amin2 = fmin(a2[0], fmin(a2[1], a2[2]));
    double lo = -amin2;
    double hi = __dadd_rn(
        __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ax[0], ax[0]), __dmul_rn(ax[1], ax[1])),
                             __dmul_rn(ax[2], ax[2]))),
        1e-300);
    bool moved = false;
    for (int it = 0; it < 1100; ++it) {
      const double mid = __dmul_rn(0.5, __dadd_rn(lo, hi));
      if (mid == lo || mid == hi) break;
      const double g0 = __ddiv_rn(ax[0], __dadd_rn(a2[0], mid));
      const double g1 = __ddiv_rn(ax[1], __dadd_rn(a2[1], mid));
      const double g2 = __ddiv_rn(ax[2], __dadd_rn(a2[2], mid));
      const double F =
          dsub(__dadd_rn(__dadd_rn(__dmul_rn(g0, g0), __dmul_rn(g1, g1)), __dmul_rn(g2, g2)), 1.0);
      if (F > 0) { lo = mid; moved = true; } else { hi = mid; }
    }
    if (!moved) {
      // root at or below -min a_i^2: x is on the medial disk, at least the
      // reach away from S; never a band or ghost node
      cp[0] = cp[1] = cp[2] = CUDART_NAN;
      dist2 = CUDART_INF;
      return;
    }
    const double t = __dmul_rn(0.5, __dadd_rn(lo, hi));
    double dd[3];
    for (int i = 0; i < 3; ++i) {
      cp[i] = __ddiv_rn(__dmul_rn(a2[i], X[i]), __dadd_rn(a2[i], t));
      dd[i] = dsub(X[i], cp[i]);
    }
    dist2 = __dadd_rn(__dadd_rn(__dmul_rn(dd[0], dd[0]), __dmul_rn(dd[1], dd[1])),
                      __dmul_rn(dd[2], dd[2]));
  }
}

// Conservative lower bound of the distance to S in FP32 (candidate filter).
__device__ inline float dist_lower_f32(const SurfaceDev& s, float x, float y, float z) {
  if (s.kind == CPM_CIRCLE) return fabsf(sqrtf(x * x + y * y) - (float)s.p[0]);
  if (s.kind == CPM_SPHERE) return fabsf(sqrtf(x * x + y * y + z * z) - (float)s.p[0]);
  if (s.kind == CPM_TORUS) {
    const float a = sqrtf(x * x + y * y) - (float)s.p[0];
    return fabsf(sqrtf(a * a + z * z) - (float)s.p[1]);
  }
  if (s.kind == CPM_DZIUK) {
    // first-order distance |phi| / |grad phi| with a factor 4 of slack for the
    // curvature (at most 10.44) over the band half-widths the reach allows
    const float a = x - z * z;
    const float phi = a * a + y * y + z * z - 1.0f;
    const float b = z * (1.0f - 2.0f * a);
    const float g = 2.0f * sqrtf(a * a + y * y + b * b);
    return g > 0.f ? 0.25f * fabsf(phi) / g : 1e30f;
  }
  // ellipsoid: |x - y| >= a_min |rho - 1| for every y on S, rho = |D^-1 x|
  const float a0 = (float)s.p[0], a1 = (float)s.p[1], a2 = (float)s.p[2];
  const float rho = sqrtf((x / a0) * (x / a0) + (y / a1) * (y / a1) + (z / a2) * (z / a2));
  return fminf(a0, fminf(a1, a2)) * fabsf(rho - 1.0f);
}

// ----------------------------------------------------------------- Morton
__host__ __device__ inline uint32_t compact1by2(uint64_t v) {
  v &= 0x1249249249249249ull;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
  v = (v ^ (v >> 32)) & 0x1fffffull;
  return (uint32_t)v;
}
__host__ __device__ inline uint32_t compact1by1(uint64_t v) {
  v &= 0x5555555555555555ull;
  v = (v ^ (v >> 1)) & 0x3333333333333333ull;
  v = (v ^ (v >> 2)) & 0x0f0f0f0f0f0f0f0full;
  v = (v ^ (v >> 4)) & 0x00ff00ff00ff00ffull;
  v = (v ^ (v >> 8)) & 0x0000ffff0000ffffull;
  v = (v ^ (v >> 16)) & 0x00000000ffffffffull;
  return (uint32_t)v;
}
__host__ __device__ inline void morton_decode(uint64_t code, int dim, int& bx, int& by, int& bz) {
  if (dim == 3) {
    bx = compact1by2(code);
    by = compact1by2(code >> 1);
    bz = compact1by2(code >> 2);
  } else {
    bx = compact1by1(code);
    by = compact1by1(code >> 1);
    bz = 0;
  }
}

// ----------------------------------------------------------------- scan
// Exclusive scan of int64 in place.  Tiles of 4 * 256 values per block; the
// per-tile totals are scanned recursively and added back.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ inline int64_t block_exclusive_scan(int64_t v, int64_t& total) {
  __shared__ int64_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  const int64_t warp_off = wid > 0 ? warp_sums[wid - 1] : 0;
  total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void k_scan_tiles(int64_t* d, int64_t n, int64_t* tile_sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? d[base + i] : 0;
    s += v[i];
  }
  int64_t total;
  int64_t off = block_exclusive_scan(s, total);
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) d[base + i] = off;
    off += v[i];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_add(int64_t* d, int64_t n, const int64_t* tile_offsets) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  const int64_t add = tile_offsets[blockIdx.x];
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) d[base + i] += add;
}

int64_t scan_exclusive_i64(int64_t* d, int64_t n, cudaStream_t st) {
  if (n <= 0) return 0;
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  DBuf<int64_t> sums(tiles + 1);
  k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(d, n, sums.get());
  CPM_CUDA_TRY(cudaGetLastError());
  int64_t total;
  if (tiles > 1) {
    total = scan_exclusive_i64(sums.get(), tiles, st);
    k_scan_add<<<(unsigned)tiles, kScanThreads, 0, st>>>(d, n, sums.get());
    CPM_CUDA_TRY(cudaGetLastError());
  } else {
    CPM_CUDA_TRY(cudaMemcpyAsync(&total, sums.get(), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CPM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return total;
}

// ----------------------------------------------------------------- kernels
struct GridDev {
  double lo, dx, thr;  // thr = lambda2 * (dx*dx)
  int n, dim;
  int nbx, nby, nbz;
};

// 1. Candidate flags: bit (code & 31) of word (code >> 5).
__global__ void k_brick_flags(SurfaceDev s, GridDev g, uint64_t ncodes, float reach_f,
                              uint32_t* words) {
  const uint64_t code = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool flag = false;
  if (code < ncodes) {
    int bx, by, bz;
    morton_decode(code, g.dim, bx, by, bz);
    if (bx < g.nbx && by < g.nby && bz < g.nbz) {
      const float h = (float)g.dx;
      const float cx = (float)g.lo + (4 * bx + 1.5f) * h;
      const float cy = (float)g.lo + (4 * by + 1.5f) * h;
      const float cz = g.dim == 3 ? (float)g.lo + (4 * bz + 1.5f) * h : 0.0f;
      flag = dist_lower_f32(s, cx, cy, cz) <= reach_f;
    }
  }
  const uint32_t bal = __ballot_sync(0xffffffffu, flag);
  if ((threadIdx.x & 31) == 0 && code < ncodes) words[code >> 5] = bal;
}

__global__ void k_word_counts(const uint32_t* words, int64_t nwords, int64_t* counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nwords) counts[i] = __popc(words[i]);
}

__global__ void k_emit_codes(const uint32_t* words, const int64_t* offsets, uint64_t ncodes, int dim,
                             uint32_t* bcoord) {
  const uint64_t code = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (code >= ncodes) return;
  const uint32_t w = words[code >> 5];
  const uint32_t bit = 1u << (code & 31);
  if (!(w & bit)) return;
  const int64_t pos = offsets[code >> 5] + __popc(w & (bit - 1));
  int bx, by, bz;
  morton_decode(code, dim, bx, by, bz);
  bcoord[pos] = (uint32_t)bx | ((uint32_t)by << 10) | ((uint32_t)bz << 20);
}

__global__ void k_fill_map(const uint32_t* bcoord, int32_t nbricks, GridDev g, int32_t* map) {
  const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbricks) return;
  const uint32_t c = bcoord[b];
  const int bx = c & 1023, by = (c >> 10) & 1023, bz = (c >> 20) & 1023;
  map[((size_t)bz * g.nby + by) * g.nbx + bx] = b;
}

__device__ inline bool node_valid(const GridDev& g, int x, int y, int z) {
  return x < g.n && y < g.n && (g.dim == 2 ? z == 0 : z < g.n);
}

// 3. Exact band membership, 64 threads per brick (2 ballots).
__global__ void k_band_mask(SurfaceDev s, GridDev g, const uint32_t* bcoord, int32_t nbricks,
                            uint64_t* bmask) {
  const int32_t b = blockIdx.x * (blockDim.x / 64) + threadIdx.x / 64;
  const int l = threadIdx.x & 63;
  bool in = false;
  if (b < nbricks) {
    const uint32_t c = bcoord[b];
    const int x = 4 * (int)(c & 1023) + (l & 3);
    const int y = 4 * (int)((c >> 10) & 1023) + ((l >> 2) & 3);
    const int z = 4 * (int)((c >> 20) & 1023) + (l >> 4);
    if (node_valid(g, x, y, z)) {
      const double X = __dadd_rn(g.lo, __dmul_rn((double)x, g.dx));
      const double Y = __dadd_rn(g.lo, __dmul_rn((double)y, g.dx));
      const double Z = g.dim == 3 ? __dadd_rn(g.lo, __dmul_rn((double)z, g.dx)) : 0.0;
      double cp[3], d2;
      closest_point_f64(s, X, Y, Z, cp, d2);
      in = d2 <= g.thr;
    }
  }
  const uint32_t bal = __ballot_sync(0xffffffffu, in);
  if (b < nbricks && (l & 31) == 0) {
    uint32_t* half = reinterpret_cast<uint32_t*>(bmask + b);
    half[l >> 5] = bal;
  }
}

__device__ inline bool in_band(const int32_t* map, const uint64_t* bmask, const GridDev& g, int x,
                               int y, int z) {
  if (x < 0 || y < 0 || z < 0 || !node_valid(g, x, y, z)) return false;
  const int32_t b = map[((size_t)(z >> 2) * g.nby + (y >> 2)) * g.nbx + (x >> 2)];
  if (b < 0) return false;
  return (bmask[b] >> ((x & 3) | ((y & 3) << 2) | ((z & 3) << 4))) & 1ull;
}

// 4. Ghost ring: nodes outside B with a 2d-neighbour in B.
__global__ void k_ghost_mask(GridDev g, const uint32_t* bcoord, const int32_t* map,
                             const uint64_t* bmask, int32_t nbricks, uint64_t* gmask) {
  const int32_t b = blockIdx.x * (blockDim.x / 64) + threadIdx.x / 64;
  const int l = threadIdx.x & 63;
  bool ghost = false;
  if (b < nbricks) {
    const uint32_t c = bcoord[b];
    const int x = 4 * (int)(c & 1023) + (l & 3);
    const int y = 4 * (int)((c >> 10) & 1023) + ((l >> 2) & 3);
    const int z = 4 * (int)((c >> 20) & 1023) + (l >> 4);
    if (node_valid(g, x, y, z) && !((bmask[b] >> l) & 1ull)) {
      ghost = in_band(map, bmask, g, x - 1, y, z) || in_band(map, bmask, g, x + 1, y, z) ||
              in_band(map, bmask, g, x, y - 1, z) || in_band(map, bmask, g, x, y + 1, z);
      if (g.dim == 3)
        ghost = ghost || in_band(map, bmask, g, x, y, z - 1) || in_band(map, bmask, g, x, y, z + 1);
    }
  }
  const uint32_t bal = __ballot_sync(0xffffffffu, ghost);
  if (b < nbricks && (l & 31) == 0) {
    uint32_t* half = reinterpret_cast<uint32_t*>(gmask + b);
    half[l >> 5] = bal;
  }
}

// 5. Occupied bricks.
__global__ void k_occupied(const uint64_t* bmask, const uint64_t* gmask, int32_t nbricks,
                           int64_t* flag) {
  const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nbricks) flag[b] = (bmask[b] | gmask[b]) != 0ull;
}

__global__ void k_compact_bricks(const uint64_t* bmask, const uint64_t* gmask, const uint32_t* bcoord,
                                 const int64_t* pos, int32_t nbricks, uint64_t* bmask2,
                                 uint64_t* gmask2, uint32_t* bcoord2, int64_t* bcount,
                                 int64_t* gcount) {
  const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbricks) return;
  const uint64_t bm = bmask[b], gm = gmask[b];
  if ((bm | gm) == 0ull) return;
  const int64_t p = pos[b];
  bmask2[p] = bm;
  gmask2[p] = gm;
  bcoord2[p] = bcoord[b];
  bcount[p] = __popcll(bm);
  gcount[p] = __popcll(gm);
}

__global__ void k_copy_i64_to_i32(const int64_t* a, int32_t* b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (int32_t)a[i];
}

// 6. Emit the points of B+.
__global__ void k_emit_points(SurfaceDev s, GridDev g, const uint32_t* bcoord, const uint64_t* bmask,
                              const uint64_t* gmask, const int32_t* bstart, const int32_t* gstart,
                              int32_t nbricks, int32_t nB, int64_t nplus, uint64_t* key, double* cp,
                              double* fr64, float* fr32, int32_t* err, double* errinfo) {
  const int32_t b = blockIdx.x * (blockDim.x / 64) + threadIdx.x / 64;
  const int l = threadIdx.x & 63;
  if (b >= nbricks) return;
  const uint64_t bit = 1ull << l;
  const uint64_t bm = bmask[b], gm = gmask[b];
  int64_t idx;
  if (bm & bit) idx = bstart[b] + __popcll(bm & (bit - 1));
  else if (gm & bit) idx = (int64_t)nB + gstart[b] + __popcll(gm & (bit - 1));
  else return;
  const uint32_t c = bcoord[b];
  const int x = 4 * (int)(c & 1023) + (l & 3);
  const int y = 4 * (int)((c >> 10) & 1023) + ((l >> 2) & 3);
  const int z = 4 * (int)((c >> 20) & 1023) + (l >> 4);
  const double X = __dadd_rn(g.lo, __dmul_rn((double)x, g.dx));
  const double Y = __dadd_rn(g.lo, __dmul_rn((double)y, g.dx));
  const double Z = g.dim == 3 ? __dadd_rn(g.lo, __dmul_rn((double)z, g.dx)) : 0.0;
  double p[3], d2;
  closest_point_f64(s, X, Y, Z, p, d2);
  const int own[3] = {x, y, z};
  uint64_t k = (uint64_t)x | ((uint64_t)y << 16) | ((uint64_t)z << 32);
  bool ok = true;
  for (int a = 0; a < g.dim; ++a) {
    if (!isfinite(p[a])) { ok = false; break; }
    const double t = __ddiv_rn(dsub(p[a], g.lo), g.dx);
    const double fl = floor(t);
    const double sfrac = dsub(t, fl);
    const int off = (int)fl - 1 - own[a];
    if (off < -8 || off > 7) { ok = false; break; }
    k |= (uint64_t)(off + 8) << (48 + 4 * a);
    cp[a * nplus + idx] = p[a];
    fr64[a * nplus + idx] = sfrac;
    fr32[a * nplus + idx] = (float)sfrac;
  }
  if (g.dim == 2) k |= (uint64_t)8 << 56;  // z offset 0
  if (!ok && atomicOr(err, 1) == 0) {
    // first failing node: coordinates, closest point and squared distance
    errinfo[0] = x; errinfo[1] = y; errinfo[2] = z;
    errinfo[3] = p[0]; errinfo[4] = p[1]; errinfo[5] = p[2]; errinfo[6] = d2;
  }
  // a band node on the edge of the grid would lose Laplacian neighbours
  if ((bm & bit) && (x == 0 || y == 0 || x == g.n - 1 || y == g.n - 1 ||
                     (g.dim == 3 && (z == 0 || z == g.n - 1))))
    atomicOr(err, 8);
  key[idx] = k;
}

// 7. Every cubic stencil node of every point of B+ must be in B.
__global__ void k_check_stencils(BrickView v, const uint64_t* key, int64_t nplus, int dim,
                                 int32_t* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nplus) return;
  const uint64_t k = key[i];
  const int bx = key_x(k) + key_ox(k), by = key_y(k) + key_oy(k), bz = key_z(k) + key_oz(k);
  const int zn = dim == 3 ? 4 : 1;
  for (int c = 0; c < zn; ++c)
    for (int b = 0; b < 4; ++b)
      for (int a = 0; a < 4; ++a)
        if (band_index(v, bx + a, by + b, dim == 3 ? bz + c : 0) < 0) {
          atomicOr(err, 2);
          return;
        }
}

// 8. Laplacian neighbours of B (order -x, +x, -y, +y, -z, +z), as B+ indices.
__global__ void k_neighbours(BrickView v, const uint64_t* key, int32_t nB, int dim, int32_t* nbr,
                             int32_t* err) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nB) return;
  const uint64_t k = key[i];
  const int x = key_x(k), y = key_y(k), z = key_z(k);
  const int d[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  for (int q = 0; q < 2 * dim; ++q) {
    const int32_t j = node_index(v, x + d[q][0], y + d[q][1], z + d[q][2]);
    if (j < 0) atomicOr(err, 16);
    nbr[(int64_t)q * nB + i] = j < 0 ? i : j;
  }
}

// 9. Brick records: masks and starts of every occupied brick and of its face
// neighbours (order -x, +x, -y, +y, -z, +z).
__global__ void k_brick_recs(BrickView v, const uint32_t* bcoord, int dim, BrickRec* rec) {
  const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= v.nbricks) return;
  const uint32_t c = bcoord[b];
  const int bx = (int)(c & 1023), by = (int)((c >> 10) & 1023), bz = (int)((c >> 20) & 1023);
  const int d[7][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  BrickRec r;
  for (int q = 0; q < 7; ++q) {
    const int x = bx + d[q][0], y = by + d[q][1], z = bz + d[q][2];
    int32_t nb = -1;
    if (q <= 2 * dim && x >= 0 && y >= 0 && z >= 0 && x < v.nbx && y < v.nby && z < v.nbz)
      nb = v.map[((size_t)z * v.nby + y) * v.nbx + x];
    r.bm[q] = nb >= 0 ? v.bmask[nb] : 0ull;
    r.gm[q] = nb >= 0 ? v.gmask[nb] : 0ull;
    r.bs[q] = nb >= 0 ? v.bstart[nb] : 0;
    r.gs[q] = nb >= 0 ? v.gstart[nb] : 0;
  }
  rec[b] = r;
}

// 10. Table 4.1 counts: per band point the number of its 2d Laplacian
// neighbours inside B (the band-restricted L) and whether the node lies outside
// its own cubic stencil (an extra diagonal entry of M = E_1 L - gamma (I - E_3)).
__global__ void k_band_counts(BrickView v, const uint64_t* key, int32_t nB, int dim,
                              unsigned long long* acc) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long nl = 0, outside = 0;
  if (i < nB) {
    const uint64_t k = key[i];
    const int x = key_x(k), y = key_y(k), z = key_z(k);
    const int d[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    for (int q = 0; q < 2 * dim; ++q)
      nl += band_index(v, x + d[q][0], y + d[q][1], z + d[q][2]) >= 0;
    const int off[3] = {-key_ox(k), -key_oy(k), dim == 3 ? -key_oz(k) : 0};
    for (int a = 0; a < dim; ++a) outside |= (off[a] < 0 || off[a] > 3);
  }
  for (int o = 16; o > 0; o >>= 1) {
    nl += __shfl_xor_sync(0xffffffffu, nl, o);
    outside += __shfl_xor_sync(0xffffffffu, outside, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc, nl);
    atomicAdd(acc + 1, outside);
  }
}

void band_counts(const Level& L, cudaStream_t st, int64_t counts[4]) {
  DBuf<unsigned long long> acc(2);
  CPM_CUDA_TRY(cudaMemsetAsync(acc.get(), 0, 2 * sizeof(unsigned long long), st));
  if (L.nB > 0)
    k_band_counts<<<(unsigned)((L.nB + 255) / 256), 256, 0, st>>>(L.view(), L.key.get(), L.nB, L.dim,
                                                                   acc.get());
  CPM_CUDA_TRY(cudaGetLastError());
  unsigned long long h[2];
  CPM_CUDA_TRY(cudaMemcpyAsync(h, acc.get(), sizeof(h), cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  const int64_t nE = (int64_t)L.nB * (L.dim == 3 ? 64 : 16);
  counts[0] = L.nB;
  counts[1] = L.nB + (int64_t)h[0];
  counts[2] = nE;
  counts[3] = nE + (int64_t)h[1];
}

// ----------------------------------------------------------------- driver
static unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

void build_level(const cpm_surface& surf, double lo, double dx, int n, double lambda2,
                 cudaStream_t st, Level& L) {
  const int dim = surface_dim(surf);
  CPM_CHECK(dx > 0 && std::isfinite(dx), CPM_ERR_ARG, "dx must be positive");
  CPM_CHECK(n >= 8 && n <= 4090, CPM_ERR_ARG, "grid size n out of range [8, 4090]");
  L.dim = dim;
  L.lo = lo;
  L.dx = dx;
  L.n = n;
  L.lambda2 = lambda2;
  L.nbx = L.nby = (n + 3) / 4;
  L.nbz = dim == 3 ? (n + 3) / 4 : 1;
  GridDev g;
  g.lo = lo;
  g.dx = dx;
  g.thr = lambda2 * (dx * dx);
  g.n = n;
  g.dim = dim;
  g.nbx = L.nbx;
  g.nby = L.nby;
  g.nbz = L.nbz;
  const SurfaceDev s = make_surface(surf);

  // 1-2. candidates in Morton order
  int bits = 0;
  while ((1 << bits) < L.nbx) ++bits;
  const uint64_t ncodes = 1ull << (dim * bits);
  const int64_t nwords = (int64_t)((ncodes + 31) / 32);
  const double halfdiag = std::sqrt((double)dim) * 1.5 * dx;
  const float reach_f = (float)((std::sqrt(lambda2) + 1.0) * dx + halfdiag + 1e-4 * dx + 1e-6);
  DBuf<uint32_t> words(nwords);
  k_brick_flags<<<blocks_for((int64_t)ncodes, 256), 256, 0, st>>>(s, g, ncodes, reach_f, words.get());
  CPM_CUDA_TRY(cudaGetLastError());
  DBuf<int64_t> woff(nwords);
  k_word_counts<<<blocks_for(nwords, 256), 256, 0, st>>>(words.get(), nwords, woff.get());
  const int64_t ncand = scan_exclusive_i64(woff.get(), nwords, st);
  CPM_CHECK(ncand > 0, CPM_ERR_ARG, "the surface does not meet the grid");
  CPM_CHECK(ncand < (1ll << 31), CPM_ERR_ARG, "too many bricks");
  DBuf<uint32_t> cand(ncand);
  k_emit_codes<<<blocks_for((int64_t)ncodes, 256), 256, 0, st>>>(words.get(), woff.get(), ncodes, dim,
                                                                  cand.get());
  words.release();
  woff.release();
  const size_t mapsize = (size_t)L.nbx * L.nby * L.nbz;
  L.map.alloc(mapsize);
  CPM_CUDA_TRY(cudaMemsetAsync(L.map.get(), 0xff, mapsize * sizeof(int32_t), st));
  const int32_t nc = (int32_t)ncand;
  k_fill_map<<<blocks_for(nc, 256), 256, 0, st>>>(cand.get(), nc, g, L.map.get());

  // 3-4. masks
  DBuf<uint64_t> bm(nc), gm(nc);
  k_band_mask<<<blocks_for((int64_t)nc * 64, 256), 256, 0, st>>>(s, g, cand.get(), nc, bm.get());
  CPM_CUDA_TRY(cudaGetLastError());
  k_ghost_mask<<<blocks_for((int64_t)nc * 64, 256), 256, 0, st>>>(g, cand.get(), L.map.get(), bm.get(),
                                                                   nc, gm.get());
  CPM_CUDA_TRY(cudaGetLastError());

  // 5. compaction to occupied bricks
  DBuf<int64_t> pos(nc);
  k_occupied<<<blocks_for(nc, 256), 256, 0, st>>>(bm.get(), gm.get(), nc, pos.get());
  const int64_t nocc = scan_exclusive_i64(pos.get(), nc, st);
  CPM_CHECK(nocc > 0, CPM_ERR_ARG, "empty band");
  L.nbricks = (int32_t)nocc;
  L.bmask.alloc(nocc);
  L.gmask.alloc(nocc);
  L.bcoord.alloc(nocc);
  DBuf<int64_t> bcount(nocc), gcount(nocc);
  k_compact_bricks<<<blocks_for(nc, 256), 256, 0, st>>>(bm.get(), gm.get(), cand.get(), pos.get(), nc,
                                                        L.bmask.get(), L.gmask.get(), L.bcoord.get(),
                                                        bcount.get(), gcount.get());
  CPM_CUDA_TRY(cudaGetLastError());
  bm.release();
  gm.release();
  cand.release();
  pos.release();
  CPM_CUDA_TRY(cudaMemsetAsync(L.map.get(), 0xff, mapsize * sizeof(int32_t), st));
  k_fill_map<<<blocks_for(nocc, 256), 256, 0, st>>>(L.bcoord.get(), (int32_t)nocc, g, L.map.get());
  const int64_t nB = scan_exclusive_i64(bcount.get(), nocc, st);
  const int64_t nG = scan_exclusive_i64(gcount.get(), nocc, st);
  CPM_CHECK(nB + nG < (1ll << 31) - 1, CPM_ERR_ARG, "band too large for 32-bit indices");
  L.nB = (int32_t)nB;
  L.nG = (int32_t)nG;
  L.bstart.alloc(nocc);
  L.gstart.alloc(nocc);
  k_copy_i64_to_i32<<<blocks_for(nocc, 256), 256, 0, st>>>(bcount.get(), L.bstart.get(), nocc);
  k_copy_i64_to_i32<<<blocks_for(nocc, 256), 256, 0, st>>>(gcount.get(), L.gstart.get(), nocc);
  L.brec.alloc(nocc);
  k_brick_recs<<<blocks_for(nocc, 256), 256, 0, st>>>(L.view(), L.bcoord.get(), dim, L.brec.get());
  CPM_CUDA_TRY(cudaGetLastError());

  // 6. points
  const int64_t np = nB + nG;
  L.key.alloc(np);
  L.cp.alloc((size_t)dim * np);
  L.fr64.alloc((size_t)dim * np);
  L.fr32.alloc((size_t)dim * np);
  DBuf<int32_t> err(1);
  DBuf<double> errinfo(8);
  CPM_CUDA_TRY(cudaMemsetAsync(err.get(), 0, sizeof(int32_t), st));
  CPM_CUDA_TRY(cudaMemsetAsync(errinfo.get(), 0, 8 * sizeof(double), st));
  k_emit_points<<<blocks_for(nocc * 64, 256), 256, 0, st>>>(
      s, g, L.bcoord.get(), L.bmask.get(), L.gmask.get(), L.bstart.get(), L.gstart.get(),
      (int32_t)nocc, L.nB, np, L.key.get(), L.cp.get(), L.fr64.get(), L.fr32.get(), err.get(),
      errinfo.get());
  CPM_CUDA_TRY(cudaGetLastError());
  // 7. stencils
  k_check_stencils<<<blocks_for(np, 256), 256, 0, st>>>(L.view(), L.key.get(), np, dim, err.get());
  CPM_CUDA_TRY(cudaGetLastError());
  int32_t herr = 0;
  CPM_CUDA_TRY(cudaMemcpyAsync(&herr, err.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  if (herr == 0) {
    build_ext_tiles(L, st);
    L.nbr.alloc((size_t)2 * dim * L.nB);
    k_neighbours<<<blocks_for(L.nB, 256), 256, 0, st>>>(L.view(), L.key.get(), L.nB, dim, L.nbr.get(),
                                                        err.get());
    CPM_CUDA_TRY(cudaGetLastError());
    CPM_CUDA_TRY(cudaMemcpyAsync(&herr, err.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CPM_CUDA_TRY(cudaStreamSynchronize(st));
    CPM_CHECK(herr == 0, CPM_ERR_CHECKED, "a Laplacian neighbour of the band is missing from B+");
  }
  CPM_CHECK(!(herr & 8), CPM_ERR_ARG, "the band touches the edge of the grid (enlarge the domain)");
  if (herr & 1) {
    double ei[8];
    CPM_CUDA_TRY(cudaMemcpy(ei, errinfo.get(), sizeof(ei), cudaMemcpyDeviceToHost));
    char buf[320];
    snprintf(buf, sizeof(buf),
             "closest point undefined or too far from a node of B+ (band wider than the reach): "
             "node (%g, %g, %g), cp (%.17g, %.17g, %.17g), dist2 %.17g",
             ei[0], ei[1], ei[2], ei[3], ei[4], ei[5], ei[6]);
    throw Error{CPM_ERR_REACH, buf};
  }
  CPM_CHECK(herr == 0, CPM_ERR_REACH, "an interpolation stencil leaves the band");
}

}  // namespace cpm
