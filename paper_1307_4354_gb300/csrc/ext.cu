// Closest-point extension w = E u (Sec. 3.1, Eq. 3.1; the re-extension of
// Eq. 4.2b): w_i = sum over the 4^d stencil nodes of cp(x_i) of the tensor
// product of 1-D cubic Lagrange weights times u.
//
// Tiling.  The points of B+ are grouped by the 4^d brick that holds their
// stencil base node, the points of B first in each tile (an extension over B
// alone stops at the tile's last point of B).  A tile's stencils all
// lie in the fixed 7^d box starting at the brick's first node, so one CTA
// stages that box from HBM/L2 into shared memory once (with the brick map and
// occupancy masks) and evaluates every point of the tile from it.  Each box
// row is stored as the four 16-byte-aligned windows of 4 consecutive values a
// stencil run can start at, so one run of the stencil is one vector load from
// shared memory.  Records are stored in this "E order" (band index and base
// position inside the brick in one 32-bit word, fractions SoA); results are
// written back to the band index.
#include <algorithm>

#include "ops.cuh"
#include "pair.cuh"

namespace cpm {

static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ----------------------------------------------------------------- tile build
__global__ void k_tile_slots(BrickView v, const uint64_t* key, int64_t nplus, int32_t nB, int dim,
                             int32_t* slot, int64_t* count, int64_t* count_B, int32_t* err,
                             int32_t* bbox) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nplus) return;
  const uint64_t k = key[i];
  const int bx = key_x(k) + key_ox(k), by = key_y(k) + key_oy(k);
  const int bz = dim == 3 ? key_z(k) + key_oz(k) : 0;
  int32_t b = -1;
  if (bx >= 0 && by >= 0 && bz >= 0 && bx < v.n && by < v.n && bz < v.n)
    b = v.map[((size_t)(bz >> 2) * v.nby + (by >> 2)) * v.nbx + (bx >> 2)];
  if (b < 0) {
    atomicOr(err, 1);
    slot[i] = -1;
    return;
  }
  const int32_t s = b;
  slot[i] = s;
  atomicAdd(reinterpret_cast<unsigned long long*>(count + s), 1ull);
  if (i < nB) atomicAdd(reinterpret_cast<unsigned long long*>(count_B + s), 1ull);
  // bounding box of the stencil bases inside the brick: bits (min, max) per axis
  const int l[3] = {bx & 3, by & 3, bz & 3};
  int32_t bits = 0;
  for (int a = 0; a < 3; ++a) bits |= (1 << l[a]) << (4 * a);
  atomicOr(bbox + s, bits);
}

__global__ void k_tile_flags(const int64_t* count, int64_t n, int64_t* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = count[i] > 0;
}

__global__ void k_tile_emit(const int64_t* count, const int64_t* count_B, const int64_t* offset,
                            const int64_t* tpos, const uint32_t* bcoord, const int32_t* bbox,
                            int64_t n, uint32_t* tile_brick, uint32_t* tile_box, int32_t* tile_start,
                            int32_t* tile_mid) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || count[s] == 0) return;
  const int64_t t = tpos[s];
  tile_brick[t] = bcoord[s];
  tile_start[t] = (int32_t)offset[s];
  tile_mid[t] = (int32_t)(offset[s] + count_B[s]);
  // packed per axis: lowest and highest base position used (2 bits each)
  uint32_t packed = 0;
  for (int a = 0; a < 3; ++a) {
    const uint32_t m = (uint32_t)(bbox[s] >> (4 * a)) & 15u;
    const uint32_t lo = __ffs(m) - 1, hi = 31 - __clz(m);
    packed |= (lo | (hi << 2)) << (4 * a);
  }
  tile_box[t] = packed;
}

__global__ void k_tile_scatter(const uint64_t* key, const int32_t* slot, const int64_t* offset,
                               int64_t* cursor, int64_t nplus, int dim, const double* fr64,
                               uint32_t* erec, float* efr32, double* ew64) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nplus) return;
  const int32_t s = slot[i];
  if (s < 0) return;
  const int64_t pos =
      offset[s] + (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(cursor + s), 1ull);
  const uint64_t k = key[i];
  const int bx = key_x(k) + key_ox(k), by = key_y(k) + key_oy(k);
  const int bz = dim == 3 ? key_z(k) + key_oz(k) : 0;
  erec[pos] = ((uint32_t)i << 6) | (uint32_t)((bx & 3) | ((by & 3) << 2) | ((bz & 3) << 4));
  for (int a = 0; a < dim; ++a) {
    const double sf = fr64[a * nplus + i];
    efr32[a * nplus + pos] = (float)sf;
    // 1-D cubic Lagrange weights at nodes -1, 0, 1, 2 (proof of Theorem 3.3)
    const double sm1 = sf - 1.0, sm2 = sf - 2.0, sp1 = sf + 1.0;
    const double p = sf * sm1, q = sp1 * sm2;
    ew64[(4 * a + 0) * nplus + pos] = -(p * sm2) * (1.0 / 6.0);
    ew64[(4 * a + 1) * nplus + pos] = (q * sm1) * 0.5;
    ew64[(4 * a + 2) * nplus + pos] = -(q * sf) * 0.5;
    ew64[(4 * a + 3) * nplus + pos] = (p * sp1) * (1.0 / 6.0);
  }
}

// Occupancy masks and band starts of the 2^d bricks each tile's box overlaps
// (brick (tbx + (j & 1), tby + (j >> 1 & 1), tbz + (j >> 2)) for j < 2^d).
__global__ void k_tile_tables(BrickView v, const uint32_t* tile_brick, int32_t ntiles, int dim,
                              uint64_t* tmask, int32_t* tstart) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nbr = dim == 3 ? 8 : 4;
  if (q >= (int64_t)ntiles * 8) return;
  const int32_t t = (int32_t)(q >> 3);
  const int j = (int)(q & 7);
  uint64_t m = 0;
  int32_t s0 = 0;
  if (j < nbr) {
    const uint32_t tb = tile_brick[t];
    const int bx = (int)(tb & 1023) + (j & 1), by = (int)((tb >> 10) & 1023) + ((j >> 1) & 1);
    const int bz = dim == 3 ? (int)((tb >> 20) & 1023) + (j >> 2) : 0;
    if (bx < v.nbx && by < v.nby && bz < v.nbz) {
      const int32_t b = v.map[((size_t)bz * v.nby + by) * v.nbx + bx];
      if (b >= 0) {
        m = v.bmask[b];
        s0 = v.bstart[b];
      }
    }
  }
  tmask[q] = m;
  tstart[q] = s0;
}

// Order the points of each tile by (point of G, stencil base position, band
// index): the points of B come first, points with equal bases become
// neighbours in a warp (shared-memory broadcasts instead of bank conflicts),
// and the E order no longer depends on atomics.  The keys are distinct (band
// indices are), so the ranks are a permutation.  Tiles of more than kSortMax
// points rank from global memory.
constexpr int kSortMax = 2048;
__device__ __forceinline__ uint64_t tile_sort_key(uint32_t r, int32_t nB) {
  const uint32_t idx = r >> 6;
  return ((uint64_t)(idx >= (uint32_t)nB) << 32) | ((uint64_t)(r & 63u) << 26) | idx;
}
__global__ void k_tile_sort(const int32_t* tile_start, int64_t nplus, int32_t nB, int dim,
                            const uint32_t* erec, const float* efr32, const double* ew64,
                            uint32_t* erec2, float* efr2, double* ew2) {
  __shared__ uint64_t keys[kSortMax];
  const int32_t beg = tile_start[blockIdx.x], end = tile_start[blockIdx.x + 1];
  const int n = end - beg;
  const bool in_smem = n <= kSortMax;
  if (in_smem)
    for (int j = threadIdx.x; j < n; j += blockDim.x) keys[j] = tile_sort_key(erec[beg + j], nB);
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const uint64_t kj = in_smem ? keys[j] : tile_sort_key(erec[beg + j], nB);
    int rank = 0;
    for (int i = 0; i < n; ++i)
      rank += (in_smem ? keys[i] : tile_sort_key(erec[beg + i], nB)) < kj;
    const int64_t src = beg + j, dst = beg + rank;
    erec2[dst] = erec[src];
    for (int a = 0; a < dim; ++a) efr2[a * nplus + dst] = efr32[a * nplus + src];
    for (int q = 0; q < 4 * dim; ++q) ew2[q * nplus + dst] = ew64[q * nplus + src];
  }
}

// Chunks.  Inside a tile the points are sorted by (point of G, base
// position), so the points that share one stencil base are consecutive; each
// such run (never crossing the B/G boundary) is cut into chunks of at most
// kChunkMax points.  One thread per tile counts (emit = false) or writes
// (emit = true) its chunks.
#ifndef CPM_EXT_CHUNK
#define CPM_EXT_CHUNK 2
#endif
constexpr int kChunkMax = CPM_EXT_CHUNK;
static_assert(kChunkMax >= 1 && kChunkMax <= 8, "chunk count must fit in 3 bits");

__global__ void k_tile_chunks(const int32_t* tile_start, const int32_t* tile_mid, int32_t ntiles,
                              const uint32_t* erec, bool emit, int32_t* count, int32_t* count_B,
                              const int32_t* cstart, uint32_t* echunk) {
  const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  const int32_t beg = tile_start[t], mid = tile_mid[t], end = tile_start[t + 1];
  int32_t n = 0, nB = 0;
  int32_t c0 = emit ? cstart[t] : 0;
  int32_t k = beg;
  while (k < end) {
    const uint32_t pos = erec[k] & 63u;
    const int32_t stop = k < mid ? mid : end;  // a run stays in B or in G
    int32_t j = k + 1;
    while (j < stop && j - k < kChunkMax && (erec[j] & 63u) == pos) ++j;
    if (emit) echunk[c0 + n] = (uint32_t)k | ((uint32_t)(j - k - 1) << 26);
    ++n;
    if (k < mid) ++nB;
    k = j;
  }
  if (!emit) {
    count[t] = n;
    count_B[t] = nB;
  }
}

void build_ext_tiles(Level& L, cudaStream_t st) {
  const int64_t np = L.nplus();
  CPM_CHECK(np < (1ll << 26), CPM_ERR_ARG, "more than 2^26 points on one level");
  const int64_t nslots = (int64_t)L.nbricks;
  DBuf<int32_t> slot(np);
  DBuf<int64_t> count(nslots), count_B(nslots), offset(nslots), cursor(nslots), tpos(nslots);
  DBuf<int32_t> err(1), bbox(nslots);
  CPM_CUDA_TRY(cudaMemsetAsync(bbox.get(), 0, nslots * sizeof(int32_t), st));
  CPM_CUDA_TRY(cudaMemsetAsync(count.get(), 0, nslots * sizeof(int64_t), st));
  CPM_CUDA_TRY(cudaMemsetAsync(count_B.get(), 0, nslots * sizeof(int64_t), st));
  CPM_CUDA_TRY(cudaMemsetAsync(cursor.get(), 0, nslots * sizeof(int64_t), st));
  CPM_CUDA_TRY(cudaMemsetAsync(err.get(), 0, sizeof(int32_t), st));
  k_tile_slots<<<nblk(np, 256), 256, 0, st>>>(L.view(), L.key.get(), np, L.nB, L.dim, slot.get(),
                                              count.get(), count_B.get(), err.get(), bbox.get());
  CPM_CUDA_TRY(cudaGetLastError());
  CPM_CUDA_TRY(cudaMemcpyAsync(offset.get(), count.get(), nslots * sizeof(int64_t),
                               cudaMemcpyDeviceToDevice, st));
  scan_exclusive_i64(offset.get(), nslots, st);
  k_tile_flags<<<nblk(nslots, 256), 256, 0, st>>>(count.get(), nslots, tpos.get());
  const int64_t ntiles = scan_exclusive_i64(tpos.get(), nslots, st);
  L.ntiles = (int32_t)ntiles;
  L.tile_brick.alloc(ntiles);
  L.tile_box.alloc(ntiles);
  L.tile_start.alloc(ntiles + 1);
  L.tile_mid.alloc(ntiles);
  k_tile_emit<<<nblk(nslots, 256), 256, 0, st>>>(count.get(), count_B.get(), offset.get(), tpos.get(),
                                                 L.bcoord.get(), bbox.get(), nslots,
                                                 L.tile_brick.get(), L.tile_box.get(),
                                                 L.tile_start.get(), L.tile_mid.get());
  const int32_t npi = (int32_t)np;
  CPM_CUDA_TRY(cudaMemcpyAsync(L.tile_start.get() + ntiles, &npi, sizeof(int32_t),
                               cudaMemcpyHostToDevice, st));
  L.tile_mask.alloc((size_t)8 * ntiles);
  L.tile_bstart.alloc((size_t)8 * ntiles);
  k_tile_tables<<<nblk((int64_t)8 * ntiles, 256), 256, 0, st>>>(L.view(), L.tile_brick.get(),
                                                                (int32_t)ntiles, L.dim,
                                                                L.tile_mask.get(), L.tile_bstart.get());
  L.erec.alloc(np);
  L.efr32.alloc((size_t)L.dim * np);
  L.ew64.alloc((size_t)4 * L.dim * np);
  k_tile_scatter<<<nblk(np, 256), 256, 0, st>>>(L.key.get(), slot.get(), offset.get(), cursor.get(),
                                                np, L.dim, L.fr64.get(), L.erec.get(),
                                                L.efr32.get(), L.ew64.get());
  CPM_CUDA_TRY(cudaGetLastError());
  {
    DBuf<uint32_t> erec2(np);
    DBuf<float> efr2((size_t)L.dim * np);
    DBuf<double> ew2((size_t)4 * L.dim * np);
    if (ntiles > 0)
      k_tile_sort<<<(unsigned)ntiles, 256, 0, st>>>(L.tile_start.get(), np, L.nB, L.dim,
                                                    L.erec.get(), L.efr32.get(), L.ew64.get(),
                                                    erec2.get(), efr2.get(), ew2.get());
    CPM_CUDA_TRY(cudaGetLastError());
    CPM_CUDA_TRY(cudaStreamSynchronize(st));
    L.erec = std::move(erec2);
    L.efr32 = std::move(efr2);
    L.ew64 = std::move(ew2);
  }
  // chunks of points with one stencil base
  L.tile_cstart.alloc(ntiles + 1);
  L.tile_cmid.alloc(ntiles);
  L.nchunks = 0;
  if (ntiles > 0) {
    DBuf<int32_t> ccount(ntiles), ccount_B(ntiles);
    DBuf<int64_t> coff(ntiles);
    k_tile_chunks<<<nblk(ntiles, 256), 256, 0, st>>>(L.tile_start.get(), L.tile_mid.get(),
                                                     (int32_t)ntiles, L.erec.get(), false,
                                                     ccount.get(), ccount_B.get(), nullptr, nullptr);
    CPM_CUDA_TRY(cudaGetLastError());
    std::vector<int32_t> hc(ntiles), hcb(ntiles);
    CPM_CUDA_TRY(cudaMemcpyAsync(hc.data(), ccount.get(), ntiles * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, st));
    CPM_CUDA_TRY(cudaMemcpyAsync(hcb.data(), ccount_B.get(), ntiles * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, st));
    CPM_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int32_t> hstart(ntiles + 1), hmid(ntiles);
    int64_t acc = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
      hstart[t] = (int32_t)acc;
      hmid[t] = (int32_t)(acc + hcb[t]);
      acc += hc[t];
    }
    hstart[ntiles] = (int32_t)acc;
    CPM_CHECK(acc < (1ll << 31), CPM_ERR_ARG, "too many extension chunks");
    L.nchunks = (int32_t)acc;
    CPM_CUDA_TRY(cudaMemcpyAsync(L.tile_cstart.get(), hstart.data(), (ntiles + 1) * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, st));
    CPM_CUDA_TRY(cudaMemcpyAsync(L.tile_cmid.get(), hmid.data(), ntiles * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, st));
    L.echunk.alloc(acc);
    k_tile_chunks<<<nblk(ntiles, 256), 256, 0, st>>>(L.tile_start.get(), L.tile_mid.get(),
                                                     (int32_t)ntiles, L.erec.get(), true, nullptr,
                                                     nullptr, L.tile_cstart.get(), L.echunk.get());
    CPM_CUDA_TRY(cudaGetLastError());
  }
  int32_t herr = 0;
  CPM_CUDA_TRY(cudaMemcpyAsync(&herr, err.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CPM_CUDA_TRY(cudaStreamSynchronize(st));
  CPM_CHECK(herr == 0, CPM_ERR_REACH, "a stencil base node is not a band node");
}

// ----------------------------------------------------------------- extension
// Four consecutive values from a 16-byte-aligned shared-memory window.
__device__ __forceinline__ void load4(const float* p, float v[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double v[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

__device__ __forceinline__ void store4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void store4(double* p, double a, double b, double c, double d) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
  *reinterpret_cast<double2*>(p + 2) = make_double2(c, d);
}

// Threads per CTA of the per-point extension and the staged box's row stride
// (values; each row holds the 4 windows of 4 values a stencil run can start at,
// plus padding that moves neighbouring rows to other shared-memory banks).
#ifndef CPM_EXT_THREADS
#define CPM_EXT_THREADS 64
#endif
#ifndef CPM_EXT_RS
#define CPM_EXT_RS 20
#endif
constexpr int kExtThreads = CPM_EXT_THREADS;
constexpr int kRS = CPM_EXT_RS;
static_assert(kRS >= 16 && kRS % 4 == 0, "rows hold four 16-byte windows");

template <typename T>
__device__ __forceinline__ T dot4(const T w[4], const T* v) {
  return w[0] * v[0] + w[1] * v[1] + w[2] * v[2] + w[3] * v[3];
}

// Cubic weights of one point: FP64 from the precomputed E-order table, FP32
// from the fraction (closed forms of the proof of Theorem 3.3).
template <typename T, int DIM>
struct PointWeights;
template <int DIM>
struct PointWeights<double, DIM> {
  double wx[4], wy[4], wz[4];
  __device__ __forceinline__ void load(const LevelView<double>& L, int32_t k) {
    const int64_t np = L.nplus;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      wx[j] = __ldg(L.ew64 + j * np + k);
      wy[j] = __ldg(L.ew64 + (4 + j) * np + k);
      wz[j] = DIM == 3 ? __ldg(L.ew64 + (8 + j) * np + k) : 0.0;
    }
  }
};
template <int DIM>
struct PointWeights<float, DIM> {
  float wx[4], wy[4], wz[4];
  __device__ __forceinline__ static void cubic(float s, float w[4]) {
    const float sm1 = s - 1.f, sm2 = s - 2.f, sp1 = s + 1.f;
    const float p = s * sm1, q = sp1 * sm2;
    w[0] = (p * sm2) * (-1.f / 6.f);
    w[1] = (q * sm1) * 0.5f;
    w[2] = (q * s) * -0.5f;
    w[3] = (p * sp1) * (1.f / 6.f);
  }
  __device__ __forceinline__ void load(const LevelView<float>& L, int32_t k) {
    const int64_t np = L.nplus;
    cubic(__ldg(L.efr + k), wx);
    cubic(__ldg(L.efr + np + k), wy);
    if (DIM == 3) cubic(__ldg(L.efr + 2 * np + k), wz);
  }
};

// The separable contraction of one point's 4^d stencil read from the windows
// at base (row stride 20 values, plane stride 7 rows).  FP64: x, then y, then
// z.  FP32: y and z first with paired FMAs (two x positions per instruction,
// Blackwell's packed FP32 FMA), then x: 32 + 8 + 2 packed operations instead
// of 84 scalar ones.
template <int DIM>
__device__ __forceinline__ double contract(const double* base, const PointWeights<double, DIM>& pw) {
  constexpr int RS = kRS;
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < (DIM == 3 ? 4 : 1); ++c) {
    double accy = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      double vv[4];
      load4(base + (c * 7 + b) * RS, vv);
      accy += pw.wy[b] * dot4(pw.wx, vv);
    }
    acc += (DIM == 3 ? pw.wz[c] : 1.0) * accy;
  }
  return acc;
}
template <int DIM>
__device__ __forceinline__ float contract(const float* base, const PointWeights<float, DIM>& pw) {
  constexpr int RS = kRS;
  float2 q01 = make_float2(0.f, 0.f), q23 = q01;
#pragma unroll
  for (int c = 0; c < (DIM == 3 ? 4 : 1); ++c) {
    float2 p01, p23;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float4 v = *reinterpret_cast<const float4*>(base + (c * 7 + b) * RS);
      const float2 wyb = make_float2(pw.wy[b], pw.wy[b]);
      if (b == 0) {
        p01 = __fmul2_rn(wyb, make_float2(v.x, v.y));
        p23 = __fmul2_rn(wyb, make_float2(v.z, v.w));
      } else {
        p01 = __ffma2_rn(wyb, make_float2(v.x, v.y), p01);
        p23 = __ffma2_rn(wyb, make_float2(v.z, v.w), p23);
      }
    }
    const float wzc = DIM == 3 ? pw.wz[c] : 1.f;
    const float2 wz2 = make_float2(wzc, wzc);
    if (c == 0) {
      q01 = __fmul2_rn(wz2, p01);
      q23 = __fmul2_rn(wz2, p23);
    } else {
      q01 = __ffma2_rn(wz2, p01, q01);
      q23 = __ffma2_rn(wz2, p23, q23);
    }
  }
  const float2 t = __ffma2_rn(make_float2(pw.wx[2], pw.wx[3]), q23,
                              __fmul2_rn(make_float2(pw.wx[0], pw.wx[1]), q01));
  return t.x + t.y;
}

// Staging of a tile's box.  Shared memory: NZ*7 box rows, each 4 windows of 4
// values plus one pad window (row stride 20 values spreads rows over banks).
// The tile's bases span [lo, hi] per axis, so box nodes lo .. hi+3 are
// staged.  Thread r owns box row (y, z): it reads the row's band nodes in
// order (consecutive band indices within each of the row's two bricks, so one
// popcount per brick gives the start) and writes the row's windows
// x0 = lo_x .. hi_x, four values each, as vector stores.  REL: values are
// staged relative to ref.  Returns after a __syncthreads with the box ready.
template <typename T, int DIM, bool REL>
struct TileBox {
  static constexpr int NZ = DIM == 3 ? 7 : 1;
  static constexpr int RS = kRS;
  static constexpr int NB = DIM == 3 ? 8 : 4;  // bricks overlapping the box
  __align__(16) T win[NZ * 7 * RS];
  uint32_t mask[NB][2];
  int32_t start[NB][2];
};

// Box row r of a tile (box rows run over y fastest, then z): its position,
// the x range of its windows, and the band indices of its first node in each
// of the two bricks it crosses (band nodes of a brick row are consecutive, so
// one popcount per brick gives the start).  False if r is past the last row.
struct BoxRow {
  int y, z, xlo, xhi;
  uint32_t rba, rbb;  // occupancy of the row's 4 nodes in the low / high brick
  int32_t ca, cb;     // band index of the row's first node at x >= xlo / x >= 4
};
template <int NB>
__device__ __forceinline__ bool box_row(const uint32_t (&mask)[NB][2], const int32_t (&start)[NB][2],
                                        uint32_t tbox, int dim, int r, BoxRow& b) {
  b.xlo = tbox & 3;
  b.xhi = (tbox >> 2) & 3;
  const int ylo = (tbox >> 4) & 3, yhi = (tbox >> 6) & 3;
  const int zlo = dim == 3 ? (tbox >> 8) & 3 : 0, zhi = dim == 3 ? ((tbox >> 10) & 3) + 3 : 0;
  const int ny = yhi + 4 - ylo;
  if (r >= ny * (zhi + 1 - zlo)) return false;
  b.y = ylo + r % ny;
  b.z = zlo + r / ny;
  const int jyz = ((b.y >> 2) << 1) | ((b.z >> 2) << 2);
  const int half = (b.z >> 1) & 1;
  const int shift = ((b.y & 3) << 2) | ((b.z & 1) << 4);
  const uint32_t wa = mask[jyz][half], wb = mask[jyz | 1][half];
  b.rba = (wa >> shift) & 0xFu;
  b.rbb = (wb >> shift) & 0xFu;
  const uint32_t below = (1u << shift) - 1u;
  b.ca = start[jyz][half] + __popc(wa & below) + __popc(b.rba & ((1u << b.xlo) - 1u));
  b.cb = start[jyz | 1][half] + __popc(wb & below);
  return true;
}

// The tile's brick masks and band starts into shared memory (threads < NB).
template <int NB>
__device__ __forceinline__ void load_box_bricks(const uint64_t* tile_mask, const int32_t* tile_bstart,
                                                int32_t tile, uint32_t (&mask)[NB][2],
                                                int32_t (&start)[NB][2]) {
  if (threadIdx.x < NB) {
    const int j = threadIdx.x;
    const uint64_t m = __ldg(tile_mask + 8 * (int64_t)tile + j);
    const int32_t s0 = __ldg(tile_bstart + 8 * (int64_t)tile + j);
    mask[j][0] = (uint32_t)m;
    mask[j][1] = (uint32_t)(m >> 32);
    start[j][0] = s0;
    start[j][1] = s0 + __popc((uint32_t)m);
  }
}

template <typename T, int DIM, bool REL, int NT>
__device__ __forceinline__ T stage_box(const LevelView<T>& L, const T* __restrict__ u, int32_t tile,
                                       uint32_t tbox, TileBox<T, DIM, REL>& sm) {
  constexpr int RS = TileBox<T, DIM, REL>::RS;
  load_box_bricks(L.tile_mask, L.tile_bstart, tile, sm.mask, sm.start);
  __syncthreads();
  const T ref = REL ? __ldg(u + sm.start[0][0]) : T(0);
  BoxRow b;
  for (int r = threadIdx.x; box_row(sm.mask, sm.start, tbox, DIM, r, b); r += NT) {
    T v[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      const int x = b.xlo + i;
      v[i] = T(0);
      if (x <= b.xhi + 3) {
        const bool hi = x >= 4;
        if (((hi ? b.rbb : b.rba) >> (x & 3)) & 1u) {
          v[i] = __ldg(u + (hi ? b.cb++ : b.ca++));
          if (REL) v[i] -= ref;
        }
      }
    }
    T* row = sm.win + (b.z * 7 + b.y) * RS;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (b.xlo + i <= b.xhi) store4(row + 4 * (b.xlo + i), v[i], v[i + 1], v[i + 2], v[i + 3]);
  }
  __syncthreads();
  return ref;
}

// One CTA per tile, one thread per point.  REL (FP64 residual form): the
// tile's values are staged relative to one reference value (u at the first
// band node of the base brick), the kernel writes delta_j = (E u)_j - ref and
// ref_j = ref.  The subtraction comes before the weighted sum, so delta
// carries rounding errors relative to the small differences only, not to |u|.
template <typename T, int DIM, bool REL = false>
__global__ void __launch_bounds__(kExtThreads) k_extend_tiles(LevelView<T> L, const T* __restrict__ u,
                                                              T* __restrict__ w, bool with_ghost,
                                                              T* __restrict__ refv) {
  constexpr int RS = kRS;
  __shared__ TileBox<T, DIM, REL> sm;
  const int32_t tile = blockIdx.x;
  const uint32_t tbox = __ldg(L.tile_box + tile);
  const int32_t beg = __ldg(L.tile_start + tile);
  const int32_t end = with_ghost ? __ldg(L.tile_start + tile + 1) : __ldg(L.tile_mid + tile);
  if (beg == end) return;  // a tile of ghost points only, extension over B
  // this thread's first point: issue its record loads before staging
  int32_t k = beg + threadIdx.x;
  uint32_t rec = 0;
  PointWeights<T, DIM> pw;
  if (k < end) {
    rec = __ldg(L.erec + k);
    pw.load(L, k);
  }
  const T ref = stage_box<T, DIM, REL, kExtThreads>(L, u, tile, tbox, sm);
  for (; k < end; k += kExtThreads) {
    const T* base = sm.win + ((rec >> 4) & 3) * 7 * RS + ((rec >> 2) & 3) * RS + (rec & 3) * 4;
    w[rec >> 6] = contract<DIM>(base, pw);
    if (REL) refv[rec >> 6] = ref;
    const int32_t kn = k + kExtThreads;
    if (kn < end) {
      rec = __ldg(L.erec + kn);
      pw.load(L, kn);
    }
  }
}

// ------------------------------------------------- relative form in FP32 pairs
// The outer residual's extension (the relative form of the FP64 kernel above)
// evaluated in FP32-pair arithmetic (pair.cuh) on the FP32 pipe.  Per tile the
// reference is ref = u at the last band node of the tile's base brick (the
// brick holding its points' stencil bases, box brick 0, which holds at least
// those bases), rounded to float, so that reference differences are exact in
// pairs; the box is staged as d = u - ref (one FP64 subtraction per node),
// split into hi and lo planes.  Per point the 4^d contraction runs in pairs,
// y for each (z, x) with two x positions per packed instruction, then z, then
// x, with the 1-D weights split into pairs when the level was built.  Output:
// delta_j = (E u)_j - ref_j as a pair and ref_j, for every point of B+.
template <int DIM>
struct PairBox {
  static constexpr int NZ = DIM == 3 ? 7 : 1;
  static constexpr int NB = DIM == 3 ? 8 : 4;
  __align__(16) float hi[NZ * 7 * kRS];
  __align__(16) float lo[NZ * 7 * kRS];
  uint32_t mask[NB][2];
  int32_t start[NB][2];
  uint32_t dmax;  // largest |hi| staged (float bits)
};

template <int DIM>
__device__ __forceinline__ float stage_box_pair(const LevelView<double>& L, const double* __restrict__ u,
                                                int32_t tile, uint32_t tbox, PairBox<DIM>& sm) {
  load_box_bricks(L.tile_mask, L.tile_bstart, tile, sm.mask, sm.start);
  if (threadIdx.x == 0) sm.dmax = 0u;
  __syncthreads();
  // brick 0 holds the tile's stencil bases, which are band nodes (checked when
  // the band is built); the clamp only keeps the index inside B regardless
  const int32_t last = min(max(sm.start[0][1] + __popc(sm.mask[0][1]) - 1, 0), L.nB - 1);
  const float ref = (float)__ldg(u + last);
  const double refd = (double)ref;
  float amax = 0.f;
  BoxRow b;
  for (int r = threadIdx.x; box_row(sm.mask, sm.start, tbox, DIM, r, b); r += kExtThreads) {
    float vh[7], vl[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      const int x = b.xlo + i;
      vh[i] = vl[i] = 0.f;
      if (x <= b.xhi + 3) {
        const bool hi = x >= 4;
        if (((hi ? b.rbb : b.rba) >> (x & 3)) & 1u) {
          const float2 d = pair_split(__ldg(u + (hi ? b.cb++ : b.ca++)) - refd);
          vh[i] = d.x;
          vl[i] = d.y;
          amax = fmaxf(amax, fabsf(d.x));
        }
      }
    }
    const int o = (b.z * 7 + b.y) * kRS;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (b.xlo + i <= b.xhi) {
        store4(sm.hi + o + 4 * (b.xlo + i), vh[i], vh[i + 1], vh[i + 2], vh[i + 3]);
        store4(sm.lo + o + 4 * (b.xlo + i), vl[i], vl[i + 1], vl[i + 2], vl[i + 3]);
      }
  }
  uint32_t am = __float_as_uint(amax);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) am = max(am, __shfl_xor_sync(0xffffffffu, am, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&sm.dmax, am);
  __syncthreads();
  return ref;
}

// The pair contraction of one point from the windows at offset o.
template <int DIM>
__device__ __forceinline__ void contract_pair(const PairBox<DIM>& sm, int o, const float2 (&w)[3][4],
                                              float& dh, float& dl) {
  Pair2 q01{}, q23{};
#pragma unroll
  for (int c = 0; c < (DIM == 3 ? 4 : 1); ++c) {
    Pair2 p01, p23;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int ob = o + (c * 7 + b) * kRS;
      const float4 xh = *reinterpret_cast<const float4*>(sm.hi + ob);
      const float4 xl = *reinterpret_cast<const float4*>(sm.lo + ob);
      const PairW2 wy = pw2(w[1][b]);
      if (b == 0) {
        p01 = pmul(wy, make_float2(xh.x, xh.y), make_float2(xl.x, xl.y));
        p23 = pmul(wy, make_float2(xh.z, xh.w), make_float2(xl.z, xl.w));
      } else {
        pmul_acc(wy, make_float2(xh.x, xh.y), make_float2(xl.x, xl.y), p01);
        pmul_acc(wy, make_float2(xh.z, xh.w), make_float2(xl.z, xl.w), p23);
      }
    }
    if (DIM == 2) {
      q01 = p01;
      q23 = p23;
    } else {
      const PairW2 wz = pw2(w[2][c]);
      if (c == 0) {
        q01 = pmul(wz, p01.h, p01.l);
        q23 = pmul(wz, p23.h, p23.l);
      } else {
        pmul_acc(wz, p01.h, p01.l, q01);
        pmul_acc(wz, p23.h, p23.l, q23);
      }
    }
  }
  // x: lanes (0, 1) then (2, 3) into one pair per lane, then the two lanes
  Pair2 s = pmul(pw2(w[0][0], w[0][1]), q01.h, q01.l);
  pmul_acc(pw2(w[0][2], w[0][3]), q23.h, q23.l, s);
  float h, t;
  two_sum(s.h.x, s.h.y, h, t);
  const float l = __fadd_rn(__fadd_rn(s.l.x, s.l.y), t);
  fast_two_sum(h, l, dh, dl);
}

template <int DIM>
// (72 registers, 14 CTAs per SM; asking for 16 CTAs gave 64 registers with a
// small spill and no gain: 396 us against 389 us at dx = 1/256)
__global__ void __launch_bounds__(kExtThreads) k_extend_pair(LevelView<double> L, const double* __restrict__ u,
                                                             float2* __restrict__ delta,
                                                             float* __restrict__ refv, uint32_t* dmax) {
  __shared__ PairBox<DIM> sm;
  const int32_t tile = blockIdx.x;
  const uint32_t tbox = __ldg(L.tile_box + tile);
  const int32_t beg = __ldg(L.tile_start + tile), end = __ldg(L.tile_start + tile + 1);
  if (beg == end) return;
  const int64_t np = L.nplus;
  int32_t k = beg + threadIdx.x;
  uint32_t rec = 0;
  float2 w[3][4];
  auto load_w = [&](int32_t kk) {
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int j = 0; j < 4; ++j) w[a][j] = __ldg(L.ewp + (4 * a + j) * np + kk);
  };
  if (k < end) {
    rec = __ldg(L.erec + k);
    load_w(k);
  }
  const float ref = stage_box_pair<DIM>(L, u, tile, tbox, sm);
  if (threadIdx.x == 0) atomicMax(dmax + (tile & (kPairSlots - 1)), sm.dmax);
  for (; k < end; k += kExtThreads) {
    const int o = ((rec >> 4) & 3) * 7 * kRS + ((rec >> 2) & 3) * kRS + (rec & 3) * 4;
    float dh, dl;
    contract_pair<DIM>(sm, o, w, dh, dl);
    delta[rec >> 6] = make_float2(dh, dl);
    refv[rec >> 6] = ref;
    const int32_t kn = k + kExtThreads;
    if (kn < end) {
      rec = __ldg(L.erec + kn);
      load_w(kn);
    }
  }
}

// FP32 extension, persistent and software-pipelined: a fixed grid of CTAs, each
// looping over tiles blockIdx.x, blockIdx.x + gridDim.x, ...; while it
// evaluates the points of one tile from one shared-memory box it has the row
// loads of its next tile in flight (into registers, one box row per thread)
// and writes them into the other box afterwards, so the staging latency of a
// tile hides behind the arithmetic of the previous one.
#ifndef CPM_EXT_PIPELINED
#define CPM_EXT_PIPELINED 0
#endif
constexpr bool kPipelined = CPM_EXT_PIPELINED != 0;
constexpr int kPipeThreads = 64;

template <int DIM>
__global__ void __launch_bounds__(kPipeThreads) k_extend_pipe(LevelView<float> L,
                                                              const float* __restrict__ u,
                                                              float* __restrict__ w, bool with_ghost) {
  constexpr int RS = kRS;
  constexpr int NZ = DIM == 3 ? 7 : 1;
  constexpr int NB = DIM == 3 ? 8 : 4;
  __shared__ __align__(16) float win[2][NZ * 7 * RS];
  __shared__ uint32_t smask[2][NB][2];
  __shared__ int32_t sstart[2][NB][2];
  static_assert(kPipeThreads >= 49, "one box row per thread");
  int32_t tile = blockIdx.x;
  if (tile >= L.ntiles) return;
  // the rows of tile t: addresses from its masks in buffer b, values into v
  auto load_rows = [&](int32_t t, int b, float v[7], int& ylo_o, int& z_o, int& y_o, int& xlo_o,
                       int& xhi_o) -> bool {
    const uint32_t tbox = __ldg(L.tile_box + t);
    const int xlo = tbox & 3, xhi = (tbox >> 2) & 3;
    const int ylo = (tbox >> 4) & 3, yhi = (tbox >> 6) & 3;
    const int zlo = DIM == 3 ? (tbox >> 8) & 3 : 0, zhi = DIM == 3 ? ((tbox >> 10) & 3) + 3 : 0;
    const int ny = yhi + 4 - ylo;
    const int r = threadIdx.x;
    if (r >= ny * (zhi + 1 - zlo)) return false;
    const int y = ylo + r % ny, z = zlo + r / ny;
    const int jyz = ((y >> 2) << 1) | ((z >> 2) << 2);
    const int half = (z >> 1) & 1;
    const int shift = ((y & 3) << 2) | ((z & 1) << 4);
    const uint32_t wa = smask[b][jyz][half], wb = smask[b][jyz | 1][half];
    const uint32_t rba = (wa >> shift) & 0xFu, rbb = (wb >> shift) & 0xFu;
    const uint32_t below = (1u << shift) - 1u;
    int32_t ca = sstart[b][jyz][half] + __popc(wa & below) + __popc(rba & ((1u << xlo) - 1u));
    int32_t cb = sstart[b][jyz | 1][half] + __popc(wb & below);
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      const int x = xlo + i;
      v[i] = 0.f;
      if (x <= xhi + 3) {
        const bool hi = x >= 4;
        if (((hi ? rbb : rba) >> (x & 3)) & 1u) v[i] = __ldg(u + (hi ? cb++ : ca++));
      }
    }
    y_o = y;
    z_o = z;
    ylo_o = ylo;
    xlo_o = xlo;
    xhi_o = xhi;
    return true;
  };
  auto load_masks = [&](int32_t t, int b) {
    if (threadIdx.x < NB) {
      const int j = threadIdx.x;
      const uint64_t m = __ldg(L.tile_mask + 8 * (int64_t)t + j);
      const int32_t s0 = __ldg(L.tile_bstart + 8 * (int64_t)t + j);
      smask[b][j][0] = (uint32_t)m;
      smask[b][j][1] = (uint32_t)(m >> 32);
      sstart[b][j][0] = s0;
      sstart[b][j][1] = s0 + __popc((uint32_t)m);
    }
  };
  auto store_rows = [&](int b, const float v[7], int y, int z, int xlo, int xhi) {
    float* row = win[b] + (z * 7 + y) * RS;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (xlo + i <= xhi) store4(row + 4 * (xlo + i), v[i], v[i + 1], v[i + 2], v[i + 3]);
  };
  // prologue: the first tile's box
  int buf = 0;
  load_masks(tile, 0);
  __syncthreads();
  {
    float v[7];
    int ylo, y, z, xlo, xhi;
    if (load_rows(tile, 0, v, ylo, z, y, xlo, xhi)) store_rows(0, v, y, z, xlo, xhi);
  }
  __syncthreads();
  for (; tile < L.ntiles; tile += gridDim.x) {
    const int32_t next = tile + gridDim.x;
    const bool has_next = next < L.ntiles;
    if (has_next) load_masks(next, buf ^ 1);
    __syncthreads();
    float v[7];
    int ylo = 0, y = 0, z = 0, xlo = 0, xhi = 0;
    const bool row = has_next && load_rows(next, buf ^ 1, v, ylo, z, y, xlo, xhi);
    // the points of this tile from win[buf]
    const int32_t beg = __ldg(L.tile_start + tile);
    const int32_t end = with_ghost ? __ldg(L.tile_start + tile + 1) : __ldg(L.tile_mid + tile);
    for (int32_t k = beg + threadIdx.x; k < end; k += kPipeThreads) {
      const uint32_t rec = __ldg(L.erec + k);
      PointWeights<float, DIM> pw;
      pw.load(L, k);
      const float* base = win[buf] + ((rec >> 4) & 3) * 7 * RS + ((rec >> 2) & 3) * RS + (rec & 3) * 4;
      w[rec >> 6] = contract<DIM>(base, pw);
    }
    if (row) store_rows(buf ^ 1, v, y, z, xlo, xhi);
    __syncthreads();
    buf ^= 1;
  }
}

#ifndef CPM_EXT_CHUNKED
#define CPM_EXT_CHUNKED 0
#endif
constexpr bool kChunked = CPM_EXT_CHUNKED != 0;
#ifndef CPM_EXT_CHUNK_THREADS
#define CPM_EXT_CHUNK_THREADS 64
#endif
constexpr int kChunkThreads = CPM_EXT_CHUNK_THREADS;

// One thread per chunk (up to kChunkMax points with one stencil base): the
// thread streams the base's 4^d stencil rows from the staged box, one 16-byte
// shared-memory load per row, and accumulates every point of the chunk from
// each row, in the order of `contract` (y and z first with paired FMAs, then
// x), so the results equal the per-point kernel's bit for bit.  A chunk of one
// point repeats it in the second slot and stores it once.
template <int DIM>
__global__ void __launch_bounds__(kChunkThreads) k_extend_chunks(LevelView<float> L,
                                                                 const float* __restrict__ u,
                                                                 float* __restrict__ w, bool with_ghost) {
  constexpr int RS = kRS;
  constexpr int NC = DIM == 3 ? 4 : 1;
  __shared__ TileBox<float, DIM, false> sm;
  const int32_t tile = blockIdx.x;
  const uint32_t tbox = __ldg(L.tile_box + tile);
  const int32_t cbeg = __ldg(L.tile_cstart + tile);
  const int32_t cend = with_ghost ? __ldg(L.tile_cstart + tile + 1) : __ldg(L.tile_cmid + tile);
  if (cbeg == cend) return;  // a tile of ghost points only, extension over B
  int32_t c = cbeg + threadIdx.x;
  uint32_t ch = c < cend ? __ldg(L.echunk + c) : 0u;
  stage_box<float, DIM, false, kChunkThreads>(L, u, tile, tbox, sm);
  for (; c < cend; c += kChunkThreads) {
    const int32_t k0 = (int32_t)(ch & 0x3FFFFFFu);
    const int cnt = (int)(ch >> 26) + 1;
    PointWeights<float, DIM> pw[kChunkMax];
    uint32_t rec[kChunkMax];
#pragma unroll
    for (int j = 0; j < kChunkMax; ++j) {
      const int32_t kj = k0 + (j < cnt ? j : 0);
      rec[j] = __ldg(L.erec + kj);
      pw[j].load(L, kj);
    }
    const int32_t cn = c + kChunkThreads;
    if (cn < cend) ch = __ldg(L.echunk + cn);
    const float* base = sm.win + ((rec[0] >> 4) & 3) * 7 * RS + ((rec[0] >> 2) & 3) * RS + (rec[0] & 3) * 4;
    float2 q01[kChunkMax], q23[kChunkMax];
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
      float2 p01[kChunkMax], p23[kChunkMax];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float4 v = *reinterpret_cast<const float4*>(base + (cc * 7 + b) * RS);
#pragma unroll
        for (int j = 0; j < kChunkMax; ++j) {
          const float2 wyb = make_float2(pw[j].wy[b], pw[j].wy[b]);
          if (b == 0) {
            p01[j] = __fmul2_rn(wyb, make_float2(v.x, v.y));
            p23[j] = __fmul2_rn(wyb, make_float2(v.z, v.w));
          } else {
            p01[j] = __ffma2_rn(wyb, make_float2(v.x, v.y), p01[j]);
            p23[j] = __ffma2_rn(wyb, make_float2(v.z, v.w), p23[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kChunkMax; ++j) {
        const float wzc = DIM == 3 ? pw[j].wz[cc] : 1.f;
        const float2 wz2 = make_float2(wzc, wzc);
        if (cc == 0) {
          q01[j] = __fmul2_rn(wz2, p01[j]);
          q23[j] = __fmul2_rn(wz2, p23[j]);
        } else {
          q01[j] = __ffma2_rn(wz2, p01[j], q01[j]);
          q23[j] = __ffma2_rn(wz2, p23[j], q23[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kChunkMax; ++j) {
      if (j < cnt) {
        const float2 t = __ffma2_rn(make_float2(pw[j].wx[2], pw[j].wx[3]), q23[j],
                                    __fmul2_rn(make_float2(pw[j].wx[0], pw[j].wx[1]), q01[j]));
        w[rec[j] >> 6] = t.x + t.y;
      }
    }
  }
}

// The FP32 extension's work decomposition ("tile variant") of a level:
// EXT_TILES one CTA per tile, one thread per point; EXT_PIPE persistent CTAs
// with the next tile's staging in flight; EXT_CHUNKS one thread per chunk of
// points with one stencil base.  The hierarchy picks one per level by timing
// (tune_extension).  CPM_EXT_PIPELINED / CPM_EXT_CHUNKED force a variant.
template <typename T>
static void extend_variant(const LevelView<T>& L, int variant, const T* u, T* w, bool with_ghost,
                           cudaStream_t st) {
  const int32_t nt = L.ntiles;
  if constexpr (sizeof(T) == 4) {
    if (variant == EXT_PIPE) {
      const unsigned grid = (unsigned)std::min<int32_t>(nt, 152 * 16);
      if (L.dim == 3)
        k_extend_pipe<3><<<grid, kPipeThreads, 0, st>>>(L, u, w, with_ghost);
      else
        k_extend_pipe<2><<<grid, kPipeThreads, 0, st>>>(L, u, w, with_ghost);
      return;
    }
    if (variant == EXT_CHUNKS) {
      if (L.dim == 3)
        k_extend_chunks<3><<<nt, kChunkThreads, 0, st>>>(L, u, w, with_ghost);
      else
        k_extend_chunks<2><<<nt, kChunkThreads, 0, st>>>(L, u, w, with_ghost);
      return;
    }
  }
  if (L.dim == 3)
    k_extend_tiles<T, 3><<<nt, kExtThreads, 0, st>>>(L, u, w, with_ghost, nullptr);
  else
    k_extend_tiles<T, 2><<<nt, kExtThreads, 0, st>>>(L, u, w, with_ghost, nullptr);
}

template <typename T>
void launch_extend(const LevelView<T>& L, const T* u, T* w, int32_t npts, cudaStream_t st) {
  if (npts <= 0) return;
  if (L.ntiles <= 0) return;
  int variant = L.ext_variant;
  if (kPipelined) variant = EXT_PIPE;
  if (kChunked) variant = EXT_CHUNKS;
  extend_variant<T>(L, variant, u, w, npts > L.nB, st);
  count_launch();
}

int tune_extension(const LevelView<float>& L, const float* u, float* w, cudaStream_t st, float ms[3]) {
  int best = EXT_TILES;
  for (int v = 0; v < 3; ++v) ms[v] = 0.f;
  if (L.ntiles <= 0) return best;
  cudaEvent_t e0, e1;
  CPM_CUDA_TRY(cudaEventCreate(&e0));
  CPM_CUDA_TRY(cudaEventCreate(&e1));
  constexpr int kReps = 3;
  for (int v = 0; v < 3; ++v) {
    extend_variant<float>(L, v, u, w, true, st);  // warm-up
    CPM_CUDA_TRY(cudaEventRecord(e0, st));
    for (int r = 0; r < kReps; ++r) extend_variant<float>(L, v, u, w, true, st);
    CPM_CUDA_TRY(cudaEventRecord(e1, st));
    CPM_CUDA_TRY(cudaEventSynchronize(e1));
    CPM_CUDA_TRY(cudaEventElapsedTime(&ms[v], e0, e1));
    ms[v] /= kReps;
    if (ms[v] < ms[best]) best = v;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CPM_CUDA_TRY(cudaGetLastError());
  return best;
}

template <typename T>
void launch_extend_rel(const LevelView<T>& L, const T* u, T* delta, T* refv, cudaStream_t st) {
  const int32_t nt = L.ntiles;
  if (nt <= 0) return;
  if (L.dim == 3)
    k_extend_tiles<T, 3, true><<<nt, kExtThreads, 0, st>>>(L, u, delta, true, refv);
  else
    k_extend_tiles<T, 2, true><<<nt, kExtThreads, 0, st>>>(L, u, delta, true, refv);
  count_launch();
}
__global__ void k_pair_weights(const double* w, float2* wp, int64_t n) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) wp[q] = pair_split(w[q]);
}

void build_pair_weights(Level& L, cudaStream_t st) {
  const int64_t n = (int64_t)4 * L.dim * L.nplus();
  L.ewp.alloc((size_t)n);
  if (n > 0) k_pair_weights<<<nblk(n, 256), 256, 0, st>>>(L.ew64.get(), L.ewp.get(), n);
  CPM_CUDA_TRY(cudaGetLastError());
}

void launch_extend_pair(const LevelView<double>& L, const double* u, float2* delta, float* refv,
                        uint32_t* dmax, cudaStream_t st) {
  const int32_t nt = L.ntiles;
  if (nt <= 0) return;
  CPM_CHECK(L.ewp != nullptr, CPM_ERR_ARG, "pair weights not built");
  if (L.dim == 3)
    k_extend_pair<3><<<nt, kExtThreads, 0, st>>>(L, u, delta, refv, dmax);
  else
    k_extend_pair<2><<<nt, kExtThreads, 0, st>>>(L, u, delta, refv, dmax);
  count_launch();
}

template void launch_extend_rel<double>(const LevelView<double>&, const double*, double*, double*,
                                        cudaStream_t);
template void launch_extend_rel<float>(const LevelView<float>&, const float*, float*, float*,
                                       cudaStream_t);

template void launch_extend<double>(const LevelView<double>&, const double*, double*, int32_t,
                                    cudaStream_t);
template void launch_extend<float>(const LevelView<float>&, const float*, float*, int32_t,
                                   cudaStream_t);

}  // namespace cpm
