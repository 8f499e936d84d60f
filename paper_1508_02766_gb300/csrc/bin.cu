// Linear binning (Sec. 2, first step): each sample inside the grid spreads a
// unit mass over its 2^d neighbouring nodes with integer weights in units of
// 2^-32 that sum to exactly 2^32 (so the counts sum to n, Sec. 3 footnote).
// Integer addition is associative, so the counts are bit-identical whatever
// order the additions happen in.
//
// Two implementations of the same arithmetic:
//   direct  one pass, 64-bit integer atomics straight into the counts (no
//           scratch; bound by the rate of scattered L2 sector operations,
//           ~2^(d-1) + 1/2 per sample);
//   tiled   the samples partitioned by the grid tile of their base node, then
//           each tile accumulated in shared memory and written once (no
//           zeroing pass, no global atomics on the counts):
//             count    records per tile (a sample whose base node is on a
//                      tile's upper face also feeds the next tile(s): one
//                      record per tile it touches), each block keeping its
//                      range inside every tile's bucket
//             scatter  bucket starts and work items of at most kItemRecords
//                      records (every block scans the tile counts), then
//                      16-byte records {q_0, q_1, q_2, tile-local base and
//                      corner mask} written into the block's ranges
//             accum    per work item, 32-bit shared atomics on split sums
//                      (exact), then every cell of the tile stored (tiles
//                      split into several items are zeroed during scatter
//                      and their items add instead)
//           the scatter and accumulation kernels are programmatic dependents
//           of the kernel before each.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "kde_debug.cuh"
#include "kde_internal.h"
#include "pdl.cuh"

namespace {

constexpr unsigned long long kOne = 1ull << 32;

// floor((w q + 2^31) / 2^32) for 0 <= w <= 2^32 and 0 <= q < 2^32, exactly,
// in 32-bit arithmetic: with w = wh 2^32 + wl (wh in {0, 1}) and
// wl q = H 2^32 + Lo, the value is wh q + H + [Lo >= 2^31].
__device__ __forceinline__ unsigned mulhi_round(unsigned long long w, unsigned q) {
  const unsigned wl = (unsigned)w, wh = (unsigned)(w >> 32);
  return wh * q + __umulhi(wl, q) + ((wl * q) >> 31);
}

template <typename T>
struct BinAxis {
  T lo;      // lo rounded to X's type
  T s;       // (M-1)/(hi-lo) computed in FP64, rounded to X's type
  T top;     // M - 1 in X's type
  int64_t stride;
  int M;
  int tile;       // tile extent along this axis (power of two)
  int tile_log2;
  int ntiles;     // tiles along this axis
  int tstride;    // stride of this axis in the tile index
  int lstride;    // stride of this axis inside a tile (row-major, last axis fastest)
};

template <typename T>
struct BinParams {
  BinAxis<T> ax[KDE_MAX_D];
  int64_t cells;   // prod(M): the counts array's length
};

__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Position of one coordinate, normalised: node i and q = round-half-even(f 2^32)
// with 0 <= q < 2^32.  A fraction that rounds to exactly 2^32 (f = 1) is
// written as (i + 1, q = 0), which gives bit-identical weights:
// floor((w 2^32 + 2^31) / 2^32) = w and floor((w 0 + 2^31) / 2^32) = 0.
// The scaling by 2^32 is exact in either type; FP32 inputs stay in 32-bit
// arithmetic throughout.  Returns false if t is outside [0, M-1] or NaN.
__device__ __forceinline__ bool fixed_frac(float f, int& i, unsigned& q) {
  if (f == 1.0f) {
    i += 1;
    q = 0;
  } else {
    q = __float2uint_rn(f * 4294967296.0f);  // f 2^32 < 2^32 exactly
  }
  return true;
}
__device__ __forceinline__ bool fixed_frac(double f, int& i, unsigned& q) {
  unsigned long long Q = __double2ull_rn(f * 4294967296.0);
  if (Q == kOne) {
    i += 1;
    q = 0;
  } else {
    q = (unsigned)Q;
  }
  return true;
}

template <typename T>
__device__ __forceinline__ bool axis_position(T x, const BinAxis<T>& a, int& i, unsigned& q) {
  T t = mul_rn(sub_rn(x, a.lo), a.s);
  if (!(t >= T(0) && t <= a.top)) return false;
  T fl = floor(t);
  i = (int)fl;
  T f = sub_rn(t, fl);  // exact
  if (i == a.M - 1) {
    i = a.M - 2;
    f = T(1);
  }
  return fixed_frac(f, i, q);
}

// The 2^d corner weights of the hierarchical split (axis 0 first); corner c
// has offset bit (c >> (D-1-k)) & 1 on axis k.  Each is <= 2^32; they sum
// to exactly 2^32.
template <int D>
__device__ __forceinline__ void corner_weights(const unsigned* q, unsigned long long* w) {
  w[0] = kOne;
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int c = (1 << k) - 1; c >= 0; --c) {
      unsigned long long hi = mulhi_round(w[c], q[k]);
      w[2 * c + 1] = hi;
      w[2 * c] = w[c] - hi;
    }
  }
}

// ---------------------------------------------------------------------------
// Direct path.
// ---------------------------------------------------------------------------
// A pair of adjacent lanes takes one sample: lane parity p adds the 2^(D-1)
// corners at offset p along the last axis.  Corners (.., j) and (.., j + 1)
// are adjacent 8-byte words, in one 32-byte sector unless j = 3 mod 4, so
// each warp instruction's lane pairs coalesce into one sector request where
// one lane per sample would issue two: the scattered-sector rate of the L2
// is what bounds this kernel.
// Block blk of nblk blocks on samples [0, n) of X into counts.
template <typename T, int D>
__device__ __forceinline__ void bin_direct_body(const T* __restrict__ X, int64_t n,
                                                const BinParams<T>& p,
                                                unsigned long long* __restrict__ counts,
                                                unsigned long long* __restrict__ n_out, int blk,
                                                int nblk) {
  constexpr int H = 1 << (D - 1);
  constexpr int U = 8;  // samples whose coordinates are loaded before any is added
  const int par = threadIdx.x & 1;
  unsigned long long outside = 0;
  const int64_t step = ((int64_t)nblk * blockDim.x) >> 1;
  for (int64_t s0 = (blk * (int64_t)blockDim.x + threadIdx.x) >> 1; s0 < n; s0 += U * step) {
    T xs[U][D];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t s = s0 + u * step;
#pragma unroll
      for (int k = 0; k < D; ++k) xs[u][k] = s < n ? X[s * D + k] : T(0);
    }
    // launched as a dependent of the kernel that zeroes the counts: the
    // samples' loads above overlap it; the adds below wait for it
    kde::pdl_wait();
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (s0 + u * step >= n) break;
      int i[D];
      unsigned q[D];
      bool in = true;
#pragma unroll
      for (int k = 0; k < D; ++k) in &= axis_position<T>(xs[u][k], p.ax[k], i[k], q[k]);
      if (!in) {
        outside += par == 0;
        continue;
      }
      int64_t base = par;
#pragma unroll
      for (int k = 0; k < D; ++k) base += (int64_t)i[k] * p.ax[k].stride;
      // weights over the first D - 1 axes, then this lane's half of the last split
      unsigned long long w[H];
      if (D == 1) {
        w[0] = kOne;
      } else {
        corner_weights<D - 1>(q, w);
      }
#pragma unroll
      for (int c = 0; c < H; ++c) {
        const unsigned long long hi = mulhi_round(w[c], q[D - 1]);
        const unsigned long long wc = par ? hi : w[c] - hi;
        if (wc == 0) continue;
        int64_t idx = base;
#pragma unroll
        for (int k = 0; k < D - 1; ++k)
          if ((c >> (D - 2 - k)) & 1) idx += p.ax[k].stride;
        if (KDE_DCHECK(idx >= 0 && idx < p.cells, KDE_DBG_BIN_DIRECT)) atomicAdd(counts + idx, wc);
      }
    }
  }
  if (n_out) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) outside += __shfl_down_sync(0xffffffffu, outside, off);
    if ((threadIdx.x & 31) == 0 && outside) atomicAdd(n_out, outside);
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(256) kde_bin_kernel(const T* __restrict__ X, int64_t n,
                                                      BinParams<T> p,
                                                      unsigned long long* __restrict__ counts,
                                                      unsigned long long* __restrict__ n_out) {
  // X is complete before the zeroing kernel starts; the counts and n_out
  // are touched only after bin_direct_body's pdl_wait
  kde::pdl_trigger();
  bin_direct_body<T, D>(X, n, p, counts, n_out, blockIdx.x, gridDim.x);
}

// Zeroes the counts before kde_bin_kernel (an ordinary launch, so it starts
// after everything before it on the stream; the binning kernel after it is
// a programmatic dependent).
__global__ void __launch_bounds__(256) kde_zero_counts_kernel(unsigned long long* __restrict__ c,
                                                              int64_t cells) {
  kde::pdl_trigger();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (((uintptr_t)c & 15) == 0) {
    ulonglong2* c2 = reinterpret_cast<ulonglong2*>(c);
    for (; i < cells / 2; i += stride) c2[i] = make_ulonglong2(0, 0);
    if (blockIdx.x == 0 && threadIdx.x == 0 && (cells & 1)) c[cells - 1] = 0;
  } else {
    for (; i < cells; i += stride) c[i] = 0;
  }
}

// Many datasets on one grid: blockIdx.y is the dataset, whose samples are
// rows [off[y], off[y + 1]) of X and whose counts start at y * cells.
template <typename T, int D>
__global__ void __launch_bounds__(256) kde_bin_sets_kernel(const T* __restrict__ X,
                                                           const int64_t* __restrict__ off,
                                                           BinParams<T> p,
                                                           unsigned long long* __restrict__ counts) {
  const int64_t a = off[blockIdx.y], b = off[blockIdx.y + 1];
  bin_direct_body<T, D>(X + a * D, b - a, p, counts + (int64_t)blockIdx.y * p.cells, nullptr,
                        blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// Tiled path.
// ---------------------------------------------------------------------------
constexpr int kBinThreads = 512;       // count and scatter kernels
constexpr int kBinU = 4;               // samples per thread per round, loaded before any is used
constexpr int kAccumThreads = 512;
constexpr int kAccumU = 4;             // records per thread per round, loaded before any is used
constexpr int kItemRecords = 8192;     // records per work item
constexpr int kMaxTiles = 16384;       // tiles per grid (shared histograms)
constexpr int kTileCells = 8192;       // cells per tile (shared accumulators)

// Tile shape per d: powers of two, kTileCells cells, the last axis the
// longest so that a tile's rows are long runs of the counts.  ls: strides
// inside a tile (row-major); lsh: log2 of ls.
template <int D>
struct Geo;
template <>
struct Geo<1> {
  __host__ __device__ static constexpr int ext(int k) { return k == 0 ? 8192 : 1; }
  __host__ __device__ static constexpr int lg(int k) { return k == 0 ? 13 : 0; }
  __host__ __device__ static constexpr int ls(int k) { return k == 0 ? 1 : 0; }
  __host__ __device__ static constexpr int lsh(int) { return 0; }
};
template <>
struct Geo<2> {
  __host__ __device__ static constexpr int ext(int k) { return k == 0 ? 64 : k == 1 ? 128 : 1; }
  __host__ __device__ static constexpr int lg(int k) { return k == 0 ? 6 : k == 1 ? 7 : 0; }
  __host__ __device__ static constexpr int ls(int k) { return k == 0 ? 128 : k == 1 ? 1 : 0; }
  __host__ __device__ static constexpr int lsh(int k) { return k == 0 ? 7 : 0; }
};
template <>
struct Geo<3> {
  __host__ __device__ static constexpr int ext(int k) { return k == 2 ? 32 : 16; }
  __host__ __device__ static constexpr int lg(int k) { return k == 2 ? 5 : 4; }
  __host__ __device__ static constexpr int ls(int k) { return k == 0 ? 512 : k == 1 ? 32 : 1; }
  __host__ __device__ static constexpr int lsh(int k) { return k == 0 ? 9 : k == 1 ? 5 : 0; }
};

// The shared accumulators of a tile carry one halo row before and after it
// along every axis (extent ext + 2), so that every corner of every record,
// the tile's own and its neighbours', has a cell: the accumulation needs no
// corner masks and no range tests, and the halo cells are not stored.
// pst: strides of the padded tile (row-major).
template <int D>
__host__ __device__ constexpr int pad_ext(int k) {
  return k < D ? Geo<D>::ext(k) + 2 : 1;
}
template <int D>
__host__ __device__ constexpr int pst(int k) {
  int s = 1;
  for (int j = k + 1; j < D; ++j) s *= pad_ext<D>(j);
  return s;
}
template <int D>
__host__ __device__ constexpr int pad_cells() {
  int c = 1;
  for (int k = 0; k < D; ++k) c *= pad_ext<D>(k);
  return c;
}
// words per accumulator array (a multiple of 4: cleared as uint4)
template <int D>
__host__ __device__ constexpr int pad_alloc() {
  return (pad_cells<D>() + 3) & ~3;
}
// Offset in the padded tile of corner c from the record's base node.
template <int D>
__host__ __device__ constexpr int corner_off(int c) {
  int o = 0;
  for (int k = 0; k < D; ++k) o += ((c >> (D - 1 - k)) & 1) * pst<D>(k);
  return o;
}
static_assert(pad_cells<3>() < (1 << 16) && pad_cells<2>() < (1 << 16) && pad_cells<1>() < (1 << 16),
              "a padded tile-local index fits the record's low 16 bits");

// Position of one coordinate, the same (i, q) as axis_position: the node
// i = floor t and q from f = t - i (exact).  At t = M - 1 this gives
// (M - 1, q = 0), which is axis_position's (M - 2, f = 1) written as its
// fixed_frac writes a fraction of one.  kWithQ = false leaves q = 0 for
// FP32 inputs, where i does not depend on it (f < 1 - 2^-25, so f 2^32
// never rounds up to 2^32); FP64 fractions can round up, which moves i, so
// they are always computed.
template <typename T, bool kWithQ = true>
__device__ __forceinline__ bool axis_node(T x, const BinAxis<T>& a, int& i, unsigned& q) {
  const T t = mul_rn(sub_rn(x, a.lo), a.s);
  const bool in = t >= T(0) && t <= a.top;
  const T fl = floor(t);
  i = (int)fl;
  q = 0;
  if (kWithQ || sizeof(T) == 8) fixed_frac(sub_rn(t, fl), i, q);
  return in;
}

// One sample located on the grid: base node i and fractions q per axis, its
// tile t0, and the axes along which it also feeds the next tile: those
// where the base is on the tile's last row and not the grid's last node.
// (Along such an axis the corners after the base lie in the next tile; if
// q = 0 there they have weight zero and the extra record adds zeros.  The
// count and scatter kernels apply the same rule, which is all the bucket
// offsets need.)  kWithQ = false: q is not computed (the count kernel).
template <int D>
struct Located {
  int i[D];
  unsigned q[D];
  int t0;
  int spill;
};

template <typename T, int D, bool kWithQ = true>
__device__ __forceinline__ bool locate(const T* x, const BinParams<T>& p, Located<D>& g) {
  bool in = true;
#pragma unroll
  for (int k = 0; k < D; ++k) in &= axis_node<T, kWithQ>(x[k], p.ax[k], g.i[k], g.q[k]);
  g.t0 = 0;
  g.spill = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    g.t0 += (g.i[k] >> Geo<D>::lg(k)) * p.ax[k].tstride;
    const bool last = (g.i[k] & (Geo<D>::ext(k) - 1)) == Geo<D>::ext(k) - 1;
    g.spill |= (last && g.i[k] < p.ax[k].M - 1) << k;
  }
  return in;
}

// Tile of target subset S of a sample's spill axes (the tile after t0 along
// every axis in S).
template <typename T, int D>
__device__ __forceinline__ int spill_tile(const Located<D>& g, int S, const BinParams<T>& p) {
  int t = g.t0;
#pragma unroll
  for (int k = 0; k < D; ++k)
    if ((S >> k) & 1) t += p.ax[k].tstride;
  return t;
}

// Record of a sample for target subset S of its spill axes: {q_0, q_1, q_2,
// j0} with j0 the index in the padded tile of the base node relative to
// that tile (the base is one row before the tile on the axes in S, in the
// halo).  Corners that fall in a halo are added there and not stored: on
// the axes in S the lower corner belongs to the tile before (its record
// adds it there), and an upper corner past the tile's last row belongs to
// the tile after, where the sample's spill record adds it, or lies past the
// grid's last node with weight zero (q = 0).
template <int D>
__device__ __forceinline__ uint4 make_record(const Located<D>& g, int S) {
  int j0 = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int l = g.i[k] & (Geo<D>::ext(k) - 1);
    const int b = ((S >> k) & 1) ? l - Geo<D>::ext(k) : l;
    j0 += (b + 1) * pst<D>(k);
  }
  return make_uint4(g.q[0], D > 1 ? g.q[D > 1 ? 1 : 0] : 0u, D > 2 ? g.q[D > 2 ? 2 : 0] : 0u,
                    (unsigned)j0);
}

// Samples of block b: the contiguous chunk [b chunk, min(n, (b + 1) chunk)),
// visited in the same order by the count and scatter kernels, each thread
// loading kBinU samples before it uses any.
template <typename T, int D, typename F>
__device__ __forceinline__ void for_block_samples(const T* __restrict__ X, int64_t n, int64_t chunk,
                                                  F&& f) {
  const int64_t beg = (int64_t)blockIdx.x * chunk;
  const int64_t end = beg + chunk < n ? beg + chunk : n;
  for (int64_t s0 = beg + threadIdx.x; s0 < end; s0 += (int64_t)kBinU * blockDim.x) {
    T x[kBinU][D];
#pragma unroll
    for (int u = 0; u < kBinU; ++u) {
      const int64_t s = s0 + (int64_t)u * blockDim.x;
#pragma unroll
      for (int k = 0; k < D; ++k) x[u][k] = s < end ? X[s * D + k] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kBinU; ++u)
      if (s0 + (int64_t)u * blockDim.x < end) f(x[u]);
  }
}

// Records per tile and samples outside the grid.  Each block adds its
// shared histogram into tile_count and keeps the offset of its range inside
// every tile's bucket (the atomicAdd's old value); the scatter kernel's
// block b writes its records of tile t into that range.  The tile counts
// start at zero (cleared before this launch).
template <typename T, int D>
__global__ void __launch_bounds__(kBinThreads, 2)
kde_bin_count_kernel(const T* __restrict__ X, int64_t n, int64_t chunk, BinParams<T> p,
                     int ntiles, unsigned* __restrict__ tile_count,
                     unsigned* __restrict__ block_off, unsigned long long* __restrict__ n_out) {
  extern __shared__ unsigned hist[];
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) hist[t] = 0;
  __syncthreads();
  // the scatter kernel may start now; it waits for this grid before it
  // reads anything written here
  kde::pdl_trigger();
  unsigned long long outside = 0;
  for_block_samples<T, D>(X, n, chunk, [&](const T* x) {
    Located<D> g;
    if (!locate<T, D, false>(x, p, g)) {
      ++outside;
      return;
    }
    atomicAdd(&hist[g.t0], 1u);
    // every nonempty subset of the spill axes (usually one axis)
    for (int S = g.spill; S; S = (S - 1) & g.spill) atomicAdd(&hist[spill_tile<T, D>(g, S, p)], 1u);
  });
  __syncthreads();
  unsigned* mine = block_off + (size_t)blockIdx.x * ntiles;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
    const unsigned v = hist[t];
    mine[t] = v ? atomicAdd(&tile_count[t], v) : 0u;
  }
  if (n_out) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) outside += __shfl_down_sync(0xffffffffu, outside, off);
    if ((threadIdx.x & 31) == 0 && outside) atomicAdd(n_out, outside);
  }
}

struct TiledMeta {
  unsigned nitems;
  unsigned cursor;   // next work item of the accumulation (zero before it starts)
};

// Exclusive prefix sum of one value per thread over the block (a multiple
// of 32 threads, at most 1024); *total gets the sum.
__device__ __forceinline__ unsigned block_scan(unsigned v, unsigned* warp_tot, unsigned* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    const unsigned t = lane < nw ? warp_tot[lane] : 0u;
    unsigned s = t;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, s, off);
      if (lane >= off) s += y;
    }
    if (lane < nw) warp_tot[lane] = s - t;
    if (lane == 31) *total = s;
  }
  __syncthreads();
  const unsigned r = warp_tot[w] + x - v;
  __syncthreads();  // warp_tot may be reused by the next scan
  return r;
}

__device__ __forceinline__ unsigned items_of(unsigned c) {
  return c == 0 ? 1u : (c + kItemRecords - 1) / kItemRecords;
}

// Global cell index of tile-local cell j of tile t (or -1 outside the grid).
template <typename T, int D>
__device__ __forceinline__ int64_t tile_cell(const BinParams<T>& p, int t, int j) {
  int64_t idx = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int tk = (t / p.ax[k].tstride) % p.ax[k].ntiles;
    const int lk = (j >> Geo<D>::lsh(k)) & (Geo<D>::ext(k) - 1);
    const int c = (tk << Geo<D>::lg(k)) + lk;
    if (c >= p.ax[k].M) return -1;
    idx += (int64_t)c * p.ax[k].stride;
  }
  return idx;
}

// Bucket starts (every block, from the tile counts), work items (block 0:
// (tile, first record, end record, split) with at most kItemRecords records
// each, one item for an empty tile so that its cells are stored as zeros),
// split tiles' cells zeroed (tile t by block t mod gridDim.x: their items
// add), then block b takes the same samples as in the count kernel and
// writes its records of tile t at bucket start + its range offset + a
// running count kept in shared memory.
template <typename T, int D>
__global__ void __launch_bounds__(kBinThreads, 2)
kde_bin_scatter_kernel(const T* __restrict__ X, int64_t n, int64_t chunk, BinParams<T> p,
                       int ntiles, const unsigned* __restrict__ tile_count,
                       const unsigned* __restrict__ block_off, uint4* __restrict__ items,
                       TiledMeta* __restrict__ meta, uint4* __restrict__ recs, unsigned rec_cap,
                       unsigned long long* __restrict__ counts, int add) {
  extern __shared__ unsigned next[];   // [ntiles]: next slot of this block per tile
  __shared__ unsigned warp_tot[32];
  __shared__ unsigned totals[2];
  kde::pdl_trigger();
  kde::pdl_wait();   // tile counts and block offsets of the count kernel
  const int per = (ntiles + blockDim.x - 1) / blockDim.x;
  const int t0 = threadIdx.x * per, t1 = min(ntiles, t0 + per);
  unsigned rec = 0, nit = 0;
  for (int t = t0; t < t1; ++t) {
    const unsigned c = __ldcg(tile_count + t);
    rec += c;
    nit += items_of(c);
  }
  unsigned r0 = block_scan(rec, warp_tot, &totals[0]);
  unsigned i0 = block_scan(nit, warp_tot, &totals[1]);
  const unsigned* mine = block_off + (size_t)blockIdx.x * ntiles;
  for (int t = t0; t < t1; ++t) {
    const unsigned c = __ldcg(tile_count + t);
    next[t] = r0 + __ldcg(mine + t);
    const unsigned it = items_of(c);
    if (blockIdx.x == 0) {
      for (unsigned j = 0; j < it; ++j) {
        const unsigned b = r0 + j * kItemRecords, e = min(r0 + c, b + kItemRecords);
        items[i0 + j] = make_uint4((unsigned)t, b, e, it > 1 ? 1u : 0u);
      }
    }
    r0 += c;
    i0 += it;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) meta->nitems = totals[1];
  // (adding into existing counts: nothing to zero)
  for (int t = blockIdx.x; t < ntiles && !add; t += gridDim.x) {
    if (__ldcg(tile_count + t) <= (unsigned)kItemRecords) continue;
    for (int j = threadIdx.x; j < kTileCells; j += blockDim.x) {
      const int64_t idx = tile_cell<T, D>(p, t, j);
      if (idx >= 0) counts[idx] = 0;
    }
  }
  __syncthreads();
  for_block_samples<T, D>(X, n, chunk, [&](const T* x) {
    Located<D> g;
    if (!locate<T, D>(x, p, g)) return;
    {
      const uint4 r = make_record<D>(g, 0);   // filled before its slot is taken
      const unsigned slot = atomicAdd(&next[g.t0], 1u);
      if (slot < rec_cap) recs[slot] = r;
    }
    for (int S = g.spill; S; S = (S - 1) & g.spill) {
      const uint4 r = make_record<D>(g, S);
      const unsigned slot = atomicAdd(&next[spill_tile<T, D>(g, S, p)], 1u);
      if (slot < rec_cap) recs[slot] = r;
    }
  });
}

// Work items taken in turn from meta->cursor: the item's records
// accumulated in shared memory, then every cell of its tile stored (added,
// for split tiles and when adding into existing counts; an empty tile's
// cells are stored as zeros directly, or skipped when adding).  A
// weight w <= 2^32 is added as its low 16 bits and its high part
// w >> 16 <= 2^16 into two 32-bit sums per cell; an item holds at most
// kItemRecords = 2^13 records and a record adds to a cell at most once, so
// neither sum exceeds 2^29 and no carry is ever lost: the cell's total is
// hi 2^16 + lo exactly.  The adds need no return value (fire-and-forget).
// Every corner of a record is added, into the padded tile (halo corners
// are not stored); a corrupt record cannot reach outside the shared arrays.
static_assert(kItemRecords <= (1 << 13), "16-bit split sums must stay below 2^32");

template <int D>
__device__ __forceinline__ void accumulate_record(unsigned* lo, unsigned* hi, const uint4& rec) {
  const unsigned q[3] = {rec.x, rec.y, rec.z};
  // clamped so that every corner stays inside the padded tile, whatever
  // the record holds
  constexpr int kMaxBase = pad_cells<D>() - 1 - corner_off<D>((1 << D) - 1);
  const int j0 = min((int)(rec.w & 0xFFFFu), kMaxBase);
  unsigned long long w[1 << D];
  corner_weights<D>(q, w);
#pragma unroll
  for (int c = 0; c < (1 << D); ++c) {
    atomicAdd(&lo[j0 + corner_off<D>(c)], (unsigned)w[c] & 0xFFFFu);
    atomicAdd(&hi[j0 + corner_off<D>(c)], (unsigned)(w[c] >> 16));
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(kAccumThreads, 2)
kde_bin_accum_kernel(const uint4* __restrict__ recs, const uint4* __restrict__ items,
                     TiledMeta* __restrict__ meta, BinParams<T> p,
                     unsigned long long* __restrict__ counts, int add) {
  extern __shared__ __align__(16) unsigned acc_sm[];
  unsigned* lo = acc_sm;
  unsigned* hi = acc_sm + pad_alloc<D>();
  __shared__ unsigned cur_item;
  kde::pdl_trigger();
  kde::pdl_wait();   // items and records of the scatter kernel
  const unsigned nitems = __ldcg(&meta->nitems);
  for (;;) {
    if (threadIdx.x == 0) cur_item = atomicAdd(&meta->cursor, 1u);
    __syncthreads();
    const unsigned it = cur_item;
    __syncthreads();   // cur_item is rewritten at the next turn
    if (it >= nitems) break;
    const uint4 item = __ldcg(items + it);
    // the tile's origin and extent inside the grid
    int64_t origin = 0;
    int ext[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int tk = ((int)item.x / p.ax[k].tstride) % p.ax[k].ntiles;
      const int o = tk << Geo<D>::lg(k);
      origin += (int64_t)o * p.ax[k].stride;
      ext[k] = min(Geo<D>::ext(k), p.ax[k].M - o);
    }
    const bool empty = item.y >= item.z;
    if (empty && add) continue;   // nothing to add
    if (!empty) {
      for (int j = threadIdx.x; j < pad_alloc<D>() / 2; j += blockDim.x)
        reinterpret_cast<uint4*>(lo)[j] = make_uint4(0, 0, 0, 0);   // lo and hi
      __syncthreads();
      for (unsigned r0 = item.y + threadIdx.x; r0 < item.z; r0 += kAccumU * blockDim.x) {
        uint4 rec[kAccumU];
#pragma unroll
        for (int u = 0; u < kAccumU; ++u) {
          const unsigned r = r0 + u * blockDim.x;
          rec[u] = r < item.z ? __ldcg(recs + r) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < kAccumU; ++u)
          if (r0 + u * blockDim.x < item.z) accumulate_record<D>(lo, hi, rec[u]);
      }
      __syncthreads();
    }
    for (int j = threadIdx.x; j < kTileCells; j += blockDim.x) {
      int64_t idx = origin;
      int jp = 0;
      bool in = true;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int l = (j >> Geo<D>::lsh(k)) & (Geo<D>::ext(k) - 1);
        in &= l < ext[k];
        idx += (int64_t)l * p.ax[k].stride;
        jp += (l + 1) * pst<D>(k);
      }
      if (!in || !KDE_DCHECK(idx >= 0 && idx < p.cells, KDE_DBG_BIN_ACCUM)) continue;
      const unsigned long long v = empty ? 0ull : ((unsigned long long)hi[jp] << 16) + lo[jp];
      if (item.w || add) {
        if (v) atomicAdd(counts + idx, v);
      } else {
        counts[idx] = v;
      }
    }
    __syncthreads();   // the shared sums are cleared at the next turn
  }
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
  }
  return sms;
}

// Tile counts (tile shapes: Geo<d>) and the workspace layout of the tiled
// path.  Grid of the count and scatter kernels (the same in both, and part
// of the workspace size, so it does not depend on the device): at most 304
// blocks (two per SM of a GB300), at least 2048 samples each.
constexpr int kBinBlocks = 304;
constexpr int64_t kMinBlockSamples = 2048;

struct TiledLayout {
  int tile[KDE_MAX_D];
  int ntiles[KDE_MAX_D];
  int ntiles_total;
  int blocks;                     // grid of the count and scatter kernels
  int64_t chunk;                  // samples per block (a multiple of kBinThreads)
  int64_t max_records, max_items;
  size_t off_count, off_meta, off_items, off_base, off_recs, total;
};

bool tiled_layout(int64_t n, int d, const int64_t* M, TiledLayout* t) {
  t->ntiles_total = 1;
  for (int k = 0; k < d; ++k) {
    t->tile[k] = d == 1 ? Geo<1>::ext(k) : d == 2 ? Geo<2>::ext(k) : Geo<3>::ext(k);
    t->ntiles[k] = (int)((M[k] + t->tile[k] - 1) / t->tile[k]);
    if ((int64_t)t->ntiles_total * t->ntiles[k] > kMaxTiles) return false;
    t->ntiles_total *= t->ntiles[k];
  }
  // every sample feeds at most 2^d tiles
  t->max_records = (n > 0 ? n : 1) << d;
  if (t->max_records >= (int64_t(1) << 32)) return false;
  t->max_items = t->ntiles_total + t->max_records / kItemRecords + 1;
  const int64_t want = (n + kMinBlockSamples - 1) / kMinBlockSamples;
  t->blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, kBinBlocks));
  const int64_t per = (std::max<int64_t>(n, 1) + t->blocks - 1) / t->blocks;
  t->chunk = (per + kBinThreads - 1) / kBinThreads * kBinThreads;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  t->off_count = 0;
  t->off_meta = up((size_t)t->ntiles_total * 4);
  t->off_items = t->off_meta + 256;
  t->off_base = t->off_items + up((size_t)t->max_items * 16);
  t->off_recs = t->off_base + up((size_t)t->blocks * t->ntiles_total * 4);
  t->total = t->off_recs + up((size_t)t->max_records * 16);
  return true;
}

template <typename T>
BinParams<T> make_params(int d, const double* lo, const double* hi, const int64_t* M,
                         const TiledLayout* t) {
  BinParams<T> p{};
  int64_t stride = 1;
  int ts = 1, ls = 1;
  p.cells = 1;
  for (int k = 0; k < d; ++k) p.cells *= M[k];
  for (int k = d - 1; k >= 0; --k) {
    double s = (double)(M[k] - 1) / (hi[k] - lo[k]);
    p.ax[k].lo = (T)lo[k];
    p.ax[k].s = (T)s;
    p.ax[k].top = (T)(M[k] - 1);
    p.ax[k].stride = stride;
    p.ax[k].M = (int)M[k];
    stride *= M[k];
    if (t) {
      p.ax[k].tile = t->tile[k];
      int lg = 0;
      while ((1 << lg) < t->tile[k]) ++lg;
      p.ax[k].tile_log2 = lg;
      p.ax[k].ntiles = t->ntiles[k];
      p.ax[k].tstride = ts;
      p.ax[k].lstride = ls;
      ts *= t->ntiles[k];
      ls *= t->tile[k];
    }
  }
  return p;
}

template <typename T>
kde_status launch_direct(const T* X, int64_t n, int d, const double* lo, const double* hi,
                         const int64_t* M, unsigned long long* counts, int64_t cells,
                         unsigned long long* n_out, cudaStream_t stream, bool zero) {
  cudaError_t e;
  if (zero) {
    const int64_t want = (cells / 2 + 255) / 256;
    const int zb = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * 8));
    kde::LaunchScope ls("kde_zero_counts_kernel", stream);
    kde_zero_counts_kernel<<<zb, 256, 0, stream>>>(counts, cells);
    if ((e = cudaGetLastError()) != cudaSuccess) return kde::cuda_fail(e, "kde_zero_counts_kernel");
  }
  if (n == 0) return KDE_OK;
  BinParams<T> p = make_params<T>(d, lo, hi, M, nullptr);
  int64_t want = (2 * n + 255) / 256;  // two lanes per sample
  int64_t cap = (int64_t)num_sms() * 16;
  int blocks = (int)(want < cap ? want : cap);
  kde::LaunchScope ls("kde_bin_kernel", stream);
  switch (d) {
    case 1: e = kde::launch_pdl(kde_bin_kernel<T, 1>, blocks, 256, 0, stream, X, n, p, counts, n_out); break;
    case 2: e = kde::launch_pdl(kde_bin_kernel<T, 2>, blocks, 256, 0, stream, X, n, p, counts, n_out); break;
    default: e = kde::launch_pdl(kde_bin_kernel<T, 3>, blocks, 256, 0, stream, X, n, p, counts, n_out); break;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : kde::cuda_fail(e, "kde_bin_kernel launch");
}

// kde_bin_sets_kernel for nsets datasets of at most n_max samples each
// (offsets on the device): counts zeroed, then about 8 blocks per SM in all.
template <typename T>
kde_status launch_sets(const T* X, const int64_t* off_dev, int nsets, int64_t n_max, int d,
                       const double* lo, const double* hi, const int64_t* M,
                       unsigned long long* counts, cudaStream_t stream) {
  BinParams<T> p = make_params<T>(d, lo, hi, M, nullptr);
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)nsets * p.cells * sizeof(int64_t), stream);
  if (e != cudaSuccess) return kde::cuda_fail(e, "cudaMemsetAsync(counts)");
  if (n_max == 0 || nsets == 0) return KDE_OK;
  const int64_t want = (2 * n_max + 255) / 256;
  const int64_t cap = std::max<int64_t>(1, (int64_t)num_sms() * 8 / nsets);
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min(want, cap)), (unsigned)nsets);
  kde::LaunchScope ls("kde_bin_sets_kernel", stream);
  switch (d) {
    case 1: kde_bin_sets_kernel<T, 1><<<grid, 256, 0, stream>>>(X, off_dev, p, counts); break;
    case 2: kde_bin_sets_kernel<T, 2><<<grid, 256, 0, stream>>>(X, off_dev, p, counts); break;
    default: kde_bin_sets_kernel<T, 3><<<grid, 256, 0, stream>>>(X, off_dev, p, counts); break;
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : kde::cuda_fail(e, "kde_bin_sets_kernel launch");
}

template <typename F>
cudaError_t allow_smem(F* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Three launches: the count kernel (after the tile counts and the item
// cursor are cleared), then the scatter and accumulation kernels as
// programmatic dependents of the kernel before each.
template <typename T, int D>
kde_status launch_tiled_d(const T* X, int64_t n, const double* lo, const double* hi,
                          const int64_t* M, unsigned long long* counts,
                          unsigned long long* n_out, const TiledLayout& t, char* ws,
                          cudaStream_t stream, int add) {
  BinParams<T> p = make_params<T>(D, lo, hi, M, &t);
  unsigned* tile_count = (unsigned*)(ws + t.off_count);
  TiledMeta* meta = (TiledMeta*)(ws + t.off_meta);
  uint4* items = (uint4*)(ws + t.off_items);
  unsigned* block_off = (unsigned*)(ws + t.off_base);
  uint4* recs = (uint4*)(ws + t.off_recs);
  const int nt = t.ntiles_total;
  const int sms = num_sms();
  cudaError_t e = cudaMemsetAsync(ws, 0, t.off_meta + sizeof(TiledMeta), stream);
  if (e != cudaSuccess) return kde::cuda_fail(e, "cudaMemsetAsync(tile counts)");
  const size_t smem_t = (size_t)nt * 4;
  {
    auto* fn = kde_bin_count_kernel<T, D>;
    if ((e = allow_smem(fn, smem_t)) != cudaSuccess) return kde::cuda_fail(e, "smem attr");
    kde::LaunchScope ls("kde_bin_count_kernel", stream);
    fn<<<t.blocks, kBinThreads, smem_t, stream>>>(X, n, t.chunk, p, nt, tile_count, block_off,
                                                  n_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return kde::cuda_fail(e, "kde_bin_count_kernel");
  }
  {
    auto* fn = kde_bin_scatter_kernel<T, D>;
    if ((e = allow_smem(fn, smem_t)) != cudaSuccess) return kde::cuda_fail(e, "smem attr");
    kde::LaunchScope ls("kde_bin_scatter_kernel", stream);
    e = kde::launch_pdl(fn, t.blocks, kBinThreads, smem_t, stream, X, n, t.chunk, p, nt,
                        (const unsigned*)tile_count, (const unsigned*)block_off, items, meta, recs,
                        (unsigned)t.max_records, counts, add);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return kde::cuda_fail(e, "kde_bin_scatter_kernel");
  }
  {
    auto* fn = kde_bin_accum_kernel<T, D>;
    const size_t smem = 2 * (size_t)pad_alloc<D>() * sizeof(unsigned);
    if ((e = allow_smem(fn, smem)) != cudaSuccess) return kde::cuda_fail(e, "smem attr");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kAccumThreads, smem);
    if (e != cudaSuccess) return kde::cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    const int grid_a = (int)std::min<int64_t>(t.max_items, (int64_t)std::max(1, per_sm) * sms);
    kde::LaunchScope ls("kde_bin_accum_kernel", stream);
    e = kde::launch_pdl(fn, grid_a, kAccumThreads, smem, stream, (const uint4*)recs,
                        (const uint4*)items, meta, p, counts, add);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return kde::cuda_fail(e, "kde_bin_accum_kernel");
  }
  return KDE_OK;
}

template <typename T>
kde_status launch_tiled(const T* X, int64_t n, int d, const double* lo, const double* hi,
                        const int64_t* M, unsigned long long* counts, unsigned long long* n_out,
                        const TiledLayout& t, char* ws, cudaStream_t stream, int add) {
  switch (d) {
    case 1: return launch_tiled_d<T, 1>(X, n, lo, hi, M, counts, n_out, t, ws, stream, add);
    case 2: return launch_tiled_d<T, 2>(X, n, lo, hi, M, counts, n_out, t, ws, stream, add);
    default: return launch_tiled_d<T, 3>(X, n, lo, hi, M, counts, n_out, t, ws, stream, add);
  }
}

kde_status check_bin_args(int d, int x_dtype, int64_t n, const void* X, const double* lo,
                          const double* hi, const int64_t* M, int64_t* cells_out) {
  using kde::fail;
  if (d < 1 || d > KDE_MAX_D) return fail(KDE_ERR_UNSUPPORTED, "d must be 1, 2 or 3");
  if (!lo || !hi || !M) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (x_dtype != KDE_F32 && x_dtype != KDE_F64) return fail(KDE_ERR_INVALID_ARG, "bad x_dtype");
  if (n < 0 || n >= (int64_t(1) << 31)) return fail(KDE_ERR_INVALID_ARG, "need 0 <= n < 2^31");
  if (n > 0 && !X) return fail(KDE_ERR_INVALID_ARG, "X is NULL");
  int64_t cells = 1;
  for (int k = 0; k < d; ++k) {
    if (M[k] < 2) return fail(KDE_ERR_INVALID_ARG, "every M_k must be >= 2");
    if (M[k] > (int64_t(1) << 24)) return fail(KDE_ERR_INVALID_ARG, "M_k too large");
    if (!std::isfinite(lo[k]) || !std::isfinite(hi[k]) || !(lo[k] < hi[k]))
      return fail(KDE_ERR_INVALID_ARG, "need finite lo[k] < hi[k]");
    cells *= M[k];
    if (cells >= (int64_t(1) << 40)) return fail(KDE_ERR_INVALID_ARG, "grid too large");
  }
  *cells_out = cells;
  return KDE_OK;
}

}  // namespace

namespace kde {
kde_status bin_sets_f32(const float* X, const int64_t* off_dev, int nsets, int64_t n_max, int d,
                        const double* lo, const double* hi, const int64_t* M, int64_t* counts,
                        cudaStream_t st) {
  return launch_sets<float>(X, off_dev, nsets, n_max, d, lo, hi, M,
                            reinterpret_cast<unsigned long long*>(counts), st);
}
}  // namespace kde

extern "C" kde_status kde_bin_workspace_bytes(int64_t n, int d, const int64_t* M, size_t* bytes) {
  if (!bytes || !M || d < 1 || d > KDE_MAX_D || n < 0)
    return kde::fail(KDE_ERR_INVALID_ARG, "bad argument");
  TiledLayout t{};
  if (!tiled_layout(n, d, M, &t)) {
    *bytes = 0;
    return kde::fail(KDE_ERR_UNSUPPORTED, "grid too large for the tiled binning path");
  }
  *bytes = t.total;
  return KDE_OK;
}

namespace {
// kde_bin (add = false: counts and *n_outside overwritten) and
// kde_bin_accumulate (add = true: added to).
kde_status bin_impl(const void* X, int x_dtype, int64_t n, int d, const double* lo, const double* hi,
                    const int64_t* M, int64_t* counts, int64_t* n_outside, void* workspace,
                    size_t workspace_bytes, kde_stream_t stream, bool add) {
  using kde::fail;
  int64_t cells = 0;
  kde_status st = check_bin_args(d, x_dtype, n, X, lo, hi, M, &cells);
  if (st != KDE_OK) return st;
  if (!counts) return fail(KDE_ERR_INVALID_ARG, "counts is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  auto* c = reinterpret_cast<unsigned long long*>(counts);
  auto* no = reinterpret_cast<unsigned long long*>(n_outside);
  if (n_outside && !add) {
    cudaError_t e = cudaMemsetAsync(n_outside, 0, sizeof(int64_t), s);
    if (e != cudaSuccess) return kde::cuda_fail(e, "cudaMemsetAsync(n_outside)");
  }
  if (!workspace) {
    if (x_dtype == KDE_F32)
      return launch_direct<float>((const float*)X, n, d, lo, hi, M, c, cells, no, s, !add);
    return launch_direct<double>((const double*)X, n, d, lo, hi, M, c, cells, no, s, !add);
  }
  TiledLayout t{};
  if (!tiled_layout(n, d, M, &t))
    return fail(KDE_ERR_UNSUPPORTED, "grid too large for the tiled binning path");
  if (cells >= (int64_t(1) << 32)) return fail(KDE_ERR_UNSUPPORTED, "tiled binning needs prod(M) < 2^32");
  if (workspace_bytes < t.total) return fail(KDE_ERR_WORKSPACE, "binning workspace too small");
  if (((uintptr_t)workspace & 255) != 0) return fail(KDE_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  if (n == 0 && add) return KDE_OK;
  if (x_dtype == KDE_F32)
    return launch_tiled<float>((const float*)X, n, d, lo, hi, M, c, no, t, (char*)workspace, s, add);
  return launch_tiled<double>((const double*)X, n, d, lo, hi, M, c, no, t, (char*)workspace, s, add);
}
}  // namespace

extern "C" kde_status kde_bin(const void* X, int x_dtype, int64_t n, int d, const double* lo,
                              const double* hi, const int64_t* M, int64_t* counts,
                              int64_t* n_outside, void* workspace, size_t workspace_bytes,
                              kde_stream_t stream) {
  return bin_impl(X, x_dtype, n, d, lo, hi, M, counts, n_outside, workspace, workspace_bytes,
                  stream, false);
}

extern "C" kde_status kde_bin_accumulate(const void* X, int x_dtype, int64_t n, int d,
                                         const double* lo, const double* hi, const int64_t* M,
                                         int64_t* counts, int64_t* n_outside, void* workspace,
                                         size_t workspace_bytes, kde_stream_t stream) {
  return bin_impl(X, x_dtype, n, d, lo, hi, M, counts, n_outside, workspace, workspace_bytes,
                  stream, true);
}

KDE_DEBUG_READER(bin)
