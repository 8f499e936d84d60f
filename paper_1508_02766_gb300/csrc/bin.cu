// Linear binning (Sec. 2, first step): each sample inside the grid spreads a
// unit mass over its 2^d neighbouring nodes with integer weights in units of
// 2^-32 that sum to exactly 2^32 (so the counts sum to n, Sec. 3 footnote).
// Integer addition is associative, so the counts are bit-identical whatever
// order the additions happen in.
//
// Two implementations of the same arithmetic:
//   direct  one pass, 64-bit integer atomics straight into the counts (no
//           scratch; bound by the L2 atomic rate, ~2^d atomics per sample);
//   tiled   a counting sort of the samples by the grid tile of their base
//           node, then one block per tile accumulating in shared memory with
//           shared 64-bit atomics and writing every cell of its tile once
//           with a plain store (no memset, no global atomics on counts):
//             hist     per-block histogram of keys (tile, face mask)
//             scan     exclusive prefix over blocks per key, then over keys
//             scatter  records {tile-local base, Q_0..Q_{d-1}} into key order
//             gather   per work item of a tile: own records plus
//                      neighbours' face records (tiles with more records
//                      than one item holds are zeroed first and their
//                      items add with 64-bit atomics)
//           A sample whose base node is the last row of its tile along axis k
//           also feeds the next tile (face-mask bit k); the owner of a cell
//           reads those records from the neighbour's face buckets.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "kde_internal.h"

namespace {

constexpr unsigned long long kOne = 1ull << 32;
constexpr int kHistThreads = 512;
constexpr int kGatherThreads = 256;
constexpr int kMaxKeys = 32768;
constexpr int kMaxBlocks = 1024;

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
};

template <typename T>
struct BinParams {
  BinAxis<T> ax[KDE_MAX_D];
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
template <typename T, int D>
__global__ void __launch_bounds__(256) kde_bin_kernel(const T* __restrict__ X, int64_t n,
                                                      BinParams<T> p,
                                                      unsigned long long* __restrict__ counts,
                                                      unsigned long long* __restrict__ n_out) {
  constexpr int H = 1 << (D - 1);
  constexpr int U = 8;  // samples whose coordinates are loaded before any is added
  const int par = threadIdx.x & 1;
  unsigned long long outside = 0;
  const int64_t step = ((int64_t)gridDim.x * blockDim.x) >> 1;
  for (int64_t s0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 1; s0 < n; s0 += U * step) {
    T xs[U][D];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t s = s0 + u * step;
#pragma unroll
      for (int k = 0; k < D; ++k) xs[u][k] = s < n ? X[s * D + k] : T(0);
    }
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
        atomicAdd(counts + idx, wc);
      }
    }
  }
  if (n_out) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) outside += __shfl_down_sync(0xffffffffu, outside, off);
    if ((threadIdx.x & 31) == 0 && outside) atomicAdd(n_out, outside);
  }
}

// ---------------------------------------------------------------------------
// Tiled path.
// ---------------------------------------------------------------------------
// Bits per axis of a record's tile-local base node.
template <int D> struct LocalBits { static constexpr int value = D == 1 ? 32 : (D == 2 ? 16 : 10); };

// A sample's key (base tile, face mask) and record {tile-local base node,
// q_0 .. q_{d-1}}.  Face-mask bit (D-1-k) is set when the base node is the
// last node of its tile along axis k (and not the grid's last node): the
// sample then also feeds the next tile along k.
template <typename T, int D>
__device__ __forceinline__ bool sample_key(const T* x, const BinParams<T>& p, int& key, uint4& rec) {
  int i[D];
  unsigned q[3] = {0, 0, 0};
  bool in = true;
#pragma unroll
  for (int k = 0; k < D; ++k) in &= axis_position<T>(x[k], p.ax[k], i[k], q[k]);
  if (!in) return false;
  int tile = 0, mask = 0;
  unsigned local = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const int tk = i[k] >> p.ax[k].tile_log2;
    const int li = i[k] & (p.ax[k].tile - 1);
    tile += tk * p.ax[k].tstride;
    local |= (unsigned)li << (LocalBits<D>::value * k);
    if (li == p.ax[k].tile - 1 && i[k] + 1 < p.ax[k].M) mask |= 1 << (D - 1 - k);
  }
  key = (tile << D) | mask;
  rec = make_uint4(local, q[0], q[1], q[2]);
  return true;
}

constexpr int kUnroll = 4;

// Coordinates of samples base + u blockDim (u < kUnroll) that lie below s1.
template <typename T, int D>
__device__ __forceinline__ void load_samples(const T* __restrict__ X, int64_t base, int64_t s1,
                                             T (&x)[kUnroll][D]) {
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const int64_t s = base + u * (int64_t)blockDim.x;
#pragma unroll
    for (int k = 0; k < D; ++k) x[u][k] = s < s1 ? X[s * D + k] : T(0);
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(kHistThreads)
kde_bin_hist_kernel(const T* __restrict__ X, int64_t n, int64_t chunk, int nkeys, BinParams<T> p,
                    unsigned* __restrict__ mat, unsigned long long* __restrict__ n_out) {
  extern __shared__ unsigned hist[];
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  const int64_t s0 = (int64_t)blockIdx.x * chunk;
  const int64_t s1 = min(n, s0 + chunk);
  unsigned long long outside = 0;
  // the next iteration's samples are loaded before this one's are keyed
  T xc[kUnroll][D], xn[kUnroll][D];
  load_samples<T, D>(X, s0 + threadIdx.x, s1, xc);
  for (int64_t base = s0 + threadIdx.x; base < s1; base += kUnroll * (int64_t)blockDim.x) {
    load_samples<T, D>(X, base + kUnroll * (int64_t)blockDim.x, s1, xn);
    int key[kUnroll];
    bool in[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t s = base + u * (int64_t)blockDim.x;
      uint4 rec;
      in[u] = s < s1 && sample_key<T, D>(xc[u], p, key[u], rec);
      if (s < s1 && !in[u]) ++outside;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
      if (in[u]) atomicAdd(&hist[key[u]], 1u);
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < D; ++k) xc[u][k] = xn[u][k];
  }
  __syncthreads();
  unsigned* row = mat + (int64_t)blockIdx.x * nkeys;
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x) row[k] = hist[k];
  if (n_out) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) outside += __shfl_down_sync(0xffffffffu, outside, off);
    if ((threadIdx.x & 31) == 0 && outside) atomicAdd(n_out, outside);
  }
}

// Exclusive prefix over blocks for each key (in place), totals per key.
// A block takes 32 keys: the [nblocks x 32] slab is staged in shared memory
// with coalesced rows, each key's column is split into 8 segments scanned by
// 8 threads, then the segment offsets are applied and the slab written back.
constexpr int kScanKeys = 32, kScanSegs = 8;
__global__ void __launch_bounds__(kScanKeys * kScanSegs)
kde_bin_scan_blocks_kernel(unsigned* __restrict__ mat, int nblocks, int nkeys,
                           unsigned* __restrict__ totals) {
  extern __shared__ unsigned slab[];  // [nblocks][kScanKeys + 1]
  __shared__ unsigned seg_sum[kScanSegs][kScanKeys];
  const int k0 = blockIdx.x * kScanKeys;
  const int W = kScanKeys + 1;
  // eight independent loads in flight per thread before their shared stores
  constexpr int kBatch = 8;
  for (int idx0 = threadIdx.x; idx0 < nblocks * kScanKeys; idx0 += kBatch * blockDim.x) {
    unsigned v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int idx = idx0 + u * blockDim.x;
      const int b = idx / kScanKeys, c = idx % kScanKeys;
      v[u] = (idx < nblocks * kScanKeys && k0 + c < nkeys) ? mat[(int64_t)b * nkeys + k0 + c] : 0u;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int idx = idx0 + u * blockDim.x;
      if (idx < nblocks * kScanKeys) slab[(idx / kScanKeys) * W + idx % kScanKeys] = v[u];
    }
  }
  __syncthreads();
  const int c = threadIdx.x % kScanKeys, sg = threadIdx.x / kScanKeys;
  const int len = (nblocks + kScanSegs - 1) / kScanSegs;
  const int b0 = sg * len, b1 = min(nblocks, b0 + len);
  unsigned sum = 0;
  for (int b = b0; b < b1; ++b) sum += slab[b * W + c];
  seg_sum[sg][c] = sum;
  __syncthreads();
  unsigned run = 0, total = 0;
  for (int g = 0; g < kScanSegs; ++g) {
    if (g < sg) run += seg_sum[g][c];
    total += seg_sum[g][c];
  }
  for (int b = b0; b < b1; ++b) {
    unsigned v = slab[b * W + c];
    slab[b * W + c] = run;
    run += v;
  }
  if (sg == 0 && k0 + c < nkeys) totals[k0 + c] = total;
  __syncthreads();
  for (int idx = threadIdx.x; idx < nblocks * kScanKeys; idx += blockDim.x) {
    int b = idx / kScanKeys, cc = idx % kScanKeys;
    if (k0 + cc < nkeys) mat[(int64_t)b * nkeys + k0 + cc] = slab[b * W + cc];
  }
}

struct TileGeom {
  int64_t M[KDE_MAX_D];
  int64_t stride[KDE_MAX_D];
  int tile[KDE_MAX_D];      // powers of two
  int tile_log2[KDE_MAX_D];
  int ntiles[KDE_MAX_D];
  int tstride[KDE_MAX_D];
  int ntiles_total;
  int tile_cells;
  int item_cap;
};

template <int D>
__device__ __forceinline__ void tile_coords(int t, const TileGeom& g, int* tc) {
  int rem = t;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    tc[k] = rem / g.tstride[k];
    rem -= tc[k] * g.tstride[k];
  }
}

// Calls f(nb_tile, o, key) for the key ranges feeding tile t, in a fixed
// order: the tile's own keys (o = 0, all masks), then for each o != 0 the
// neighbour t - o and its masks that contain o.
template <int D, typename F>
__device__ __forceinline__ void for_each_source(const int* tc, const TileGeom& g, F f) {
  for (int o = 0; o < (1 << D); ++o) {
    int ntile = 0;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      int nk = tc[k] - ((o >> (D - 1 - k)) & 1);
      ok &= nk >= 0;
      ntile += nk * g.tstride[k];
    }
    if (!ok) continue;
    for (int mask = 0; mask < (1 << D); ++mask)
      if ((mask & o) == o) f(ntile, o, (ntile << D) | mask);
  }
}

// Exclusive prefix of v[0, n) into out[0, n) and the total into out[n],
// by the whole block: each warp scans a contiguous segment 32 values at a
// time (coalesced, no bank conflicts), after an exclusive scan of the
// segments' totals.  v and out may live in global or shared memory.
__device__ void block_segment_scan(const unsigned* v, int n, unsigned* out, unsigned* warp_sums) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int seg = (n + nw - 1) / nw;
  const int k0 = min(n, warp * seg), k1 = min(n, k0 + seg);
  unsigned sum = 0;
  for (int k = k0 + lane; k < k1; k += 32) sum += v[k];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
  __syncthreads();
  if (lane == 0) warp_sums[warp] = sum;
  __syncthreads();
  if (warp == 0) {
    const unsigned x = lane < nw ? warp_sums[lane] : 0u;
    unsigned inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    warp_sums[lane] = inc - x;
    if (lane == 31) warp_sums[32] = inc;
  }
  __syncthreads();
  unsigned carry = warp_sums[warp];
  for (int kb = k0; kb < k1; kb += 32) {
    const int k = kb + lane;
    const unsigned x = k < k1 ? v[k] : 0u;
    unsigned inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    if (k < k1) out[k] = carry + inc - x;
    carry += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (threadIdx.x == 0) out[n] = warp_sums[32];
  __syncthreads();
}

// One block: starts[key] = exclusive prefix of key totals (starts[nkeys] =
// all records); per tile the records feeding it (own plus neighbours' face
// records), its number of work items (ceil(records / cap), at least 1) and
// the exclusive prefix of items over tiles (item_start[ntiles] = all
// items).  The per-tile sums read a mask-major copy of the totals in shared
// memory, so the lanes of a warp (consecutive tiles) read consecutive words.
template <int D>
__global__ void __launch_bounds__(1024)
kde_bin_scan_keys_kernel(const unsigned* __restrict__ totals, int nkeys, TileGeom g,
                         unsigned* __restrict__ starts, unsigned* __restrict__ item_start) {
  extern __shared__ unsigned smem_scan[];
  __shared__ unsigned warp_sums[33];
  const int ntiles = g.ntiles_total, nm = 1 << D;
  unsigned* s_tot = smem_scan;            // [mask][tile]
  unsigned* s_items = smem_scan + nkeys;  // [tile]
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x) s_tot[(k & (nm - 1)) * ntiles + (k >> D)] = totals[k];
  block_segment_scan(totals, nkeys, starts, warp_sums);
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
    int tc[KDE_MAX_D];
    tile_coords<D>(t, g, tc);
    unsigned recs = 0;
    for_each_source<D>(tc, g, [&](int nbt, int, int key) {
      recs += s_tot[(key & (nm - 1)) * ntiles + nbt];
    });
    s_items[t] = recs == 0 ? 1u : (recs + g.item_cap - 1) / g.item_cap;
  }
  __syncthreads();
  block_segment_scan(s_items, ntiles, item_start, warp_sums);
}

template <typename T, int D>
__global__ void __launch_bounds__(kHistThreads)
kde_bin_scatter_kernel(const T* __restrict__ X, int64_t n, int64_t chunk, int nkeys,
                       BinParams<T> p, const unsigned* __restrict__ mat,
                       const unsigned* __restrict__ starts, uint4* __restrict__ recs) {
  extern __shared__ unsigned cursor[];
  const unsigned* row = mat + (int64_t)blockIdx.x * nkeys;
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x) cursor[k] = starts[k] + row[k];
  __syncthreads();
  const int64_t s0 = (int64_t)blockIdx.x * chunk;
  const int64_t s1 = min(n, s0 + chunk);
  T xc[kUnroll][D], xn[kUnroll][D];
  load_samples<T, D>(X, s0 + threadIdx.x, s1, xc);
  for (int64_t base = s0 + threadIdx.x; base < s1; base += kUnroll * (int64_t)blockDim.x) {
    load_samples<T, D>(X, base + kUnroll * (int64_t)blockDim.x, s1, xn);
    int key[kUnroll];
    uint4 rec[kUnroll];
    bool in[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t s = base + u * (int64_t)blockDim.x;
      in[u] = s < s1 && sample_key<T, D>(xc[u], p, key[u], rec[u]);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
      if (in[u]) recs[atomicAdd(&cursor[key[u]], 1u)] = rec[u];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < D; ++k) xc[u][k] = xn[u][k];
  }
}

// Global offset of tile-local cell c (last axis fastest; tile extents are
// powers of two), or -1 if the cell lies beyond the grid's edge.
template <int D>
__device__ __forceinline__ int64_t tile_cell_offset(const int* tc, const TileGeom& g, int c) {
  int64_t off = 0;
  bool in = true;
#pragma unroll
  for (int k = D - 1; k >= 0; --k) {
    const int x = c & (g.tile[k] - 1);
    c >>= g.tile_log2[k];
    const int64_t gx = (int64_t)tc[k] * g.tile[k] + x;
    in &= gx < g.M[k];
    off += gx * g.stride[k];
  }
  return in ? off : -1;
}

// Store a tile's owned cells (clipped at the grid's edge), last axis fastest.
template <int D, typename F>
__device__ __forceinline__ void store_tile(const int* tc, const TileGeom& g, int c0, int cstep,
                                           unsigned long long* __restrict__ counts, F value) {
  for (int c = c0; c < g.tile_cells; c += cstep) {
    const int64_t off = tile_cell_offset<D>(tc, g, c);
    if (off >= 0) counts[off] = value(c);
  }
}

// Accumulate records [r0, r1) of one source bucket into this tile's cells.
// The bucket is (neighbour tile t - o, face mask m ⊇ o): along axis k its
// records' corners at offset 1 land here if o has axis k (the base is the
// neighbour's last row), only those at offset 0 if m has axis k but o not
// (the offset-1 corner belongs to the next tile), and both otherwise.  So
// the corners to add are the same for every record of the bucket (mask cm)
// and land inside the tile; a corner beyond the grid's last node has weight
// 0 and is skipped with every other zero weight.  A weight w <= 2^32 is
// added as two parts into separate 32-bit words, lo += w mod 2^16 and
// hi += w >> 16 (shared 32-bit atomics run about six times faster than
// 64-bit ones).  A work item adds at most item_cap <= 65535 records to a
// cell, so neither word can overflow; the cell is hi 2^16 + lo.
// One record's corners (those in cm) added into the tile's two accumulator
// words per cell; base is the record's base node as a tile-local index.
template <int D, bool ALL>
__device__ __forceinline__ void add_record(const uint4& rec, int base, int cm, const int* cstride,
                                           unsigned cells, unsigned* acc_lo, unsigned* acc_hi) {
  const unsigned q[3] = {rec.y, rec.z, rec.w};
  unsigned long long w[1 << D];
  corner_weights<D>(q, w);
#pragma unroll
  for (int c = 0; c < (1 << D); ++c) {
    if (!ALL && !((cm >> c) & 1)) continue;
    int lidx = base;
#pragma unroll
    for (int k = 0; k < D; ++k)
      if ((c >> (D - 1 - k)) & 1) lidx += cstride[k];
    const unsigned wl = (unsigned)w[c] & 0xffffu, wh = (unsigned)(w[c] >> 16);
    if ((unsigned)lidx < cells) {
      if (wl) atomicAdd(&acc_lo[lidx], wl);
      if (wh) atomicAdd(&acc_hi[lidx], wh);
    }
  }
}

// Records [r0, r1) of one bucket, one per thread per iteration, the next
// record's load issued before the current one is added.
template <int D, bool ALL>
__device__ __forceinline__ void add_records(const uint4* __restrict__ recs, unsigned r0, unsigned r1,
                                            int shift, int cm, const int* cstride, unsigned cells,
                                            unsigned* acc_lo, unsigned* acc_hi) {
  constexpr int B = LocalBits<D>::value;
  const unsigned lmask = B == 32 ? 0xffffffffu : ((1u << B) - 1u);
  unsigned r = r0 + threadIdx.x;
  if (r >= r1) return;
  uint4 cur = recs[r];
  for (;;) {
    const unsigned rn = r + blockDim.x;
    uint4 nxt;
    if (rn < r1) nxt = recs[rn];
    int base = shift;
#pragma unroll
    for (int k = 0; k < D; ++k) base += (int)((cur.x >> (B * k)) & lmask) * cstride[k];
    add_record<D, ALL>(cur, base, cm, cstride, cells, acc_lo, acc_hi);
    if (rn >= r1) break;
    cur = nxt;
    r = rn;
  }
}

// Accumulate records [r0, r1) of one source bucket into this tile's cells.
// The bucket is (neighbour tile t - o, face mask m ⊇ o): along axis k its
// records' corners at offset 1 land here if o has axis k (the base is the
// neighbour's last row), only those at offset 0 if m has axis k but o not
// (the offset-1 corner belongs to the next tile), and both otherwise.  So
// the corners to add are the same for every record of the bucket (mask cm)
// and land inside the tile; a corner beyond the grid's last node has weight
// 0 and is skipped with every other zero weight.  Own records off every face
// (o = m = 0, nearly all of them) take all corners with no mask test.  A
// weight w <= 2^32 is added as two parts into separate 32-bit words,
// lo += w mod 2^16 and hi += w >> 16 (shared 32-bit atomics run about six
// times faster than 64-bit ones).  A work item adds at most
// item_cap <= 65535 records to a cell, so neither word can overflow; the
// cell is hi 2^16 + lo.
template <int D>
__device__ __forceinline__ void accumulate(const uint4* __restrict__ recs, unsigned r0, unsigned r1,
                                           int o, int m, const TileGeom& g, unsigned* acc_lo,
                                           unsigned* acc_hi) {
  int cm = 0;
#pragma unroll
  for (int c = 0; c < (1 << D); ++c) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const int bit = D - 1 - k, ck = (c >> bit) & 1;
      if ((o >> bit) & 1) ok &= ck == 1;
      else if ((m >> bit) & 1) ok &= ck == 0;
    }
    cm |= (int)ok << c;
  }
  // tile-local index strides; the base shifts by -tile along every axis of o
  int cstride[KDE_MAX_D];
  int shift = 0;
  {
    int st = 1;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) {
      cstride[k] = st;
      if ((o >> (D - 1 - k)) & 1) shift -= g.tile[k] * st;
      st *= g.tile[k];
    }
  }
  const unsigned cells = (unsigned)g.tile_cells;
  if (cm == (1 << (1 << D)) - 1)
    add_records<D, true>(recs, r0, r1, shift, cm, cstride, cells, acc_lo, acc_hi);
  else
    add_records<D, false>(recs, r0, r1, shift, cm, cstride, cells, acc_lo, acc_hi);
}

// Zero the cells of tiles that are split into several work items (their
// items add into the counts with atomics); every other cell is stored once.
template <int D>
__global__ void __launch_bounds__(kGatherThreads)
kde_bin_zero_split_kernel(const unsigned* __restrict__ item_start, TileGeom g,
                          unsigned long long* __restrict__ counts) {
  const int t = blockIdx.x;
  if (item_start[t + 1] - item_start[t] <= 1) return;
  int tc[KDE_MAX_D];
  tile_coords<D>(t, g, tc);
  store_tile<D>(tc, g, blockIdx.y * blockDim.x + threadIdx.x, gridDim.y * blockDim.x, counts,
                [](int) { return 0ull; });
}

// One block per work item.  The records feeding tile t (own, then each
// neighbour's face records, in for_each_source order) are numbered
// 0 .. R-1; item j takes [j cap, (j+1) cap).  A tile with one item stores
// its cells; items of a split tile add their nonzero cells with 64-bit
// atomics (integer sums: the result does not depend on their order).
template <int D>
__global__ void __launch_bounds__(kGatherThreads)
kde_bin_gather_kernel(const uint4* __restrict__ recs, const unsigned* __restrict__ starts,
                      const unsigned* __restrict__ item_start, TileGeom g,
                      unsigned long long* __restrict__ counts) {
  extern __shared__ unsigned acc_words[];
  unsigned* acc_lo = acc_words;
  unsigned* acc_hi = acc_words + g.tile_cells;
  const unsigned b = blockIdx.x;
  if (b >= item_start[g.ntiles_total]) return;
  int lo = 0, hi = g.ntiles_total - 1;  // largest t with item_start[t] <= b
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (item_start[mid] <= b) lo = mid; else hi = mid - 1;
  }
  const int t = lo;
  const unsigned j = b - item_start[t];
  const unsigned items = item_start[t + 1] - item_start[t];
  int tc[KDE_MAX_D];
  tile_coords<D>(t, g, tc);
  for (int c = threadIdx.x; c < 2 * g.tile_cells; c += blockDim.x) acc_words[c] = 0;
  __syncthreads();
  const unsigned w0 = j * (unsigned)g.item_cap, w1 = w0 + (unsigned)g.item_cap;
  unsigned v = 0;  // running record number
  for_each_source<D>(tc, g, [&](int, int o, int key) {
    const unsigned a = starts[key], len = starts[key + 1] - a;
    const unsigned lo_v = max(v, w0), hi_v = min(v + len, w1);
    if (lo_v < hi_v)
      accumulate<D>(recs, a + (lo_v - v), a + (hi_v - v), o, key & ((1 << D) - 1), g, acc_lo, acc_hi);
    v += len;
  });
  __syncthreads();
  auto cell = [&](int c) {
    return ((unsigned long long)acc_hi[c] << 16) + (unsigned long long)acc_lo[c];
  };
  if (items == 1) {
    store_tile<D>(tc, g, threadIdx.x, blockDim.x, counts, cell);
  } else {
    for (int c = threadIdx.x; c < g.tile_cells; c += blockDim.x) {
      const unsigned long long v = cell(c);
      if (!v) continue;
      const int64_t off = tile_cell_offset<D>(tc, g, c);
      if (off >= 0) atomicAdd(counts + off, v);
    }
  }
}

// Tile extents: start from 2048 / 32x64 / 16x16x32 cells and grow while the
// key count (tiles x 2^d) exceeds what one block's shared histogram holds.
bool choose_tiles(int d, const int64_t* M, int* tile, int* ntiles, int* nkeys) {
  static const int init[3][3] = {{2048, 0, 0}, {32, 64, 0}, {16, 16, 32}};
  for (int k = 0; k < d; ++k) tile[k] = init[d - 1][k];
  for (int iter = 0; iter < 64; ++iter) {
    int64_t nt = 1;
    for (int k = 0; k < d; ++k) {
      ntiles[k] = (int)((M[k] + tile[k] - 1) / tile[k]);
      nt *= ntiles[k];
    }
    if (nt * (1 << d) <= kMaxKeys) {
      *nkeys = (int)(nt << d);
      return true;
    }
    // grow the axis with the most tiles, keeping shared memory per tile <= 128 KB
    int best = -1;
    for (int k = 0; k < d; ++k)
      if (tile[k] < 256 && (best < 0 || ntiles[k] > ntiles[best])) best = k;
    int64_t cells = 1;
    for (int k = 0; k < d; ++k) cells *= tile[k];
    if (best < 0 || cells * 2 * 8 > 128 * 1024) return false;
    tile[best] *= 2;
  }
  return false;
}

struct TiledLayout {
  int tile[KDE_MAX_D], ntiles[KDE_MAX_D], nkeys, nblocks, tile_cells, item_cap, ntiles_total;
  int64_t chunk, max_items;
  size_t off_mat, off_tot, off_starts, off_items, off_recs, total;
};

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

bool tiled_layout(int64_t n, int d, const int64_t* M, TiledLayout* t) {
  if (!choose_tiles(d, M, t->tile, t->ntiles, &t->nkeys)) return false;
  // chunks of at least 4096 samples, at most one resident wave of
  // histogram blocks (their shared key histograms bound the blocks per SM)
  const int64_t per_sm = std::max<int64_t>(
      1, std::min<int64_t>(2048 / kHistThreads, (int64_t)(200 * 1024) / ((int64_t)t->nkeys * 4)));
  const int64_t cap = std::min<int64_t>(kMaxBlocks, per_sm * num_sms());
  int64_t nb = (n + 4095) / 4096;
  t->nblocks = (int)(nb < 1 ? 1 : (nb > cap ? cap : nb));
  t->chunk = (n + t->nblocks - 1) / t->nblocks;
  t->tile_cells = 1;
  t->ntiles_total = 1;
  for (int k = 0; k < d; ++k) {
    t->tile_cells *= t->tile[k];
    t->ntiles_total *= t->ntiles[k];
  }
  // records per work item: about twice the tile's cells (each item zeroes
  // and stores a whole tile; larger items leave the heaviest tiles to few
  // blocks), at most 65535 (the accumulator bound)
  t->item_cap = std::max(2048, std::min(65535, 2 * t->tile_cells));
  // A record feeds at most 2^d tiles: items <= tiles + 2^d n / cap.
  const int64_t feeds = (int64_t)n << d;
  t->max_items = t->ntiles_total + feeds / t->item_cap + 1;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  t->off_mat = 0;
  t->off_tot = up((size_t)t->nblocks * t->nkeys * 4);
  t->off_starts = t->off_tot + up((size_t)t->nkeys * 4);
  t->off_items = t->off_starts + up((size_t)(t->nkeys + 1) * 4);
  t->off_recs = t->off_items + up((size_t)(t->ntiles_total + 1) * 4);
  t->total = t->off_recs + up((size_t)(n > 0 ? n : 1) * 16);
  return true;
}

template <typename T>
BinParams<T> make_params(int d, const double* lo, const double* hi, const int64_t* M,
                         const TiledLayout* t) {
  BinParams<T> p{};
  int64_t stride = 1;
  int ts = 1;
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
      ts *= t->ntiles[k];
    }
  }
  return p;
}


template <typename T>
kde_status launch_direct(const T* X, int64_t n, int d, const double* lo, const double* hi,
                         const int64_t* M, unsigned long long* counts, int64_t cells,
                         unsigned long long* n_out, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)cells * sizeof(int64_t), stream);
  if (e != cudaSuccess) return kde::cuda_fail(e, "cudaMemsetAsync(counts)");
  if (n == 0) return KDE_OK;
  BinParams<T> p = make_params<T>(d, lo, hi, M, nullptr);
  int64_t want = (2 * n + 255) / 256;  // two lanes per sample
  int64_t cap = (int64_t)num_sms() * 8;
  int blocks = (int)(want < cap ? want : cap);
  kde::LaunchScope ls("kde_bin_kernel", stream);
  switch (d) {
    case 1: kde_bin_kernel<T, 1><<<blocks, 256, 0, stream>>>(X, n, p, counts, n_out); break;
    case 2: kde_bin_kernel<T, 2><<<blocks, 256, 0, stream>>>(X, n, p, counts, n_out); break;
    default: kde_bin_kernel<T, 3><<<blocks, 256, 0, stream>>>(X, n, p, counts, n_out); break;
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : kde::cuda_fail(e, "kde_bin_kernel launch");
}

template <typename F>
cudaError_t allow_smem(F* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int D>
kde_status launch_tiled_d(const T* X, int64_t n, const double* lo, const double* hi,
                          const int64_t* M, unsigned long long* counts,
                          unsigned long long* n_out, const TiledLayout& t, char* ws,
                          cudaStream_t stream) {
  BinParams<T> p = make_params<T>(D, lo, hi, M, &t);
  unsigned* mat = (unsigned*)(ws + t.off_mat);
  unsigned* tot = (unsigned*)(ws + t.off_tot);
  unsigned* starts = (unsigned*)(ws + t.off_starts);
  unsigned* item_start = (unsigned*)(ws + t.off_items);
  uint4* recs = (uint4*)(ws + t.off_recs);
  TileGeom g{};
  for (int k = 0; k < D; ++k) {
    g.M[k] = M[k];
    g.stride[k] = p.ax[k].stride;
    g.tile[k] = t.tile[k];
    g.tile_log2[k] = p.ax[k].tile_log2;
    g.ntiles[k] = t.ntiles[k];
    g.tstride[k] = p.ax[k].tstride;
  }
  g.ntiles_total = t.ntiles_total;
  g.tile_cells = t.tile_cells;
  g.item_cap = t.item_cap;
  const size_t hist_smem = (size_t)t.nkeys * 4;
  cudaError_t e;
  {
    auto* fn = kde_bin_hist_kernel<T, D>;
    if ((e = allow_smem(fn, hist_smem)) != cudaSuccess) return kde::cuda_fail(e, "smem attr");
    kde::LaunchScope ls("kde_bin_hist_kernel", stream);
    fn<<<t.nblocks, kHistThreads, hist_smem, stream>>>(X, n, t.chunk, t.nkeys, p, mat, n_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return kde::cuda_fail(e, "kde_bin_hist_kernel");
  }
  {
    const size_t smem = (size_t)t.nblocks * (kScanKeys + 1) * 4;
    if ((e = allow_smem(kde_bin_scan_blocks_kernel, smem)) != cudaSuccess)
      return kde::cuda_fail(e, "smem attr");
    kde::LaunchScope ls("kde_bin_scan_blocks_kernel", stream);
    kde_bin_scan_blocks_kernel<<<(t.nkeys + kScanKeys - 1) / kScanKeys, kScanKeys * kScanSegs, smem,
                                 stream>>>(mat, t.nblocks, t.nkeys, tot);
    if ((e = cudaGetLastError()) != cudaSuccess) return kde::cuda_fail(e, "kde_bin_scan_blocks_kernel");
  }
  {
    auto* fn = kde_bin_scan_keys_kernel<D>;
    const size_t ssmem = (size_t)(t.nkeys + t.ntiles_total) * 4;
    if ((e = allow_smem(fn, ssmem)) != cudaSuccess) return kde::cuda_fail(e, "smem attr");
    kde::LaunchScope ls("kde_bin_scan_keys_kernel", stream);
    fn<<<1, 1024, ssmem, stream>>>(tot, t.nkeys, g, starts, item_start);
    if ((e = cudaGetLastError()) != cudaSuccess) return kde::cuda_fail(e, "kde_bin_scan_keys_kernel");
  }
  {
    auto* fn = kde_bin_scatter_kernel<T, D>;
    if ((e = allow_smem(fn, hist_smem)) != cudaSuccess) return kde::cuda_fail(e, "smem attr");
    kde::LaunchScope ls("kde_bin_scatter_kernel", stream);
    fn<<<t.nblocks, kHistThreads, hist_smem, stream>>>(X, n, t.chunk, t.nkeys, p, mat, starts, recs);
    if ((e = cudaGetLastError()) != cudaSuccess) return kde::cuda_fail(e, "kde_bin_scatter_kernel");
  }
  {
    kde::LaunchScope ls("kde_bin_zero_split_kernel", stream);
    kde_bin_zero_split_kernel<D><<<dim3((unsigned)t.ntiles_total, 4), kGatherThreads, 0, stream>>>(
        item_start, g, counts);
    if ((e = cudaGetLastError()) != cudaSuccess) return kde::cuda_fail(e, "kde_bin_zero_split_kernel");
  }
  const size_t gsmem = (size_t)t.tile_cells * 8;
  {
    auto* fn = kde_bin_gather_kernel<D>;
    if ((e = allow_smem(fn, gsmem)) != cudaSuccess) return kde::cuda_fail(e, "smem attr");
    kde::LaunchScope ls("kde_bin_gather_kernel", stream);
    fn<<<(unsigned)t.max_items, kGatherThreads, gsmem, stream>>>(recs, starts, item_start, g, counts);
    if ((e = cudaGetLastError()) != cudaSuccess) return kde::cuda_fail(e, "kde_bin_gather_kernel");
  }
  return KDE_OK;
}

template <typename T>
kde_status launch_tiled(const T* X, int64_t n, int d, const double* lo, const double* hi,
                        const int64_t* M, unsigned long long* counts, unsigned long long* n_out,
                        const TiledLayout& t, char* ws, cudaStream_t stream) {
  switch (d) {
    case 1: return launch_tiled_d<T, 1>(X, n, lo, hi, M, counts, n_out, t, ws, stream);
    case 2: return launch_tiled_d<T, 2>(X, n, lo, hi, M, counts, n_out, t, ws, stream);
    default: return launch_tiled_d<T, 3>(X, n, lo, hi, M, counts, n_out, t, ws, stream);
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

extern "C" kde_status kde_bin(const void* X, int x_dtype, int64_t n, int d, const double* lo,
                              const double* hi, const int64_t* M, int64_t* counts,
                              int64_t* n_outside, void* workspace, size_t workspace_bytes,
                              kde_stream_t stream) {
  using kde::fail;
  int64_t cells = 0;
  kde_status st = check_bin_args(d, x_dtype, n, X, lo, hi, M, &cells);
  if (st != KDE_OK) return st;
  if (!counts) return fail(KDE_ERR_INVALID_ARG, "counts is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  auto* c = reinterpret_cast<unsigned long long*>(counts);
  auto* no = reinterpret_cast<unsigned long long*>(n_outside);
  if (n_outside) {
    cudaError_t e = cudaMemsetAsync(n_outside, 0, sizeof(int64_t), s);
    if (e != cudaSuccess) return kde::cuda_fail(e, "cudaMemsetAsync(n_outside)");
  }
  if (!workspace) {
    if (x_dtype == KDE_F32)
      return launch_direct<float>((const float*)X, n, d, lo, hi, M, c, cells, no, s);
    return launch_direct<double>((const double*)X, n, d, lo, hi, M, c, cells, no, s);
  }
  TiledLayout t{};
  if (!tiled_layout(n, d, M, &t))
    return fail(KDE_ERR_UNSUPPORTED, "grid too large for the tiled binning path");
  if (cells >= (int64_t(1) << 32)) return fail(KDE_ERR_UNSUPPORTED, "tiled binning needs prod(M) < 2^32");
  if (workspace_bytes < t.total) return fail(KDE_ERR_WORKSPACE, "binning workspace too small");
  if (((uintptr_t)workspace & 255) != 0) return fail(KDE_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  if (x_dtype == KDE_F32)
    return launch_tiled<float>((const float*)X, n, d, lo, hi, M, c, no, t, (char*)workspace, s);
  return launch_tiled<double>((const double*)X, n, d, lo, hi, M, c, no, t, (char*)workspace, s);
}
