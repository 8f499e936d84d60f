// Linear binning (Sec. 2, first step): each sample inside the grid spreads a
// unit mass over its 2^d neighbouring nodes with integer weights in units of
// 2^-32 that sum to exactly 2^32 (so the counts sum to n, Sec. 3 footnote),
// accumulated with 64-bit integer atomics.  Integer addition is associative,
// so the counts are bit-identical whatever order the atomics land in.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "kde_internal.h"

namespace {

constexpr unsigned long long kOne = 1ull << 32;

// floor((w*Q + 2^31) / 2^32) for 0 <= w, Q <= 2^32 using the full 128-bit product.
__device__ __forceinline__ unsigned long long mulhi_round(unsigned long long w,
                                                          unsigned long long Q) {
  unsigned long long lo = w * Q;
  unsigned long long hi = __umul64hi(w, Q);
  unsigned long long lo2 = lo + (1ull << 31);
  hi += (lo2 < lo) ? 1ull : 0ull;
  return (hi << 32) | (lo2 >> 32);
}

template <typename T>
struct BinAxis {
  T lo;      // lo rounded to X's type
  T s;       // (M-1)/(hi-lo) computed in FP64, rounded to X's type
  T top;     // M - 1 in X's type
  int64_t stride;
  int64_t M;
};

template <typename T>
struct BinParams {
  BinAxis<T> ax[KDE_MAX_D];
};

__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Position of one coordinate: node index i and fixed-point fraction Q.
// Returns false if the coordinate is outside [0, M-1] or NaN.
template <typename T>
__device__ __forceinline__ bool axis_position(T x, const BinAxis<T>& a, int64_t& i,
                                              unsigned long long& Q) {
  T t = mul_rn(sub_rn(x, a.lo), a.s);
  if (!(t >= T(0) && t <= a.top)) return false;
  T fl = floor(t);
  i = (int64_t)fl;
  T f = sub_rn(t, fl);  // exact
  if (i == a.M - 1) {
    i = a.M - 2;
    f = T(1);
  }
  Q = __double2ull_rn((double)f * 4294967296.0);  // exact scaling, ties to even
  return true;
}

template <typename T, int D>
__global__ void __launch_bounds__(256) kde_bin_kernel(const T* __restrict__ X, int64_t n,
                                                      BinParams<T> p,
                                                      unsigned long long* __restrict__ counts,
                                                      unsigned long long* __restrict__ n_out) {
  unsigned long long outside = 0;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    int64_t i[D];
    unsigned long long Q[D];
    bool in = true;
#pragma unroll
    for (int k = 0; k < D; ++k) in &= axis_position<T>(X[s * D + k], p.ax[k], i[k], Q[k]);
    if (!in) {
      ++outside;
      continue;
    }
    int64_t base = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) base += i[k] * p.ax[k].stride;
    // Hierarchical split of the unit mass, axis 0 first; corner c has offset
    // bit (c >> (D-1-k)) & 1 on axis k.
    unsigned long long w[1 << D];
    w[0] = kOne;
#pragma unroll
    for (int k = 0; k < D; ++k) {
#pragma unroll
      for (int c = (1 << k) - 1; c >= 0; --c) {
        unsigned long long hi = mulhi_round(w[c], Q[k]);
        w[2 * c + 1] = hi;
        w[2 * c] = w[c] - hi;
      }
    }
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
      if (w[c] == 0) continue;
      int64_t idx = base;
#pragma unroll
      for (int k = 0; k < D; ++k)
        if ((c >> (D - 1 - k)) & 1) idx += p.ax[k].stride;
      atomicAdd(counts + idx, w[c]);
    }
  }
  if (n_out) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) outside += __shfl_down_sync(0xffffffffu, outside, off);
    if ((threadIdx.x & 31) == 0 && outside) atomicAdd(n_out, outside);
  }
}

template <typename T>
kde_status launch_bin(const T* X, int64_t n, int d, const double* lo, const double* hi,
                      const int64_t* M, unsigned long long* counts, unsigned long long* n_out,
                      cudaStream_t stream) {
  BinParams<T> p{};
  int64_t stride = 1;
  for (int k = d - 1; k >= 0; --k) {
    double s = (double)(M[k] - 1) / (hi[k] - lo[k]);
    p.ax[k].lo = (T)lo[k];
    p.ax[k].s = (T)s;
    p.ax[k].top = (T)(M[k] - 1);
    p.ax[k].stride = stride;
    p.ax[k].M = M[k];
    stride *= M[k];
  }
  if (n == 0) return KDE_OK;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = (n + 255) / 256;
  int64_t cap = (int64_t)sms * 8;
  int blocks = (int)(want < cap ? want : cap);
  kde::LaunchScope ls("kde_bin_kernel", stream);
  switch (d) {
    case 1: kde_bin_kernel<T, 1><<<blocks, 256, 0, stream>>>(X, n, p, counts, n_out); break;
    case 2: kde_bin_kernel<T, 2><<<blocks, 256, 0, stream>>>(X, n, p, counts, n_out); break;
    default: kde_bin_kernel<T, 3><<<blocks, 256, 0, stream>>>(X, n, p, counts, n_out); break;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : kde::cuda_fail(e, "kde_bin_kernel launch");
}

}  // namespace

extern "C" kde_status kde_bin(const void* X, int x_dtype, int64_t n, int d, const double* lo,
                              const double* hi, const int64_t* M, int64_t* counts,
                              int64_t* n_outside, kde_stream_t stream) {
  using kde::fail;
  if (d < 1 || d > KDE_MAX_D) return fail(KDE_ERR_UNSUPPORTED, "d must be 1, 2 or 3");
  if (!lo || !hi || !M || !counts) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
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
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)cells * sizeof(int64_t), s);
  if (e != cudaSuccess) return kde::cuda_fail(e, "cudaMemsetAsync(counts)");
  if (n_outside) {
    e = cudaMemsetAsync(n_outside, 0, sizeof(int64_t), s);
    if (e != cudaSuccess) return kde::cuda_fail(e, "cudaMemsetAsync(n_outside)");
  }
  auto* c = reinterpret_cast<unsigned long long*>(counts);
  auto* no = reinterpret_cast<unsigned long long*>(n_outside);
  if (x_dtype == KDE_F32)
    return launch_bin<float>((const float*)X, n, d, lo, hi, M, c, no, s);
  return launch_bin<double>((const double*)X, n, d, lo, hi, M, c, no, s);
}
