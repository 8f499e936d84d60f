// The convolution step (Eq. 10) in wrapped, zero-padded form:
//   kde_kernel_grid: k_l on |l_k| <= L_k at index l mod P_k (Eq. 6, Eq. 12
//                    without the shift), transformed to its real spectrum K;
//   kde_fft_eval:    C = F(c) of the zero-padded counts, S = C K,
//                    s = F^{-1}(S), cropped to [0, M_k) (Eq. 14 shifted).
// Passes (row-major, last axis contiguous, Q = P_last/2 + 1):
//   rows_r2c  real rows -> half spectra; two real rows ride in one complex
//             FFT (x + i y) and are separated afterwards;
//   cols      FFT along a strided axis on a tile of T adjacent columns in
//             shared memory: forward, forward-to-real (kernel spectrum),
//             forward * K * inverse with crop (the middle axis), or inverse
//             with crop;
//   rows_c2r  half spectra -> real rows, cropped (two rows per complex FFT);
//   line1d    d = 1: forward, * K, inverse and crop in one block.
// Only lines that hold data are transformed and only lines that survive the
// crop are inverse-transformed.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <set>
#include <string>

#include "fft_engine.cuh"
#include "kde_internal.h"

namespace kde {
namespace {

constexpr int kThreads = 256;

template <typename T>
struct KGen {
  int d;
  int L[KDE_MAX_D];
  int wand;
  T A[KDE_MAX_D][KDE_MAX_D];  // delta_a delta_b (H^-1)_ab
  T C;                        // (2 pi)^{-d/2} |H|^{-1/2} / (n 2^32 prod P)
};

__device__ __forceinline__ float ex(float x) { return expf(x); }
__device__ __forceinline__ double ex(double x) { return exp(x); }

// k at lag l (Eq. 6 with the normalisations folded in).
template <typename T>
__device__ __forceinline__ T kernel_value(const KGen<T>& g, const int* l) {
  T q = 0;
#pragma unroll
  for (int a = 0; a < KDE_MAX_D; ++a) {
    if (a >= g.d) break;
    T la = (T)(g.wand ? abs(l[a]) : l[a]);
#pragma unroll
    for (int b = 0; b < KDE_MAX_D; ++b) {
      if (b >= g.d) break;
      T lb = (T)(g.wand ? abs(l[b]) : l[b]);
      q += g.A[a][b] * la * lb;
    }
  }
  return g.C * ex(T(-0.5) * q);
}

// Signed lag stored at wrapped position p of a length-P axis with support L,
// or a value > L if the position holds zero padding.
__device__ __forceinline__ int wrapped_lag(int p, int P, int L) {
  if (p <= L) return p;
  if (p >= P - L) return p - P;
  return L + 1;
}

template <typename T>
struct RowsParams {
  using V = typename Cplx<T>::type;
  int64_t nrows;      // real rows
  int Min;            // data length of a row (zero-padded to P)
  int64_t in_stride;  // elements between input rows
  int P, Q;
  V* out;             // complex half spectra, row stride Q
  T* out_real;        // real part only (d = 1 kernel spectrum)
  int G;              // complex lines (row pairs) per block
  Radices rp;
  const V* tw;
};

template <typename V, typename T>
__device__ __forceinline__ void load_twiddles(V* tw_s, const V* tw, int P) {
  for (int i = threadIdx.x; i < P; i += blockDim.x) tw_s[i] = tw[i];
}

// Split Z = F(x + i y) into X = F(x), Y = F(y) for k in [0, Q) and store.
template <typename T>
__device__ __forceinline__ void store_r2c(const RowsParams<T>& p, const typename Cplx<T>::type* z,
                                          int64_t r0, int g) {
  using V = typename Cplx<T>::type;
  const int P = p.P;
  for (int k = threadIdx.x; k < p.Q; k += blockDim.x) {
    V zk = z[g * P + k];
    V zm = z[g * P + (k == 0 ? 0 : P - k)];
    V X = mk<V>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
    V Y = mk<V>(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
    if (p.out_real) {
      p.out_real[r0 * p.Q + k] = X.x;
    } else {
      p.out[r0 * p.Q + k] = X;
      if (r0 + 1 < p.nrows) p.out[(r0 + 1) * p.Q + k] = Y;
    }
  }
}

// Counts rows -> half spectra.  Counts are int64 in units of 2^-32; the unit
// is folded into the kernel spectrum, so they enter the transform unscaled.
template <typename T>
__global__ void __launch_bounds__(kThreads)
kde_rows_r2c_counts_kernel(const long long* __restrict__ counts, RowsParams<T> p) {
  using V = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  V* a = tw_s + p.P;
  V* b = a + p.G * p.P;
  load_twiddles<V, T>(tw_s, p.tw, p.P);
  const int64_t pair0 = (int64_t)blockIdx.x * p.G;
  for (int idx = threadIdx.x; idx < p.G * p.P; idx += blockDim.x) {
    int g = idx / p.P, x = idx - g * p.P;
    int64_t r0 = 2 * (pair0 + g);
    T re = 0, im = 0;
    if (x < p.Min && r0 < p.nrows) {
      re = (T)counts[r0 * p.in_stride + x];
      if (r0 + 1 < p.nrows) im = (T)counts[(r0 + 1) * p.in_stride + x];
    }
    a[idx] = mk<V>(re, im);
  }
  __syncthreads();
  V* z = fft_lines<V, false, true>(a, b, p.rp, p.G, 1, p.P, tw_s);
  for (int g = 0; g < p.G; ++g) {
    int64_t r0 = 2 * (pair0 + g);
    if (r0 < p.nrows) store_r2c<T>(p, z, r0, g);
  }
}

// Kernel-grid rows -> half spectra (or real spectrum for d = 1).  Row r
// enumerates the leading lags (l_0, ..., l_{d-2}) with |l_k| <= L_k; the last
// axis holds lag l at position l mod P.
template <typename T>
__global__ void __launch_bounds__(kThreads)
kde_rows_r2c_kgen_kernel(KGen<T> gen, RowsParams<T> p) {
  using V = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  V* a = tw_s + p.P;
  V* b = a + p.G * p.P;
  load_twiddles<V, T>(tw_s, p.tw, p.P);
  const int64_t pair0 = (int64_t)blockIdx.x * p.G;
  const int dl = gen.d - 1;  // index of the last axis
  for (int idx = threadIdx.x; idx < p.G * p.P; idx += blockDim.x) {
    int g = idx / p.P, x = idx - g * p.P;
    int64_t r0 = 2 * (pair0 + g);
    T val[2] = {0, 0};
    int ll = wrapped_lag(x, p.P, gen.L[dl]);
    if (ll <= gen.L[dl]) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int64_t r = r0 + h;
        if (r >= p.nrows) break;
        int l[KDE_MAX_D] = {0, 0, 0};
        if (gen.d == 2) {
          l[0] = (int)r - gen.L[0];
        } else if (gen.d == 3) {
          int w1 = 2 * gen.L[1] + 1;
          l[0] = (int)(r / w1) - gen.L[0];
          l[1] = (int)(r % w1) - gen.L[1];
        }
        l[dl] = ll;
        val[h] = kernel_value<T>(gen, l);
      }
    }
    a[idx] = mk<V>(val[0], val[1]);
  }
  __syncthreads();
  V* z = fft_lines<V, false, true>(a, b, p.rp, p.G, 1, p.P, tw_s);
  for (int g = 0; g < p.G; ++g) {
    int64_t r0 = 2 * (pair0 + g);
    if (r0 < p.nrows) store_r2c<T>(p, z, r0, g);
  }
}

template <typename T>
struct C2RParams {
  using V = typename Cplx<T>::type;
  const V* in;        // half spectra, row stride Q
  T* out;             // real rows, row stride Mout
  int64_t nrows;
  int Mout;
  int P, Q;
  int G;
  Radices rp;
  const V* tw;
};

// Half spectra -> real rows cropped to [0, Mout).  Z = X + i Y is rebuilt on
// the full length from Hermitian symmetry: Z_k = conj(X_{P-k}) + i conj(Y_{P-k})
// for k >= Q; then x + i y = F^{-1}(Z).
template <typename T>
__global__ void __launch_bounds__(kThreads) kde_rows_c2r_kernel(C2RParams<T> p) {
  using V = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  V* a = tw_s + p.P;
  V* b = a + p.G * p.P;
  load_twiddles<V, T>(tw_s, p.tw, p.P);
  const int64_t pair0 = (int64_t)blockIdx.x * p.G;
  for (int idx = threadIdx.x; idx < p.G * p.P; idx += blockDim.x) {
    int g = idx / p.P, k = idx - g * p.P;
    int64_t r0 = 2 * (pair0 + g);
    V z = mk<V>(0, 0);
    if (r0 < p.nrows) {
      bool lo_half = k < p.Q;
      int kk = lo_half ? k : p.P - k;
      V X = p.in[r0 * p.Q + kk];
      V Y = (r0 + 1 < p.nrows) ? p.in[(r0 + 1) * p.Q + kk] : mk<V>(0, 0);
      z = lo_half ? mk<V>(X.x - Y.y, X.y + Y.x) : mk<V>(X.x + Y.y, Y.x - X.y);
    }
    a[idx] = z;
  }
  __syncthreads();
  V* z = fft_lines<V, true, true>(a, b, p.rp, p.G, 1, p.P, tw_s);
  for (int idx = threadIdx.x; idx < p.G * p.Mout; idx += blockDim.x) {
    int g = idx / p.Mout, m = idx - g * p.Mout;
    int64_t r0 = 2 * (pair0 + g);
    if (r0 >= p.nrows) continue;
    V v = z[g * p.P + m];
    p.out[r0 * p.Mout + m] = v.x;
    if (r0 + 1 < p.nrows) p.out[(r0 + 1) * p.Mout + m] = v.y;
  }
}

// d = 1: counts -> F -> * K (real, even: K_k = K_{P-k}) -> F^{-1} -> crop.
template <typename T>
__global__ void __launch_bounds__(kThreads)
kde_line1d_kernel(const long long* __restrict__ counts, const T* __restrict__ K, T* out, int M,
                  int P, int Q, Radices rp, const typename Cplx<T>::type* tw) {
  using V = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  V* a = tw_s + P;
  V* b = a + P;
  load_twiddles<V, T>(tw_s, tw, P);
  for (int x = threadIdx.x; x < P; x += blockDim.x) a[x] = mk<V>(x < M ? (T)counts[x] : T(0), 0);
  __syncthreads();
  V* z = fft_lines<V, false, true>(a, b, rp, 1, 1, P, tw_s);
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    T kv = K[k < Q ? k : P - k];
    z[k] = mk<V>(z[k].x * kv, z[k].y * kv);
  }
  __syncthreads();
  V* other = (z == a) ? b : a;
  V* y = fft_lines<V, true, true>(z, other, rp, 1, 1, P, tw_s);
  for (int m = threadIdx.x; m < M; m += blockDim.x) out[m] = y[m].x;
}

enum ColMode { COL_FWD = 0, COL_FWD_REAL = 1, COL_MID = 2, COL_INV = 3 };

template <typename T>
struct ColsParams {
  using V = typename Cplx<T>::type;
  const V* in;     // [O][Nin][S]
  V* out;          // [O][Nout][S]
  T* out_real;     // COL_FWD_REAL: [O][P][S]
  const T* K;      // COL_MID: [P][S] real spectrum
  int64_t S;
  int Nin, Nout, P;
  int Lw;          // >= 0: input row n holds lag n - Lw (wrapped); < 0: row n at position n
  int Tc;          // columns per block
  Radices rp;
  const V* tw;
};

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) kde_cols_kernel(ColsParams<T> p) {
  using V = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  V* a = tw_s + p.P;
  V* b = a + p.Tc * p.P;
  load_twiddles<V, T>(tw_s, p.tw, p.P);
  const int64_t o = blockIdx.y;
  const int64_t s0 = (int64_t)blockIdx.x * p.Tc;
  const int Tc = p.Tc;
  const V* in = p.in + o * (int64_t)p.Nin * p.S;
  for (int idx = threadIdx.x; idx < p.P * Tc; idx += blockDim.x) {
    int pos = idx / Tc, t = idx - pos * Tc;
    int n;
    if (p.Lw >= 0) {
      int l = wrapped_lag(pos, p.P, p.Lw);
      n = (l <= p.Lw) ? l + p.Lw : p.Nin;
    } else {
      n = pos;
    }
    int64_t s = s0 + t;
    V v = mk<V>(0, 0);
    if (n < p.Nin && s < p.S) v = in[(int64_t)n * p.S + s];
    a[idx] = v;
  }
  __syncthreads();
  V* z;
  if (MODE == COL_INV) {
    z = fft_lines<V, true, false>(a, b, p.rp, Tc, Tc, 1, tw_s);
  } else {
    z = fft_lines<V, false, false>(a, b, p.rp, Tc, Tc, 1, tw_s);
  }
  if (MODE == COL_MID) {
    for (int idx = threadIdx.x; idx < p.P * Tc; idx += blockDim.x) {
      int pos = idx / Tc, t = idx - pos * Tc;
      int64_t s = s0 + t;
      T kv = (s < p.S) ? p.K[(int64_t)pos * p.S + s] : T(0);
      z[idx] = mk<V>(z[idx].x * kv, z[idx].y * kv);
    }
    __syncthreads();
    V* other = (z == a) ? b : a;
    z = fft_lines<V, true, false>(z, other, p.rp, Tc, Tc, 1, tw_s);
  }
  const int nout = (MODE == COL_FWD || MODE == COL_FWD_REAL) ? p.P : p.Nout;
  for (int idx = threadIdx.x; idx < nout * Tc; idx += blockDim.x) {
    int pos = idx / Tc, t = idx - pos * Tc;
    int64_t s = s0 + t;
    if (s >= p.S) continue;
    int64_t off = (o * nout + pos) * p.S + s;
    if (MODE == COL_FWD_REAL)
      p.out_real[off] = z[idx].x;
    else
      p.out[off] = z[idx];
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
constexpr size_t kSmemMax = 227 * 1024;

template <typename F>
cudaError_t allow_smem(F* fn) {
  static std::mutex mu;
  static std::set<const void*> done;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count((const void*)fn)) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
  if (e == cudaSuccess) done.insert((const void*)fn);
  return e;
}

Radices radices_of(const kde_plan_info& info, int k) {
  Radices r{};
  r.n = (int)info.P[k];
  r.nst = info.nstages[k];
  for (int s = 0; s < r.nst; ++s) r.r[s] = info.radix[k][s];
  return r;
}

template <typename T>
const typename Cplx<T>::type* twiddles(const kde_plan_s* plan, int k) {
  return reinterpret_cast<const typename Cplx<T>::type*>((const char*)plan->tw_dev + plan->tw_offset[k]);
}

static int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
  }
  return sms;
}

// Row pairs per block: enough lines to give the block work, few enough that
// the grid still covers every SM twice where possible, and within shared memory.
template <typename T>
int rows_per_block(int64_t pairs, int P) {
  size_t cb = sizeof(typename Cplx<T>::type);
  int g_smem = (int)((kSmemMax / cb - P) / (2 * (size_t)P));
  int g = (int)std::max<int64_t>(1, std::min<int64_t>(4096 / P, pairs / (2 * num_sms())));
  g = std::max(1, std::min(g, std::min(g_smem, 8)));
  return g;
}

template <typename T>
kde_status launch_rows_r2c_counts(const long long* counts, RowsParams<T> p, cudaStream_t st) {
  int64_t pairs = (p.nrows + 1) / 2;
  p.G = rows_per_block<T>(pairs, p.P);
  size_t smem = (size_t)(1 + 2 * p.G) * p.P * sizeof(typename Cplx<T>::type);
  auto* fn = kde_rows_r2c_counts_kernel<T>;
  cudaError_t e = allow_smem(fn);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  LaunchScope ls("kde_rows_r2c_counts_kernel", st);
  fn<<<(unsigned)((pairs + p.G - 1) / p.G), kThreads, smem, st>>>(counts, p);
  e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_rows_r2c_counts_kernel");
}

template <typename T>
kde_status launch_rows_r2c_kgen(const KGen<T>& gen, RowsParams<T> p, cudaStream_t st) {
  int64_t pairs = (p.nrows + 1) / 2;
  p.G = rows_per_block<T>(pairs, p.P);
  size_t smem = (size_t)(1 + 2 * p.G) * p.P * sizeof(typename Cplx<T>::type);
  auto* fn = kde_rows_r2c_kgen_kernel<T>;
  cudaError_t e = allow_smem(fn);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  LaunchScope ls("kde_rows_r2c_kgen_kernel", st);
  fn<<<(unsigned)((pairs + p.G - 1) / p.G), kThreads, smem, st>>>(gen, p);
  e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_rows_r2c_kgen_kernel");
}

template <typename T>
kde_status launch_rows_c2r(C2RParams<T> p, cudaStream_t st) {
  int64_t pairs = (p.nrows + 1) / 2;
  p.G = rows_per_block<T>(pairs, p.P);
  size_t smem = (size_t)(1 + 2 * p.G) * p.P * sizeof(typename Cplx<T>::type);
  auto* fn = kde_rows_c2r_kernel<T>;
  cudaError_t e = allow_smem(fn);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  LaunchScope ls("kde_rows_c2r_kernel", st);
  fn<<<(unsigned)((pairs + p.G - 1) / p.G), kThreads, smem, st>>>(p);
  e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_rows_c2r_kernel");
}

template <typename T, int MODE>
kde_status launch_cols(ColsParams<T> p, int64_t O, cudaStream_t st, const char* name) {
  size_t cb = sizeof(typename Cplx<T>::type);
  // Columns per block: a 32-byte run of each row per tile (4 complex64 or 2
  // complex128), fewer if shared memory is short.
  int Tc = (int)(32 / cb);
  while (Tc > 1 && (size_t)(1 + 2 * Tc) * p.P * cb > kSmemMax) Tc /= 2;
  p.Tc = Tc;
  size_t smem = (size_t)(1 + 2 * Tc) * p.P * cb;
  auto* fn = kde_cols_kernel<T, MODE>;
  cudaError_t e = allow_smem(fn);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  dim3 grid((unsigned)((p.S + Tc - 1) / Tc), (unsigned)O);
  LaunchScope ls(name, st);
  fn<<<grid, kThreads, smem, st>>>(p);
  e = cudaGetLastError();
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, name);
}

template <typename T>
kde_status kernel_grid_impl(kde_plan_s* plan, int64_t n, void* Kspec, void* ws, cudaStream_t st) {
  using V = typename Cplx<T>::type;
  const kde_plan_info& I = plan->info;
  const int d = I.d;
  KGen<T> gen{};
  gen.d = d;
  gen.wand = plan->layout_mode == KDE_LAYOUT_WAND;
  double prodP = 1.0;
  for (int k = 0; k < d; ++k) {
    gen.L[k] = (int)I.L[k];
    prodP *= (double)I.P[k];
  }
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) gen.A[a][b] = (T)(I.delta[a] * I.delta[b] * plan->Hinv[a * d + b]);
  const double two_pi = 6.283185307179586476925287;
  double C = std::pow(two_pi, -0.5 * d) / std::sqrt(I.det_H) / ((double)n * 4294967296.0 * prodP);
  gen.C = (T)C;
  const int dl = d - 1;
  RowsParams<T> rp{};
  rp.P = (int)I.P[dl];
  rp.Q = (int)I.Q;
  rp.Min = 0;
  rp.rp = radices_of(I, dl);
  rp.tw = twiddles<T>(plan, dl);
  if (d == 1) {
    rp.nrows = 1;
    rp.out_real = (T*)Kspec;
    return launch_rows_r2c_kgen<T>(gen, rp, st);
  }
  V* t1 = (V*)ws;
  int64_t rows = 1;
  for (int k = 0; k < d - 1; ++k) rows *= 2 * I.L[k] + 1;
  rp.nrows = rows;
  rp.out = t1;
  kde_status s = launch_rows_r2c_kgen<T>(gen, rp, st);
  if (s != KDE_OK) return s;
  if (d == 2) {
    ColsParams<T> cp{};
    cp.in = t1;
    cp.out_real = (T*)Kspec;
    cp.S = I.Q;
    cp.Nin = (int)(2 * I.L[0] + 1);
    cp.P = (int)I.P[0];
    cp.Lw = (int)I.L[0];
    cp.rp = radices_of(I, 0);
    cp.tw = twiddles<T>(plan, 0);
    return launch_cols<T, COL_FWD_REAL>(cp, 1, st, "kde_cols_kgen_real_kernel");
  }
  // d == 3: axis 1 (wrapped) into t2, then axis 0 (wrapped) to the real spectrum.
  V* t2 = t1 + rows * I.Q;
  ColsParams<T> c1{};
  c1.in = t1;
  c1.out = t2;
  c1.S = I.Q;
  c1.Nin = (int)(2 * I.L[1] + 1);
  c1.P = (int)I.P[1];
  c1.Lw = (int)I.L[1];
  c1.rp = radices_of(I, 1);
  c1.tw = twiddles<T>(plan, 1);
  s = launch_cols<T, COL_FWD>(c1, 2 * I.L[0] + 1, st, "kde_cols_kgen_kernel");
  if (s != KDE_OK) return s;
  ColsParams<T> c0{};
  c0.in = t2;
  c0.out_real = (T*)Kspec;
  c0.S = I.P[1] * I.Q;
  c0.Nin = (int)(2 * I.L[0] + 1);
  c0.P = (int)I.P[0];
  c0.Lw = (int)I.L[0];
  c0.rp = radices_of(I, 0);
  c0.tw = twiddles<T>(plan, 0);
  return launch_cols<T, COL_FWD_REAL>(c0, 1, st, "kde_cols_kgen_real_kernel");
}

template <typename T>
kde_status fft_eval_impl(kde_plan_s* plan, const int64_t* counts, const void* Kspec, void* density,
                         void* ws, cudaStream_t st) {
  using V = typename Cplx<T>::type;
  const kde_plan_info& I = plan->info;
  const int d = I.d;
  const int dl = d - 1;
  const long long* cnt = reinterpret_cast<const long long*>(counts);
  if (d == 1) {
    size_t smem = (size_t)3 * I.P[0] * sizeof(V);
    auto* fn = kde_line1d_kernel<T>;
    cudaError_t e = allow_smem(fn);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    LaunchScope ls("kde_line1d_kernel", st);
    fn<<<1, kThreads, smem, st>>>(cnt, (const T*)Kspec, (T*)density, (int)I.M[0], (int)I.P[0],
                                  (int)I.Q, radices_of(I, 0), twiddles<T>(plan, 0));
    e = cudaGetLastError();
    return e == cudaSuccess ? KDE_OK : cuda_fail(e, "kde_line1d_kernel");
  }
  V* A = (V*)ws;  // [M_0 .. M_{d-2}][Q]
  int64_t rows = 1;
  for (int k = 0; k < d - 1; ++k) rows *= I.M[k];
  RowsParams<T> rp{};
  rp.nrows = rows;
  rp.Min = (int)I.M[dl];
  rp.in_stride = I.M[dl];
  rp.P = (int)I.P[dl];
  rp.Q = (int)I.Q;
  rp.out = A;
  rp.rp = radices_of(I, dl);
  rp.tw = twiddles<T>(plan, dl);
  kde_status s = launch_rows_r2c_counts<T>(cnt, rp, st);
  if (s != KDE_OK) return s;
  if (d == 2) {
    ColsParams<T> cp{};
    cp.in = A;
    cp.out = A;
    cp.K = (const T*)Kspec;
    cp.S = I.Q;
    cp.Nin = (int)I.M[0];
    cp.Nout = (int)I.M[0];
    cp.P = (int)I.P[0];
    cp.Lw = -1;
    cp.rp = radices_of(I, 0);
    cp.tw = twiddles<T>(plan, 0);
    s = launch_cols<T, COL_MID>(cp, 1, st, "kde_cols_mid_kernel");
    if (s != KDE_OK) return s;
  } else {
    V* B = A + rows * I.Q;  // [M_0][P_1][Q]
    ColsParams<T> c1{};
    c1.in = A;
    c1.out = B;
    c1.S = I.Q;
    c1.Nin = (int)I.M[1];
    c1.P = (int)I.P[1];
    c1.Lw = -1;
    c1.rp = radices_of(I, 1);
    c1.tw = twiddles<T>(plan, 1);
    s = launch_cols<T, COL_FWD>(c1, I.M[0], st, "kde_cols_fwd_kernel");
    if (s != KDE_OK) return s;
    ColsParams<T> c0{};
    c0.in = B;
    c0.out = B;
    c0.K = (const T*)Kspec;
    c0.S = I.P[1] * I.Q;
    c0.Nin = (int)I.M[0];
    c0.Nout = (int)I.M[0];
    c0.P = (int)I.P[0];
    c0.Lw = -1;
    c0.rp = radices_of(I, 0);
    c0.tw = twiddles<T>(plan, 0);
    s = launch_cols<T, COL_MID>(c0, 1, st, "kde_cols_mid_kernel");
    if (s != KDE_OK) return s;
    ColsParams<T> ci{};
    ci.in = B;
    ci.out = A;
    ci.S = I.Q;
    ci.Nin = (int)I.P[1];
    ci.Nout = (int)I.M[1];
    ci.P = (int)I.P[1];
    ci.Lw = -1;
    ci.rp = radices_of(I, 1);
    ci.tw = twiddles<T>(plan, 1);
    s = launch_cols<T, COL_INV>(ci, I.M[0], st, "kde_cols_inv_kernel");
    if (s != KDE_OK) return s;
  }
  C2RParams<T> cr{};
  cr.in = A;
  cr.out = (T*)density;
  cr.nrows = rows;
  cr.Mout = (int)I.M[dl];
  cr.P = (int)I.P[dl];
  cr.Q = (int)I.Q;
  cr.rp = radices_of(I, dl);
  cr.tw = twiddles<T>(plan, dl);
  return launch_rows_c2r<T>(cr, st);
}

kde_status check_ws(const kde_plan_s* plan, void* ws, size_t bytes) {
  if (plan->info.workspace_bytes == 0) return KDE_OK;
  if (!ws) return fail(KDE_ERR_WORKSPACE, "workspace is NULL");
  if (bytes < plan->info.workspace_bytes) return fail(KDE_ERR_WORKSPACE, "workspace too small");
  if (((uintptr_t)ws & 15) != 0) return fail(KDE_ERR_INVALID_ARG, "workspace not 16-byte aligned");
  return KDE_OK;
}

kde_status check_device(const kde_plan_s* plan) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != plan->device) return fail(KDE_ERR_INVALID_ARG, "plan was made on another device");
  return KDE_OK;
}

}  // namespace
}  // namespace kde

using namespace kde;

extern "C" kde_status kde_kernel_grid(kde_plan plan, int64_t n, void* Kspec, void* workspace,
                                      size_t workspace_bytes, kde_stream_t stream) {
  if (!plan || !Kspec) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (n < 1) return fail(KDE_ERR_INVALID_ARG, "n must be >= 1 (the 1/n of Eq. 2)");
  kde_status s = check_ws(plan, workspace, workspace_bytes);
  if (s != KDE_OK) return s;
  if ((s = check_device(plan)) != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->info.precision == KDE_F32) return kernel_grid_impl<float>(plan, n, Kspec, workspace, st);
  return kernel_grid_impl<double>(plan, n, Kspec, workspace, st);
}

extern "C" kde_status kde_fft_eval(kde_plan plan, const int64_t* counts, const void* Kspec,
                                   void* density, void* workspace, size_t workspace_bytes,
                                   kde_stream_t stream) {
  if (!plan || !counts || !Kspec || !density) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  kde_status s = check_ws(plan, workspace, workspace_bytes);
  if (s != KDE_OK) return s;
  if ((s = check_device(plan)) != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->info.precision == KDE_F32)
    return fft_eval_impl<float>(plan, counts, Kspec, density, workspace, st);
  return fft_eval_impl<double>(plan, counts, Kspec, density, workspace, st);
}

// ---------------------------------------------------------------------------
// kde_fft_eval_noalloc: kde_fft_eval with its scratch in a fixed device array
// instead of a caller-provided workspace, for callers that cannot allocate
// device memory at the point of the call (for example code running inside a
// framework that owns every allocation, or a real-time loop that must not
// enter the allocator).  Its size is fixed at build time and the array lives
// on every device that loads this library until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // KDE_NOALLOC_SCRATCH_BYTES
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol's name is only a host-side handle, so the address is looked up
// once per device with that device current and cached.
kde_status noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(KDE_ERR_UNSUPPORTED, "device ordinal too large");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return KDE_OK;
}

}  // namespace

extern "C" kde_status kde_fft_eval_noalloc(kde_plan plan, const int64_t* counts, const void* Kspec,
                                           void* density, kde_stream_t stream) {
  if (!plan || !counts || !Kspec || !density) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  if (plan->info.workspace_bytes > kNoAllocScratchBytes)
    return fail(KDE_ERR_WORKSPACE,
                "kde_fft_eval_noalloc: the plan needs " + std::to_string(plan->info.workspace_bytes) +
                    " bytes of scratch, above the fixed " + std::to_string(kNoAllocScratchBytes) +
                    "; use kde_fft_eval with a workspace");
  kde_status s = check_device(plan);
  if (s != KDE_OK) return s;
  void* scratch = nullptr;
  if ((s = noalloc_scratch(plan->device, &scratch)) != KDE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->info.precision == KDE_F32)
    return fft_eval_impl<float>(plan, counts, Kspec, density, scratch, st);
  return fft_eval_impl<double>(plan, counts, Kspec, density, scratch, st);
}
