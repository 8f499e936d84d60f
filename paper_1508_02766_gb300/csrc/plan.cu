// Host-side planning (FP64): problem checks, Cholesky factor, inverse and
// determinant of H, its largest eigenvalue, the effective support L (Eq. 15),
// the padded sizes P and their radix plans; plus plan lifetime, device
// twiddle tables, error reporting, launch counting and per-kernel timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fx_pairs.h"
#include "kde_debug.cuh"
#include "kde_internal.h"

namespace kde {

static thread_local std::string g_last_error;

kde_status fail(kde_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

kde_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return KDE_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Small host-to-device uploads of call arguments (offsets, sample counts,
// per-candidate parameters) through page-locked staging slots, so that the
// copy is asynchronous: a copy from pageable memory may wait for the stream,
// which would stop the host from enqueueing the next batch while the GPU
// works on this one.  Each thread keeps, per device, a ring of slots; a slot
// is refilled only after the event recorded behind its last copy completed.
// ---------------------------------------------------------------------------
namespace {
struct UploadSlot {
  void* host = nullptr;
  size_t cap = 0;
  cudaEvent_t ev = nullptr;
  bool pending = false;
};
constexpr int kUploadSlots = 8;
constexpr int kUploadDevices = 64;
struct UploadRing {
  UploadSlot slot[kUploadSlots];
  int next = 0;
};
thread_local UploadRing g_upload[kUploadDevices];
}  // namespace

kde_status upload_async(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return KDE_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kUploadDevices) {   // no ring: a plain (possibly waiting) copy
    e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    return e == cudaSuccess ? KDE_OK : cuda_fail(e, "cudaMemcpyAsync(upload)");
  }
  UploadRing& r = g_upload[dev];
  UploadSlot& sl = r.slot[r.next];
  r.next = (r.next + 1) % kUploadSlots;
  if (sl.pending) {
    if ((e = cudaEventSynchronize(sl.ev)) != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize(upload)");
    sl.pending = false;
  }
  if (!sl.ev && (e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "cudaEventCreate(upload)");
  if (sl.cap < bytes) {
    if (sl.host) cudaFreeHost(sl.host);
    sl.host = nullptr;
    sl.cap = 0;
    const size_t cap = std::max<size_t>(bytes, 64 << 10);
    if ((e = cudaHostAlloc(&sl.host, cap, cudaHostAllocPortable)) != cudaSuccess)
      return cuda_fail(e, "cudaHostAlloc(upload)");
    sl.cap = cap;
  }
  std::memcpy(sl.host, src, bytes);
  if ((e = cudaMemcpyAsync(dst, sl.host, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync(upload)");
  if ((e = cudaEventRecord(sl.ev, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord(upload)");
  sl.pending = true;
  return KDE_OK;
}

// ---------------------------------------------------------------------------
// Launch counting and per-kernel event timing.
// ---------------------------------------------------------------------------
static std::atomic<int64_t> g_launches{0};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
struct ProfRec {
  const char* name;
  cudaEvent_t start, stop;
};
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_event_pool;

static cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Every launch is also an NVTX range named after its kernel (host side,
// around the launch call), visible to Nsight tools when one is attached;
// without a tool the calls return at once.
LaunchScope::LaunchScope(const char* name, cudaStream_t s) : slot(-1), stream(s) {
  nvtxRangePushA(name);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return;
  ProfRec r{name, take_event(), take_event()};
  if (!r.start || !r.stop) return;
  cudaEventRecord(r.start, s);
  slot = (int)g_prof.size();
  g_prof.push_back(r);
}

LaunchScope::~LaunchScope() {
  nvtxRangePop();
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEventRecord(g_prof[slot].stop, stream);
}

// ---------------------------------------------------------------------------
// Linear algebra on d <= 3 (FP64).
// ---------------------------------------------------------------------------
static bool cholesky(int d, const double* H, double* R) {  // H = R R^T, R lower
  for (int i = 0; i < 9; ++i) R[i] = 0.0;
  for (int j = 0; j < d; ++j) {
    double s = H[j * d + j];
    for (int k = 0; k < j; ++k) s -= R[j * 3 + k] * R[j * 3 + k];
    if (!(s > 0.0)) return false;
    double rjj = std::sqrt(s);
    R[j * 3 + j] = rjj;
    for (int i = j + 1; i < d; ++i) {
      double t = H[i * d + j];
      for (int k = 0; k < j; ++k) t -= R[i * 3 + k] * R[j * 3 + k];
      R[i * 3 + j] = t / rjj;
    }
  }
  return true;
}

static void spd_inverse(int d, const double* R, double* Hinv) {  // from H = R R^T
  double Rinv[9] = {0};
  for (int j = 0; j < d; ++j) {
    Rinv[j * 3 + j] = 1.0 / R[j * 3 + j];
    for (int i = j + 1; i < d; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s += R[i * 3 + k] * Rinv[k * 3 + j];
      Rinv[i * 3 + j] = -s / R[i * 3 + i];
    }
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += Rinv[k * 3 + i] * Rinv[k * 3 + j];  // R^-T R^-1
      Hinv[i * d + j] = s;
    }
}

// Exponent of K_A at lag l on bins of width delta, in completed squares:
// with A = R R^T (Cholesky) and y = R^-1 (delta o l), (delta o l)^T A^-1
// (delta o l) = |y|^2 and y_k = (R^-1)_kk delta_k (l_k + sum_{j<k} B_kj l_j),
//   -q/2 = sum_k D_k (l_k + sum_{j<k} B_kj l_j)^2,
//   D_k = -delta_k^2 / (2 R_kk^2),  B_kj = (R^-1)_kj delta_j / ((R^-1)_kk delta_k).
// B[0] = B_10, B[1] = B_20, B[2] = B_21.
kde_status gauss_factor(int d, const double* A, const double* delta, double* D, double* B) {
  double R[9];
  if (!cholesky(d, A, R)) return fail(KDE_ERR_NOT_SPD, "bandwidth is not positive definite");
  double Rinv[9] = {0};
  for (int j = 0; j < d; ++j) {
    Rinv[j * 3 + j] = 1.0 / R[j * 3 + j];
    for (int i = j + 1; i < d; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s += R[i * 3 + k] * Rinv[k * 3 + j];
      Rinv[i * 3 + j] = -s / R[i * 3 + i];
    }
  }
  for (int k = 0; k < 3; ++k) {
    D[k] = 0.0;
    B[k] = 0.0;
  }
  for (int k = 0; k < d; ++k) D[k] = -0.5 * delta[k] * delta[k] * Rinv[k * 3 + k] * Rinv[k * 3 + k];
  const int kj[3][2] = {{1, 0}, {2, 0}, {2, 1}};
  for (int e = 0; e < 3; ++e) {
    const int k = kj[e][0], j = kj[e][1];
    if (k < d) B[e] = Rinv[k * 3 + j] * delta[j] / (Rinv[k * 3 + k] * delta[k]);
  }
  return KDE_OK;
}

// Largest eigenvalue of a symmetric d x d matrix: closed form for d <= 2,
// cyclic Jacobi rotations for d = 3.
static double lambda_max(int d, const double* H) {
  if (d == 1) return H[0];
  if (d == 2) {
    double a = H[0], b = H[1], c = H[3];
    double m = 0.5 * (a + c), h = 0.5 * (a - c);
    return m + std::sqrt(h * h + b * b);
  }
  double A[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[i][j] = H[i * 3 + j];
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    double diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-36 * diag) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 3; ++k) {  // A <- A J
          double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  // A <- J^T A
          double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
      }
  }
  return std::fmax(A[0][0], std::fmax(A[1][1], A[2][2]));
}

static bool is_7smooth(int64_t x) {
  for (int p : {2, 3, 5, 7})
    while (x % p == 0) x /= p;
  return x == 1;
}

// Two-phase engine: a line length and its split.  Up to 400 the generic
// kernels take any P = N1 N2 with 2 <= N1 <= N2 <= 20, both 7-smooth (the
// most balanced split, smallest N2), unless a split with kernels of its own
// (fx_pairs.h) is at most 10% longer; longer lines take the smallest listed
// three-factor length.  Returns the length >= need and its factors (N3 = 0
// for two), or 0 if there is none.
static int64_t two_phase_plan(int64_t need, int* sp) {
  int64_t best_c = 0;
  int c[3] = {0, 0, 0};
  for (int i = 0; i < fxp::kNumPairs; ++i) {
    const int64_t P = (int64_t)fxp::kPairs[i].N1 * fxp::kPairs[i].N2;
    if (P >= need && (best_c == 0 || P < best_c)) {
      best_c = P;
      c[0] = fxp::kPairs[i].N1;
      c[1] = fxp::kPairs[i].N2;
      c[2] = 0;
    }
  }
  for (int64_t P = need; P <= fxp::kGenericMaxP; ++P) {
    int a_best = 0;
    for (int a = 2; a * a <= P; ++a) {
      if (P % a) continue;
      const int64_t b = P / a;
      if (b > fxp::kGenericMax || !is_7smooth(a) || !is_7smooth(b)) continue;
      a_best = a;  // later a are larger, so b is smaller: more balanced
    }
    if (!a_best) continue;
    if (best_c && (double)best_c <= 1.1 * (double)P) break;  // the compiled split
    sp[0] = a_best;
    sp[1] = (int)(P / a_best);
    sp[2] = 0;
    return P;
  }
  if (!best_c) {
    for (int i = 0; i < fxp::kNumTriples; ++i) {
      const fxp::Triple& t = fxp::kTriples[i];
      const int64_t P = (int64_t)t.N1 * t.N2 * t.N3;
      if (P >= need && (best_c == 0 || P < best_c)) {
        best_c = P;
        c[0] = t.N1;
        c[1] = t.N2;
        c[2] = t.N3;
      }
    }
  }
  for (int i = 0; i < 3; ++i) sp[i] = c[i];
  return best_c;
}

// Factor P into the engine's radices with the fewest stages (then the
// fewest odd radices), largest radix first.  Dynamic programming over the
// divisors of P.
static int radix_plan(int64_t P, int* radix) {
  static const int kRadices[] = {8, 7, 5, 4, 3, 2};
  std::vector<int> best_n(P + 1, 1 << 20), best_odd(P + 1, 1 << 20), choice(P + 1, 0);
  best_n[1] = 0;
  best_odd[1] = 0;
  for (int64_t x = 2; x <= P; ++x) {
    if (P % x) continue;
    for (int r : kRadices) {
      if (x % r) continue;
      int64_t y = x / r;
      if (best_n[y] >= (1 << 20)) continue;
      int n = best_n[y] + 1, odd = best_odd[y] + (r % 2);
      if (n < best_n[x] || (n == best_n[x] && odd < best_odd[x])) {
        best_n[x] = n;
        best_odd[x] = odd;
        choice[x] = r;
      }
    }
  }
  int n = 0;
  for (int64_t x = P; x > 1; x /= choice[x]) radix[n++] = choice[x];
  std::sort(radix, radix + n, [](int a, int b) { return a > b; });
  return n;
}

// Factors of a bandwidth matrix A evaluated under an existing plan: A^-1,
// |A| and the support L (Eq. 15 with the plan's tau and range mode).  Fails
// if A is not symmetric positive definite or needs more padding than the
// plan has (M_k + L_k > P_k).
kde_status matrix_support(const kde_plan_s* plan, const double* A, double* Ainv, double* detA,
                          int64_t* L) {
  const kde_plan_info& I = plan->info;
  const int d = I.d;
  double amax = 0.0;
  for (int i = 0; i < d * d; ++i) {
    if (!std::isfinite(A[i])) return fail(KDE_ERR_INVALID_ARG, "bandwidth has a non-finite entry");
    amax = std::fmax(amax, std::fabs(A[i]));
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < i; ++j)
      if (std::fabs(A[i * d + j] - A[j * d + i]) > 1e-12 * amax)
        return fail(KDE_ERR_INVALID_ARG, "bandwidth is not symmetric");
  double R[9];
  if (!cholesky(d, A, R)) return fail(KDE_ERR_NOT_SPD, "bandwidth is not positive definite");
  double det = 1.0;
  for (int i = 0; i < d; ++i) det *= R[i * 3 + i] * R[i * 3 + i];
  *detA = det;
  spd_inverse(d, R, Ainv);
  const double lam = lambda_max(d, A);
  for (int k = 0; k < d; ++k) {
    const double half = (plan->range_mode == KDE_RANGE_CORRECTED)
                            ? plan->tau * std::sqrt(std::fabs(lam))
                            : plan->tau * std::sqrt(A[k * d + k]);
    const double c = std::ceil(half / I.delta[k]);
    L[k] = (c >= (double)(I.M[k] - 1)) ? I.M[k] - 1 : (int64_t)c;
    if (I.M[k] + L[k] > I.P[k])
      return fail(KDE_ERR_INVALID_ARG, "bandwidth needs more padding than the plan has (raise P_min)");
  }
  return KDE_OK;
}

}  // namespace kde

using namespace kde;

static kde_status compute_info(int d, const int64_t* M, const double* lo, const double* hi,
                               const double* H, const kde_opts* opts, kde_plan_info* info,
                               double* Hinv_out, double* tau_out) {
  if (!info) return fail(KDE_ERR_INVALID_ARG, "info is NULL");
  if (d < 1 || d > KDE_MAX_D) return fail(KDE_ERR_UNSUPPORTED, "d must be 1, 2 or 3");
  if (!M || !lo || !hi || !H) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  kde_opts o{};
  o.tau = 3.7;
  if (opts) o = *opts;
  if (!(o.tau > 0.0)) o.tau = 3.7;
  if (!std::isfinite(o.tau)) return fail(KDE_ERR_INVALID_ARG, "tau must be finite");
  if (o.precision != KDE_F32 && o.precision != KDE_F64)
    return fail(KDE_ERR_INVALID_ARG, "precision must be KDE_F32 or KDE_F64");
  if (o.range_mode != KDE_RANGE_CORRECTED && o.range_mode != KDE_RANGE_PER_AXIS)
    return fail(KDE_ERR_INVALID_ARG, "bad range_mode");
  if (o.layout_mode != KDE_LAYOUT_CORRECTED && o.layout_mode != KDE_LAYOUT_WAND)
    return fail(KDE_ERR_INVALID_ARG, "bad layout_mode");
  if (o.cols_variant < KDE_COLS_AUTO || o.cols_variant > KDE_COLS_SIMD)
    return fail(KDE_ERR_INVALID_ARG, "bad cols_variant");
  std::memset(info, 0, sizeof(*info));
  info->d = d;
  info->precision = o.precision;
  double hmax = 0.0;
  for (int i = 0; i < d * d; ++i) {
    if (!std::isfinite(H[i])) return fail(KDE_ERR_INVALID_ARG, "H has a non-finite entry");
    hmax = std::fmax(hmax, std::fabs(H[i]));
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < i; ++j)
      if (std::fabs(H[i * d + j] - H[j * d + i]) > 1e-12 * hmax)
        return fail(KDE_ERR_INVALID_ARG, "H is not symmetric");
  double R[9];
  if (!cholesky(d, H, R)) return fail(KDE_ERR_NOT_SPD, "H is not positive definite");
  double det = 1.0;
  for (int i = 0; i < d; ++i) det *= R[i * 3 + i] * R[i * 3 + i];
  info->det_H = det;
  spd_inverse(d, R, Hinv_out);
  info->lambda_max = lambda_max(d, H);
  for (int k = 0; k < d; ++k) {
    if (M[k] < 2) return fail(KDE_ERR_INVALID_ARG, "every M_k must be >= 2");
    if (!std::isfinite(lo[k]) || !std::isfinite(hi[k]) || !(lo[k] < hi[k]))
      return fail(KDE_ERR_INVALID_ARG, "need finite lo[k] < hi[k]");
    info->M[k] = M[k];
    info->delta[k] = (hi[k] - lo[k]) / (double)(M[k] - 1);  // Eq. 4
    double half = (o.range_mode == KDE_RANGE_CORRECTED)
                      ? o.tau * std::sqrt(std::fabs(info->lambda_max))  // Eq. 15
                      : o.tau * std::sqrt(H[k * d + k]);
    double c = std::ceil(half / info->delta[k]);
    int64_t L = (c >= (double)(M[k] - 1)) ? M[k] - 1 : (int64_t)c;
    info->L[k] = L;
    int64_t need = M[k] + L;
    if (o.P_min[k] > need) need = o.P_min[k];
    if (need > KDE_MAX_P) return fail(KDE_ERR_UNSUPPORTED, "padded size above KDE_MAX_P");
    info->P[k] = need;
  }
  // Engine and padded sizes.  The two-phase engine takes the smallest
  // product N1 N2 >= M_k + L_k per axis; the Stockham engine the smallest
  // 7-smooth size.  Either is a valid P (Eq. 10 needs only P_k >= M_k + L_k).
  if (o.engine < KDE_ENGINE_AUTO || o.engine > KDE_ENGINE_TWO_PHASE)
    return fail(KDE_ERR_INVALID_ARG, "bad engine");
  const bool tp_ok = o.precision == KDE_F32 && d >= 2;
  if (o.engine == KDE_ENGINE_TWO_PHASE && !tp_ok)
    return fail(KDE_ERR_UNSUPPORTED, "the two-phase engine needs a KDE_F32 plan with d >= 2");
  bool tp = tp_ok && o.engine != KDE_ENGINE_STOCKHAM;
  int64_t Ptp[KDE_MAX_D] = {0, 0, 0};
  int sp[KDE_MAX_D][3] = {};
  for (int k = 0; tp && k < d; ++k) {
    const int64_t P = two_phase_plan(info->P[k], sp[k]);
    if (P == 0) {
      if (o.engine == KDE_ENGINE_TWO_PHASE)
        return fail(KDE_ERR_UNSUPPORTED, "padded size above the two-phase engine's largest line");
      tp = false;
    }
    Ptp[k] = P;
  }
  info->engine = tp ? KDE_ENGINE_TWO_PHASE : KDE_ENGINE_STOCKHAM;
  for (int k = 0; k < d; ++k) {
    int64_t P = info->P[k];
    if (tp) {
      P = Ptp[k];
      for (int i = 0; i < 3; ++i) info->split[k][i] = sp[k][i];
    } else {
      while (!is_7smooth(P)) ++P;
    }
    if (P > KDE_MAX_P) return fail(KDE_ERR_UNSUPPORTED, "padded size above KDE_MAX_P");
    info->P[k] = P;
    info->nstages[k] = radix_plan(P, info->radix[k]);
  }
  info->Q = info->P[d - 1] / 2 + 1;
  if (o.slab_passes != KDE_SLAB_OFF && o.slab_passes != KDE_SLAB_ON)
    return fail(KDE_ERR_INVALID_ARG, "bad slab_passes");
  if (d == 3 && tp && !o.dft_tc && o.slab_passes == KDE_SLAB_ON)
    info->slab_passes = kde::fxp::slab_geometry(M[1], info->Q, info->split[2], info->split[1]).ok;
  int64_t ke = info->Q;
  for (int k = 0; k < d - 1; ++k) ke *= info->P[k];
  info->kspec_elems = ke;
  size_t real_b = (o.precision == KDE_F32) ? 4 : 8;
  info->kspec_bytes = (size_t)ke * real_b;
  // Scratch (complex elements): evaluation and kernel-grid intermediates.
  int64_t Q = info->Q, ev = 0, kg = 0;
  if (d == 1) {
    ev = Q;  // the half spectrum of the count spectrum (kde_power_spectrum)
  } else if (d == 2) {
    ev = M[0] * Q;
    kg = (2 * info->L[0] + 1) * Q;
  } else if (d == 3) {
    ev = M[0] * M[1] * Q + M[0] * info->P[1] * Q;
    kg = (2 * info->L[0] + 1) * (2 * info->L[1] + 1) * Q + (2 * info->L[0] + 1) * info->P[1] * Q;
  }
  int64_t ws = ev > kg ? ev : kg;
  info->workspace_bytes = (size_t)ws * 2 * real_b;
  *tau_out = o.tau;
  return KDE_OK;
}

template <typename T2, typename T>
__global__ void kde_twiddle_kernel(T2* tw, int P) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= P) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)P, &s, &c);  // e^{-2 pi i m / P}
  tw[m].x = (T)c;
  tw[m].y = (T)(-s);
}

extern "C" {

kde_status kde_plan_info_compute(int d, const int64_t* M, const double* lo, const double* hi,
                                 const double* H, const kde_opts* opts, kde_plan_info* info) {
  double Hinv[9], tau;
  return compute_info(d, M, lo, hi, H, opts, info, Hinv, &tau);
}

kde_status kde_plan_create(int d, const int64_t* M, const double* lo, const double* hi,
                           const double* H, const kde_opts* opts, kde_plan* out) {
  if (!out) return fail(KDE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  kde_plan_s* p = new (std::nothrow) kde_plan_s();
  if (!p) return fail(KDE_ERR_INVALID_ARG, "out of host memory");
  kde_status st = compute_info(d, M, lo, hi, H, opts, &p->info, p->Hinv, &p->tau);
  if (st != KDE_OK) {
    delete p;
    return st;
  }
  for (int i = 0; i < d * d; ++i) p->H[i] = H[i];
  for (int k = 0; k < d; ++k) {
    p->lo[k] = lo[k];
    p->hi[k] = hi[k];
  }
  p->range_mode = opts ? opts->range_mode : KDE_RANGE_CORRECTED;
  p->layout_mode = opts ? opts->layout_mode : KDE_LAYOUT_CORRECTED;
  p->cols_variant = opts ? opts->cols_variant : KDE_COLS_AUTO;
  p->dft_tc = opts ? opts->dft_tc : 0;
  if (p->dft_tc && (p->info.precision != KDE_F32 || d < 2)) {
    delete p;
    return fail(KDE_ERR_UNSUPPORTED, "dft_tc needs a KDE_F32 plan with d >= 2");
  }
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaGetDevice");
  }
  size_t cb = (p->info.precision == KDE_F32) ? sizeof(float2) : sizeof(double2);
  size_t total = 0;
  for (int k = 0; k < d; ++k) {
    p->tw_offset[k] = total;
    total += ((size_t)p->info.P[k] * cb + 255) & ~(size_t)255;
  }
  e = cudaMalloc(&p->tw_dev, total + 256);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaMalloc(twiddles)");
  }
  p->status_dev = (int*)((char*)p->tw_dev + total);
  e = cudaMemset(p->status_dev, 0, 256);
  if (e != cudaSuccess) {
    cudaFree(p->tw_dev);
    delete p;
    return cuda_fail(e, "cudaMemset(status)");
  }
  for (int k = 0; k < d; ++k) {
    int P = (int)p->info.P[k];
    char* base = (char*)p->tw_dev + p->tw_offset[k];
    {
      LaunchScope ls("kde_twiddle_kernel", 0);
      if (p->info.precision == KDE_F32)
        kde_twiddle_kernel<float2, float><<<(P + 255) / 256, 256>>>((float2*)base, P);
      else
        kde_twiddle_kernel<double2, double><<<(P + 255) / 256, 256>>>((double2*)base, P);
    }
  }
  e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFree(p->tw_dev);
    delete p;
    return cuda_fail(e, "twiddle generation");
  }
  if (p->dft_tc) {
    st = dft_tc_setup(p);
    if (st != KDE_OK) {
      cudaFree(p->tw_dev);
      delete p;
      return st;
    }
  }
  *out = p;
  return KDE_OK;
}

kde_status kde_plan_get_info(kde_plan plan, kde_plan_info* info) {
  if (!plan || !info) return fail(KDE_ERR_INVALID_ARG, "NULL argument");
  *info = plan->info;
  return KDE_OK;
}

kde_status kde_plan_destroy(kde_plan plan) {
  if (!plan) return KDE_OK;
  cudaError_t e = cudaSuccess;
  if (plan->tw_dev) e = cudaFree(plan->tw_dev);
  if (plan->dft_tab) cudaFree(plan->dft_tab);
  delete plan;
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, "cudaFree(twiddles)");
}

kde_status kde_debug_status(int* enabled, int* code) {
  if (enabled) *enabled = KDE_DEBUG_ENABLED;
  if (!code) return KDE_OK;
  *code = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "kde_debug_status");
  int (*readers[])() = {kde::debug_read_bin, kde::debug_read_eval, kde::debug_read_fx_rows_counts,
                        kde::debug_read_fx_rows_kgen, kde::debug_read_fx_rows_c2r,
                        kde::debug_read_fx_cols_fwd, kde::debug_read_fx_cols_real,
                        kde::debug_read_fx_cols_mid, kde::debug_read_fx_cols_inv,
                        kde::debug_read_fx_cols_auto, kde::debug_read_fx_slab_fwd,
                        kde::debug_read_fx_slab_inv};
  for (auto rd : readers) {
    const int v = rd();
    if (v < 0) return fail(KDE_ERR_CUDA, "kde_debug_status: reading a check word failed");
    if (v && !*code) *code = v;
  }
  return KDE_OK;
}

const char* kde_status_string(kde_status s) {
  switch (s) {
    case KDE_OK: return "KDE_OK";
    case KDE_ERR_INVALID_ARG: return "KDE_ERR_INVALID_ARG";
    case KDE_ERR_NOT_SPD: return "KDE_ERR_NOT_SPD";
    case KDE_ERR_WORKSPACE: return "KDE_ERR_WORKSPACE";
    case KDE_ERR_OUT_OF_RANGE: return "KDE_ERR_OUT_OF_RANGE";
    case KDE_ERR_CUDA: return "KDE_ERR_CUDA";
    case KDE_ERR_TIMEOUT: return "KDE_ERR_TIMEOUT";
    case KDE_ERR_UNSUPPORTED: return "KDE_ERR_UNSUPPORTED";
  }
  return "unknown kde_status";
}

kde_status kde_plan_check(kde_plan plan, kde_stream_t stream) {
  if (!plan) return fail(KDE_ERR_INVALID_ARG, "plan is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int flag = 0;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(&flag, plan->status_dev, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && flag) e = cudaMemset(plan->status_dev, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "kde_plan_check");
  if (flag) return fail(KDE_ERR_TIMEOUT, "a bounded device-side wait gave up; the output is invalid");
  return KDE_OK;
}

kde_status kde_outside_check(const int64_t* n_outside, kde_stream_t stream, int64_t* count) {
  if (!n_outside) return fail(KDE_ERR_INVALID_ARG, "n_outside is NULL");
  int64_t v = 0;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemcpy(&v, n_outside, sizeof(int64_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "kde_outside_check");
  if (count) *count = v;
  if (v) return fail(KDE_ERR_OUT_OF_RANGE, "samples fell outside the grid");
  return KDE_OK;
}

const char* kde_last_error(void) { return g_last_error.c_str(); }

int64_t kde_launch_count(void) { return g_launches.load(); }

kde_status kde_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (on) {
    for (auto& r : g_prof) {
      g_event_pool.push_back(r.start);
      g_event_pool.push_back(r.stop);
    }
    g_prof.clear();
  }
  g_prof_on = on != 0;
  return KDE_OK;
}

struct ProfAgg {
  std::string name;
  double ms;
  int64_t n;
};
static std::vector<ProfAgg> g_agg;

int kde_profile_count(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_agg.clear();
  for (auto& r : g_prof) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.stop) != cudaSuccess) continue;
    if (cudaEventElapsedTime(&ms, r.start, r.stop) != cudaSuccess) continue;
    bool found = false;
    for (auto& a : g_agg)
      if (a.name == r.name) {
        a.ms += ms;
        a.n += 1;
        found = true;
      }
    if (!found) g_agg.push_back({r.name, (double)ms, 1});
  }
  return (int)g_agg.size();
}

kde_status kde_profile_entry(int i, const char** name, double* total_ms, int64_t* launches) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (i < 0 || i >= (int)g_agg.size()) return fail(KDE_ERR_INVALID_ARG, "no such entry");
  if (name) *name = g_agg[i].name.c_str();
  if (total_ms) *total_ms = g_agg[i].ms;
  if (launches) *launches = g_agg[i].n;
  return KDE_OK;
}

}  // extern "C"
