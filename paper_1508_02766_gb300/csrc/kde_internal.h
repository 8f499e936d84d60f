// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/kde_gb300.h"

struct kde_plan_s {
  kde_plan_info info;
  double H[9];
  double Hinv[9];
  double lo[KDE_MAX_D];
  double hi[KDE_MAX_D];
  double tau;
  int range_mode;
  int layout_mode;
  int cols_variant;
  int device;
  // Twiddle tables e^{-2 pi i m / P_k}, m in [0, P_k): one per axis, in the
  // plan's precision (float2 or double2), owned by the plan.
  void* tw_dev;
  size_t tw_offset[KDE_MAX_D];  // byte offset of axis k's table in tw_dev
  // Device status word (inside the twiddle allocation, after the tables):
  // nonzero once a bounded wait in one of the plan's kernels gave up.
  int* status_dev;
  // Tensor-core DFT of the first pass (opts.dft_tc): the real DFT matrix of
  // the last axis restricted to its M_last data points, split into TF32
  // high and low parts, each dft_N x dft_K floats (rows 2q, 2q+1 = cos,
  // -sin of 2 pi q x / P; zero beyond 2Q and M_last).
  int dft_tc;
  float* dft_tab;
  int dft_N, dft_K, dft_BN;
};

namespace kde {

kde_status fail(kde_status s, const std::string& msg);
kde_status matrix_support(const kde_plan_s* plan, const double* A, double* Ainv, double* detA,
                          int64_t* L);
kde_status cuda_fail(cudaError_t e, const char* what);
// Asynchronous upload of a small host array (copied into a page-locked
// staging slot first, so the caller's array may be reused at once).  Not for
// stream capture: a captured copy would replay the slot's later contents.
kde_status upload_async(void* dst, const void* src, size_t bytes, cudaStream_t st);
// K_A(delta o l) = C exp(sum_k D_k (l_k + sum_{j<k} B_kj l_j)^2) from the
// Cholesky factor of A (no cancellation when A is nearly singular);
// B = {B_10, B_20, B_21}, entries beyond d zero.
kde_status gauss_factor(int d, const double* A, const double* delta, double* D, double* B);
// Tensor-core first pass (dft_tc.cu): build the plan's DFT matrix; run the
// counts rows -> half spectra pass (rows of length M_last, out [rows][Q]).
kde_status dft_tc_setup(kde_plan_s* plan);
kde_status dft_tc_rows(const kde_plan_s* plan, const long long* counts, int64_t rows, void* out,
                       cudaStream_t st);

// Two-phase engine (eval_fx.cu, KDE_F32 plans with engine
// KDE_ENGINE_TWO_PHASE): the kernel grid and its spectrum, and the
// evaluation, with the same arguments as the Stockham passes.
template <typename T>
struct KGen;
kde_status fx_kernel_grid(kde_plan_s* plan, const KGen<float>& gen, void* Kspec, void* ws,
                          cudaStream_t st);
kde_status fx_fft_eval(kde_plan_s* plan, const long long* counts, const float* Kspec,
                       float* density, void* ws, cudaStream_t st,
                       unsigned long long* clear = nullptr);
kde_status fx_count_spectra(kde_plan_s* plan, const long long* counts, float2* A, cudaStream_t st);
kde_status fx_autocorr(kde_plan_s* plan, const long long* counts, float* R, float2* A, float2* B,
                       int64_t nsets, cudaStream_t st);
kde_status fx_eval_batch2(kde_plan_s* plan, const float2* A, int nh, const KGen<float>* gens,
                          const int* L0, int Lmax0, float2* t1, float* Kb, float2* Sb,
                          float* density, cudaStream_t st);

// Prepared batches of 2-D datasets (kde_prepare2_batch): binning of nsets
// datasets onto one grid (bin.cu; samples rows [off[s], off[s+1]) of X,
// offsets on the device, counts [nsets][prod M] zeroed first), and the
// standardisation and features of each (learn.cu; same offsets, moments
// [nsets][8], features [nsets][KDE_FEAT_DIM]).
kde_status bin_sets_f32(const float* X, const int64_t* off_dev, int nsets, int64_t n_max, int d,
                        const double* lo, const double* hi, const int64_t* M, int64_t* counts,
                        cudaStream_t st);
kde_status standardize2_sets(const float* X, const int64_t* off_dev, int nsets, float* Z,
                             double* moments, cudaStream_t st);
kde_status features2_sets(const int64_t* counts, int M, int nsets, const int64_t* off_dev,
                          const double* moments, float* feat, cudaStream_t st);

// Readers of the per-translation-unit check words of a debug build (0 in a
// release build; -1 if the word could not be read).
int debug_read_bin();
int debug_read_eval();
int debug_read_fx_rows_counts();
int debug_read_fx_rows_kgen();
int debug_read_fx_rows_c2r();
int debug_read_fx_cols_fwd();
int debug_read_fx_cols_real();
int debug_read_fx_cols_mid();
int debug_read_fx_cols_auto();
int debug_read_fx_cols_inv();
int debug_read_fx_slab_fwd();
int debug_read_fx_slab_inv();

// Launch bookkeeping: counts launches and, when profiling is on, records a
// pair of events around each launch on its stream.
struct LaunchScope {
  LaunchScope(const char* name, cudaStream_t stream);
  ~LaunchScope();
  int slot;
  cudaStream_t stream;
};

}  // namespace kde
