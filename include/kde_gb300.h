/*
 * kde_gb300.h -- C ABI of the GB300 (sm_103a) binned FFT kernel density
 * estimator with an unconstrained (full, symmetric positive definite)
 * bandwidth matrix H, after Gramacki & Gramacki, "FFT-Based Fast Computation
 * of Multivariate Kernel Density Estimators with Unconstrained Bandwidth
 * Matrices" (arXiv 1508.02766).
 *
 * The estimate is the truncated binned estimator of Eq. 7,
 *     f_j = sum_{|l_k| <= L_k} c_{j-l} k_l,   k_l = (1/n) K_H(delta_1 l_1, ..., delta_d l_d)
 * (Eq. 6), computed by the discrete convolution theorem (Eq. 10) with every
 * signed lag of the kernel kept (the corrected layout of Eq. 12-14, in its
 * equivalent wrapped form: k_l at index l mod P_k, counts at the origin, crop
 * [0, M_k)), and L_k from Eq. 15.
 *
 * Conventions shared by every call:
 *   - d is 1, 2 or 3.  Arrays are row-major with the last axis contiguous.
 *   - Pointers named X, counts, n_outside, Kspec, density and workspace are
 *     CUDA device pointers owned by the caller; the library never frees or
 *     keeps them.  X (read once, in order, by binning) and density (written
 *     once by the last pass) may also be page-locked host memory, which the
 *     kernels then read or write in place over the host link (unified
 *     addressing makes such memory device-accessible).  lo, hi, M, H and
 *     opts are host pointers read during the call only.
 *   - Calls taking a stream are asynchronous on that stream (NULL = legacy
 *     default stream).  Host-side argument checks happen before any launch
 *     and a failed check launches nothing.
 *   - Every call returns a kde_status; kde_last_error() gives a message for
 *     the most recent failure on the calling thread.
 */
#ifndef KDE_GB300_H
#define KDE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* kde_stream_t; /* same type as cudaStream_t */

typedef enum {
  KDE_OK = 0,
  KDE_ERR_INVALID_ARG = 1,  /* bad size, pointer, dtype, non-finite value, asymmetric H */
  KDE_ERR_NOT_SPD = 2,      /* H is not positive definite (Cholesky failed) */
  KDE_ERR_OUT_OF_RANGE = 3, /* samples fell outside the grid (kde_outside_check) */
  KDE_ERR_WORKSPACE = 4,    /* workspace smaller than the plan's workspace_bytes */
  KDE_ERR_CUDA = 5,         /* a CUDA runtime call or launch failed */
  KDE_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up (kde_plan_check) */
  KDE_ERR_UNSUPPORTED = 7   /* d not in 1..3, or a padded size above KDE_MAX_P */
} kde_status;

enum { KDE_F32 = 0, KDE_F64 = 1 };                   /* element types */
enum { KDE_RANGE_CORRECTED = 0, KDE_RANGE_PER_AXIS = 1 };
enum { KDE_LAYOUT_CORRECTED = 0, KDE_LAYOUT_WAND = 1 };
enum { KDE_COLS_AUTO = 0, KDE_COLS_LINES = 1, KDE_COLS_SIMD = 2 };
enum { KDE_ENGINE_AUTO = 0, KDE_ENGINE_STOCKHAM = 1, KDE_ENGINE_TWO_PHASE = 2 };
enum { KDE_SLAB_OFF = 0, KDE_SLAB_ON = 1 };

#define KDE_MAX_D 3
#define KDE_MAX_P 4096      /* largest padded length of one axis */
#define KDE_MAX_STAGES 16

/* Evaluation options.
 *   tau         Eq. 15's support constant (the paper finds about 3.7 for the
 *               2-D normal kernel); a value <= 0 selects 3.7.
 *   precision   KDE_F32 or KDE_F64: arithmetic of the kernel grid, the
 *               transforms and the density.
 *   range_mode  KDE_RANGE_CORRECTED: L_k = min(M_k-1, ceil(tau sqrt(lambda_max(H)) / delta_k))
 *               (Eq. 15).  KDE_RANGE_PER_AXIS: ceil(tau sqrt(H_kk) / delta_k),
 *               the axis-aligned range, kept to show what it truncates.
 *   layout_mode KDE_LAYOUT_CORRECTED: all signed lags (Eq. 12).
 *               KDE_LAYOUT_WAND: k_{|l_1|,...,|l_d|} at lag l, which is what
 *               Wand's wrap-around layout (Eq. 8) convolves with; wrong for
 *               non-diagonal H (Sec. 3-4.1), kept for demonstration.
 *   P_min       optional lower bounds on the padded sizes (0 = none).
 *   cols_variant  how passes along strided axes are organised: KDE_COLS_AUTO
 *               (by size), KDE_COLS_LINES (a thread group per column) or
 *               KDE_COLS_SIMD (16 columns side by side; used only where its
 *               shared-memory tile fits).  The result is the same up to
 *               rounding; this exists for testing and tuning.
 *   dft_tc      0: every transform is a mixed-radix FFT.  1 (KDE_F32 plans,
 *               d >= 2): the first pass of kde_fft_eval and kde_power_spectrum
 *               (each zero-padded row of counts -> its half spectrum, Eq. 10
 *               along the last axis) is a dense DFT-matrix product on the
 *               tensor cores in split TF32 (operands x = x_hi + x_lo, three
 *               products hi*hi + hi*lo + lo*hi, FP32 accumulation), about 2^-21
 *               relative per product; the plan then holds the DFT matrix
 *               (2 x 4 x roundup(2Q, 64) x roundup(M_last, 32) bytes).
 *   engine      how kde_kernel_grid and kde_fft_eval transform.
 *               KDE_ENGINE_TWO_PHASE (KDE_F32 plans, d >= 2): every line of
 *               length P_k = N1 N2 is an N1-point DFT per thread in
 *               registers, one exchange through shared memory, an N2-point
 *               DFT per thread (P_k <= 400); longer lines, P_k = N1 N2 N3
 *               (each about 10), take three such phases.  P_k is then the
 *               smallest supported length >= M_k + L_k (at most 2048).
 *               KDE_ENGINE_STOCKHAM: mixed-radix passes through shared
 *               memory, P_k the smallest 7-smooth size >= M_k + L_k.
 *               KDE_ENGINE_AUTO: two-phase where it applies (KDE_F32, d >= 2,
 *               every padded length a product as above), else Stockham.
 *               The result is the same up to rounding.
 *   slab_passes KDE_SLAB_OFF (default): separate row and column passes
 *               through global memory.  KDE_SLAB_ON (3-D two-phase plans
 *               without dft_tc, where the slab fits, see
 *               kde_plan_info.slab_passes): kde_fft_eval transforms the last
 *               two axes of each slab of the leading axis in one launch per
 *               direction, on clusters of 8 thread blocks that pass the
 *               intermediate half spectra between them in distributed shared
 *               memory (st.async stores counted on the receiver's mbarrier;
 *               bounded waits report through kde_plan_check).  The same
 *               arithmetic as the separate passes: the same result up to
 *               rounding.  Measured on GB300 at 256^3 it is not faster (the
 *               separate passes are bound by their transforms, not by the
 *               intermediate's round trip), so it is off by default. */
typedef struct {
  double tau;
  int precision;
  int range_mode;
  int layout_mode;
  int64_t P_min[KDE_MAX_D];
  int cols_variant;
  int dft_tc;
  int engine;
  int slab_passes;
} kde_opts;

/* Everything the plan derives on the host, in FP64.
 *   delta[k]   binwidth (Eq. 4); lambda_max  largest eigenvalue of H;
 *   L[k]       effective support (Eq. 15, or the per-axis range);
 *   P[k]       padded FFT length >= M_k + L_k (and >= P_min[k]): the smallest
 *              2^a 3^b 5^c 7^e (Stockham engine) or the smallest length the
 *              two-phase engine supports (see split);
 *              cyclic convolution of that length equals the linear one of
 *              Eq. 7 on [0, M_k) (Eq. 10, zero padding);
 *   Q          P[d-1]/2 + 1, the half-spectrum length of the last axis;
 *   kspec_elems   elements of the real kernel spectrum: P_0 ... P_{d-2} Q;
 *   workspace_bytes  scratch needed by kde_kernel_grid and kde_fft_eval;
 *   radix/nstages    the mixed-radix factorisation used per axis;
 *   engine     KDE_ENGINE_STOCKHAM or KDE_ENGINE_TWO_PHASE, as chosen;
 *   split[k]   the factors of P_k with the two-phase engine: N1, N2 and 0
 *              for lines up to 400, N1, N2, N3 (three exchanges instead of
 *              two, about 10 values per thread) for longer ones; all 0 with
 *              the Stockham engine;
 *   slab_passes  1 if kde_fft_eval takes the last two axes slab by slab on
 *              thread-block clusters (opts.slab_passes): d = 3, two-phase
 *              engine, two-factor splits of axes 1 and 2 with factors <= 20,
 *              no dft_tc, and a slab whose exchange fits in at most 113 KB
 *              of shared memory per block (2 blocks per SM).
 *              0 otherwise. */
typedef struct {
  int d;
  int precision;
  int64_t M[KDE_MAX_D];
  int64_t L[KDE_MAX_D];
  int64_t P[KDE_MAX_D];
  int64_t Q;
  double delta[KDE_MAX_D];
  double lambda_max;
  double det_H;
  int64_t kspec_elems;
  size_t kspec_bytes;
  size_t workspace_bytes;
  int nstages[KDE_MAX_D];
  int radix[KDE_MAX_D][KDE_MAX_STAGES];
  int engine;
  int split[KDE_MAX_D][3];
  int slab_passes;
} kde_plan_info;

typedef struct kde_plan_s* kde_plan;

/* Host-only planning (no GPU needed): checks the problem and fills *info.
 * H is d x d row-major, symmetric to 1e-12 relative (else INVALID_ARG) and
 * positive definite (else NOT_SPD).  lo[k] < hi[k] are the first and last
 * grid nodes g_{k1}, g_{kM_k} (Eq. 3-4); M[k] >= 2.  opts may be NULL. */
kde_status kde_plan_info_compute(int d, const int64_t* M, const double* lo, const double* hi,
                                 const double* H, const kde_opts* opts, kde_plan_info* info);

/* As kde_plan_info_compute, then builds the device-side twiddle tables
 * (e^{-2 pi i m / P_k}, generated in FP64) on the current device.  This is
 * set-up, not part of an evaluation: it allocates and synchronises.  The
 * plan owns the tables; free them with kde_plan_destroy. */
kde_status kde_plan_create(int d, const int64_t* M, const double* lo, const double* hi,
                           const double* H, const kde_opts* opts, kde_plan* out);
kde_status kde_plan_get_info(kde_plan plan, kde_plan_info* info);
kde_status kde_plan_destroy(kde_plan plan);

/* Linear binning (Sec. 2, first step).  X: n x d row-major device array of
 * float (x_dtype KDE_F32) or double (KDE_F64).  counts: prod(M) int64 in
 * units of 2^-32 of a sample; every cell is written by the call: each sample
 * inside the grid adds integer weights summing to exactly 2^32 to its 2^d
 * neighbouring nodes, so sum(counts) = (n - outside) * 2^32 (the paper's
 * requirement that counts sum to n, Sec. 3) and the result does not depend
 * on the order of the additions.  Rounding rules, per axis:
 *   t = (x - lo) * s in X's type, lo and s = (M-1)/(hi-lo) rounded to X's
 *   type, no fused multiply-add; t < 0, t > M-1 or NaN on any axis drops the
 *   sample and counts it in *n_outside; i = floor(t), f = t - i, a sample at
 *   t = M-1 uses i = M-2, f = 1; Q = round-half-even(f 2^32); the mass 2^32
 *   is split axis by axis (axis 0 first): part w gives
 *   floor((w Q + 2^31) / 2^32) to node i+1 and the rest to node i.
 * n_outside: device int64, zeroed then incremented; may be NULL.  n may be 0.
 * workspace: NULL selects the direct method (64-bit atomics into counts);
 * otherwise at least kde_bin_workspace_bytes(n, d, M) bytes, 256-byte
 * aligned, select the tiled method (the samples partitioned by grid tile,
 * then each tile accumulated in shared memory and stored once).  Both give
 * identical counts.  Requires n < 2^31 and prod(M) < 2^40 (tiled: < 2^32). */
kde_status kde_bin(const void* X, int x_dtype, int64_t n, int d, const double* lo,
                   const double* hi, const int64_t* M, int64_t* counts, int64_t* n_outside,
                   void* workspace, size_t workspace_bytes, kde_stream_t stream);

/* Linear binning added to existing counts (Sec. 2, first step; the binned
 * counts of Eq. 7 are a sum over samples, so binning the samples in parts
 * and adding gives the counts of all of them, bit for bit).  Arguments and
 * rounding as kde_bin, except that counts is not overwritten: every sample
 * inside the grid adds its 2^d weights to what counts holds, and the number
 * of samples outside is added to *n_outside (not zeroed).  Both methods
 * (workspace NULL or not) add; the tiled one touches only the tiles that
 * receive samples.  Counts that start at zero (for example after
 * kde_fft_eval_consume) give kde_bin's result. */
kde_status kde_bin_accumulate(const void* X, int x_dtype, int64_t n, int d, const double* lo,
                              const double* hi, const int64_t* M, int64_t* counts,
                              int64_t* n_outside, void* workspace, size_t workspace_bytes,
                              kde_stream_t stream);

/* Scratch bytes the tiled binning method needs for n samples on grid M:
 * a 16-byte record for every tile a sample can touch (2^d of them at most,
 * so 16 2^d n bytes) plus per-tile tables.  KDE_ERR_UNSUPPORTED for grids
 * of more than 16384 tiles (64^2 cells in 2-D, 16^3 in 3-D, 4096 in 1-D) or
 * 2^d n >= 2^32.  Host only. */
kde_status kde_bin_workspace_bytes(int64_t n, int d, const int64_t* M, size_t* bytes);

/* Kernel grid and its spectrum (Eq. 6, Eq. 10's K = F(k)).  Evaluates
 * k_l = K_H(delta o l) / (n 2^32 prod P) for |l_k| <= L_k at wrapped index
 * l mod P_k (zero elsewhere) and transforms it.  k_{-l} = k_l, so the
 * spectrum is real; Kspec receives it as plan.kspec_elems values of the
 * plan's precision: the half spectrum along the last axis (Q values) for
 * every leading frequency, in a plan-defined order (row-major
 * [P_0][P_1 ... P_{d-2}][Q], or with axis 0 innermost, depending on how the
 * plan organises the axis-0 pass); pass it unchanged to kde_fft_eval of the
 * same plan.  The 1/n of Eq. 2, the 2^-32 count unit and the 1/prod(P)
 * normalisation of Eq. 11/14 are folded in here.  n >= 1 is the number of
 * samples that were binned (the n of Eq. 2).  workspace: at least
 * plan.workspace_bytes of device scratch, 16-byte aligned. */
kde_status kde_kernel_grid(kde_plan plan, int64_t n, void* Kspec, void* workspace,
                           size_t workspace_bytes, kde_stream_t stream);

/* Density on the grid (Eq. 10 then the crop of Eq. 14 in wrapped form):
 * density = F^{-1}(F(c) K) restricted to [0, M_k) per axis.  counts come from
 * kde_bin with the plan's M, Kspec from kde_kernel_grid with the same plan.
 * density: prod(M) values of the plan's precision.  workspace as above;
 * it may be shared with kde_kernel_grid's when the calls are ordered. */
kde_status kde_fft_eval(kde_plan plan, const int64_t* counts, const void* Kspec, void* density,
                        void* workspace, size_t workspace_bytes, kde_stream_t stream);

/* kde_fft_eval (Eq. 10, Eq. 14), after which the counts are all zero, ready
 * for the next kde_bin_accumulate: a stream of datasets on one grid then
 * needs no separate zeroing before each binning.  The density is the same,
 * bit for bit, as kde_fft_eval's.  FP32 plans on the two-phase engine clear
 * the counts inside the evaluation's second pass, once the first pass (the
 * only one that reads them) has finished; other plans clear them with one
 * more operation at the end.  Arguments as kde_fft_eval; counts is
 * written. */
kde_status kde_fft_eval_consume(kde_plan plan, int64_t* counts, const void* Kspec, void* density,
                                void* workspace, size_t workspace_bytes, kde_stream_t stream);

/* Densities for many bandwidths on one binned grid (Eq. 10: the count
 * spectrum C = F(c) is computed once and reused, only the kernel spectrum K
 * changes with H).  H: nH x 2 x 2 host (row-major) bandwidths, each
 * symmetric positive definite and fitting the plan's padding
 * (M_k + L_k(H_i) <= P_k, Eq. 15; raise opts.P_min), else
 * KDE_ERR_NOT_SPD / KDE_ERR_INVALID_ARG before any launch.  n: the samples
 * binned.  density (device): nH x prod(M) values, bandwidth-major, each
 * grid exactly what kde_kernel_grid + kde_fft_eval give for that H (same
 * plan, layout and range rule).  Bandwidths go in chunks of 64 per launch:
 * kernel-grid rows, kernel spectrum, middle axis and output rows of the
 * chunk's bandwidths in four launches; their parameters are copied from
 * pageable host memory on the stream, so the call is not for graph capture.
 * KDE_F32 2-D plans with the two-phase engine (else KDE_ERR_UNSUPPORTED).
 * workspace: at least kde_fft_eval_multi_workspace_bytes(plan), 256-byte
 * aligned.  (Reusing F(c) is Eq. 10's structure; the batching is not in the
 * paper.) */
kde_status kde_fft_eval_multi(kde_plan plan, int64_t n, int nH, const double* H,
                              const int64_t* counts, void* density, void* workspace,
                              size_t workspace_bytes, kde_stream_t stream);
kde_status kde_fft_eval_multi_workspace_bytes(kde_plan plan, size_t* bytes);

/* Count spectrum for functionals of the estimate (Sec. 1 and Sec. 5: the
 * same FFT machinery serves fast bandwidth selection).  W receives
 * w_k |F(c)|^2 on the half spectrum, with c the counts in sample units
 * (2^-32 folded in) and w_k = 2 on the last axis except 1 at k = 0 and at
 * the Nyquist frequency, so that sum(W K) over the half spectrum is the
 * full-spectrum sum.  Same element count, order and precision as the
 * plan's kernel spectrum (plan.kspec_elems).  workspace as kde_fft_eval. */
kde_status kde_power_spectrum(kde_plan plan, const int64_t* counts, void* W, void* workspace,
                              size_t workspace_bytes, kde_stream_t stream);

/* Least-squares cross-validation for nH candidate bandwidths H_i (host,
 * nH x d x d row-major) on binned data, d = 1 or 2:
 *   LSCV(H) = S(2H) / n^2 - 2 (S(H) - n K_H(0)) / (n (n - 1)),
 *   S(A) = sum_j c_j sum_{|l| <= L(A)} c_{j-l} K_A(delta o l),
 * the textbook criterion with every double sum over samples replaced by the
 * binned sum (Eq. 2 form) that the FFT evaluates: S(A) = (1/prod P)
 * sum_w |C(w)|^2 K_A(w) (Eq. 10 with Parseval), with L(A) from Eq. 15.  W is
 * kde_power_spectrum's output for the same plan and counts; n the number of
 * samples binned.  Every H_i and 2 H_i must be symmetric positive definite
 * and fit the plan's padding (M_k + L_k <= P_k; raise opts.P_min), else
 * KDE_ERR_NOT_SPD / KDE_ERR_INVALID_ARG before any launch.  Outputs (device,
 * may alias nothing): lscv[nH]; pair_sums[2 nH] = S(H_0), S(2H_0), S(H_1), ...
 * (may be NULL).  Kernel spectra are computed in batches of 32 candidates
 * and never stored: their last pass is fused with the dot product against
 * W; partial sums are FP64 and reduced in a fixed order.  workspace: at
 * least kde_lscv_workspace_bytes(plan), 256-byte aligned. */
kde_status kde_lscv(kde_plan plan, int64_t n, int nH, const double* H, const void* W,
                    double* pair_sums, double* lscv, void* workspace, size_t workspace_bytes,
                    kde_stream_t stream);
kde_status kde_lscv_workspace_bytes(kde_plan plan, size_t* bytes);

/* The same criterion from the counts' autocorrelation (d = 2).  The binned
 * pair sum is S(A) = sum_j c_j sum_{|l| <= L(A)} c_{j-l} K_A(delta o l)
 * = sum_{|l| <= L(A)} K_A(delta o l) R(l) with R(l) = sum_j c_j c_{j-l}, the
 * autocorrelation of the counts (sample units), which the FFT gives once per
 * grid: R = F^{-1}(|F(c)|^2) on the plan's padding (Eq. 10 with the kernel
 * replaced by the counts; P_k >= M_k + L_k makes the cyclic sum the linear
 * one for every lag of the support).  Each candidate then costs one weighted
 * sum over its support (half of it: K_A and R are even) and no transform.
 *   kde_autocorrelation: R (device, P_0 x P_1 values of the plan's
 *     precision, lag (l_0, l_1) at (l_0 mod P_0, l_1 mod P_1)) from counts.
 *   kde_lscv_autocorr: as kde_lscv, with R in place of W.
 * Both take a workspace of at least kde_lscv_autocorr_workspace_bytes,
 * 256-byte aligned.  kde_lscv_autocorr copies the candidates' kernel
 * parameters (host-prepared, FP64 factorisations) into the workspace with
 * host-to-device copies on the stream, up to 1024 candidates per launch;
 * the copies read pageable host memory that the call frees on return, so
 * these calls are not for CUDA-graph capture (kde_lscv_autocorr_cands,
 * below, launches kernels only and can be captured). */
kde_status kde_lscv_autocorr_workspace_bytes(kde_plan plan, size_t* bytes);
kde_status kde_autocorrelation(kde_plan plan, const int64_t* counts, void* R, void* workspace,
                               size_t workspace_bytes, kde_stream_t stream);
kde_status kde_lscv_autocorr(kde_plan plan, int64_t n, int nH, const double* H, const void* R,
                             double* pair_sums, double* lscv, void* workspace,
                             size_t workspace_bytes, kde_stream_t stream);
/* The same for nsets datasets on one plan, each with its own candidates:
 * R holds the sets' autocorrelations back to back (nsets x P_0 x P_1), n
 * (host) the sets' sample counts, H (host) nsets x nH matrices (set-major),
 * lscv and pair_sums (device; pair_sums may be NULL) nsets x nH and
 * nsets x nH x 2 values.  Every candidate of every set goes into the same
 * lag-sum launches (up to 1024 candidates each), so a batch of small
 * candidate lists costs a few launches instead of two per set.  Same
 * workspace and errors as kde_lscv_autocorr; nsets = 0 or nH = 0 does
 * nothing.  (Batching over datasets has no counterpart in the paper.) */
kde_status kde_lscv_autocorr_batch(kde_plan plan, int nsets, const int64_t* n, int nH,
                                   const double* H, const void* R, double* pair_sums,
                                   double* lscv, void* workspace, size_t workspace_bytes,
                                   kde_stream_t stream);
/* A candidate list prepared once for repeated scoring (the plain search
 * scores the same candidates on every dataset): kde_lscv_cands_create
 * factorises the nH bandwidths H (host, nH x 2 x 2) on the host in FP64 and
 * keeps their lag-sum parameters in device memory it allocates (set-up, not
 * per evaluation; KDE_ERR_CUDA if the allocation fails); the set refers to
 * its plan, which must outlive it.  kde_lscv_autocorr_cands then scores the
 * set against the autocorrelation R of n samples exactly as
 * kde_lscv_autocorr(plan, n, nH, H, R, ...) does — same workspace, outputs
 * and results — with no host work and no copy: two launches per 1024
 * candidates.  (Caching candidates has no counterpart in the paper.) */
typedef struct kde_lscv_cands_s* kde_lscv_cands;
kde_status kde_lscv_cands_create(kde_plan plan, int nH, const double* H, kde_lscv_cands* out);
kde_status kde_lscv_cands_destroy(kde_lscv_cands cands);
kde_status kde_lscv_autocorr_cands(kde_lscv_cands cands, int64_t n, const void* R,
                                   double* pair_sums, double* lscv, void* workspace,
                                   size_t workspace_bytes, kde_stream_t stream);
/* The same candidate set scored against nsets autocorrelations at once
 * (R: nsets x P_0 x P_1 in the plan's precision, device; n: nsets sample
 * counts, host, each >= 2): lscv[s nH + i] (and pair_sums[2 (s nH + i)],
 * [2 (s nH + i) + 1] when not NULL; device) equal what
 * kde_lscv_autocorr_cands gives for dataset s alone.  Two launches per 1024
 * candidates whatever nsets (<= 65535).  workspace: at least
 * kde_lscv_autocorr_cands_batch_workspace_bytes(cands, nsets), 256-byte
 * aligned; n is copied from pageable memory, so the call is not for
 * CUDA-graph capture. */
kde_status kde_lscv_autocorr_cands_batch(kde_lscv_cands cands, int nsets, const int64_t* n,
                                         const void* R, double* pair_sums, double* lscv,
                                         void* workspace, size_t workspace_bytes,
                                         kde_stream_t stream);
kde_status kde_lscv_autocorr_cands_batch_workspace_bytes(kde_lscv_cands cands, int nsets,
                                                         size_t* bytes);
/* Candidates built on the device from per-dataset parameters (the learned
 * proposal's refinement, so that no bandwidth crosses to the host): theta =
 * (a, beta, c) stands for H = R R^T with R = [[e^a, 0], [beta e^c, e^c]]
 * (standardised coordinates).  For dataset s < nsets, candidate j < J is
 * clip(theta_s, box) + offsets[j] (theta: device, nsets x 3 FP32, e.g. a
 * network's output; box: host, lo[3] then hi[3]; offsets: host, J x 3) and
 * candidate J is ref[s] (host, nsets x 3).  Each candidate's H and 2H get the
 * support of Eq. 15 and the completed-square constants in FP64 on the device
 * (the host path's steps), then the LSCV of kde_lscv_autocorr against R
 * (device, nsets x P_0 x P_1 FP32) with n[s] samples (host).  A candidate
 * whose support does not fit the plan's padding scores +inf (no error).
 * Outputs (device): lscv[s (J + 1) + j] when not NULL; out[6 s ..] = {index
 * of the smallest LSCV among j < J (the first on ties; J if none fits), that
 * LSCV, the reference candidate's LSCV, that candidate's theta (3 values; 0
 * if none fits)}.  KDE_F32 2-D plans.  workspace: at
 * least kde_lscv_theta_select_workspace_bytes(plan, nsets, J), 256-byte
 * aligned; the host inputs are copied from pageable memory, so the call is
 * not for CUDA-graph capture.  (Not in the paper.) */
kde_status kde_lscv_theta_select(kde_plan plan, int nsets, const int64_t* n, const float* theta,
                                 const double* box, int J, const double* offsets,
                                 const double* ref, const void* R, double* lscv, double* out,
                                 void* workspace, size_t workspace_bytes, kde_stream_t stream);
kde_status kde_lscv_theta_select_workspace_bytes(kde_plan plan, int nsets, int J, size_t* bytes);

/* Ragged batches of independent 2-D problems (each with its own samples,
 * grid and bandwidth; Sec. 2 for each).  Two modes:
 *   KDE_BATCH_PERSISTENT (default): one persistent launch.  The work items
 *     of every problem and stage (zeroing of its counts, kernel rows,
 *     binning chunks, kernel spectrum, count rows, middle axis, output rows)
 *     form one device queue in stage order that the blocks claim with an
 *     atomic counter; an item waits, with a bounded spin, until the stages of
 *     its own problem that it reads from are complete (per-problem
 *     counters).  A wait that runs out (about a second by default) records
 *     a timeout, the launch's remaining items are abandoned and
 *     kde_batch_check reports KDE_ERR_TIMEOUT.
 *   KDE_BATCH_STAGED: seven launches, a memset and one grid-stride kernel
 *     per pass covering every problem; the two kernel-grid passes run on a
 *     stream the plan owns beside the binning (fork and join through events
 *     on the caller's stream).
 * Either way small and large grids share the GPU, the result is the same,
 * graph capture works and one plan evaluates one batch at a time.  X: the problems' samples concatenated in problem order (x_rows rows
 * of 2 values, the plan's precision).  density: the problems' grids
 * concatenated (density_elems values).  Dropped samples are not reported.
 * The plan allocates device tables (set-up, not per evaluation). */
typedef struct {
  int64_t M[2];
  double lo[2], hi[2];
  double H[4];
  int64_t n;
} kde_batch_item;
typedef struct kde_batch_plan_s* kde_batch_plan;
kde_status kde_batch_plan_create(int count, const kde_batch_item* items, const kde_opts* opts,
                                 kde_batch_plan* out);
kde_status kde_batch_plan_query(kde_batch_plan plan, int64_t* x_rows, int64_t* density_elems,
                                size_t* workspace_bytes);
/* Threads per line of the row passes and of the column passes (32, 64 or
 * 128); chosen by a caller-side tuner. */
kde_status kde_batch_set_shape(kde_batch_plan plan, int tpl_rows, int tpl_cols);
kde_status kde_batch_get_shape(kde_batch_plan plan, int* tpl_rows, int* tpl_cols);
/* The padding policy, the radix order in use (bits 0-7: 0 largest radix
 * first, 1 smallest first; bits 8-15: the queue order) and every problem's
 * padded lengths P (host, 2 x count int64, may be NULL). */
kde_status kde_batch_get_config(kde_batch_plan plan, int* pad_policy, int* radix_order, int64_t* P);
/* Autotuner: times kde_batch_eval on the given buffers (reps timed runs each,
 * CUDA events on the stream, which it synchronises) over
 *   the padding policy: KDE_BATCH_PAD_SMALLEST (each axis the smallest
 *     7-smooth length >= M + L) or KDE_BATCH_PAD_FEWEST_STAGES (the length
 *     with the fewest radix stages up to 25% longer);
 *   the radix order of every axis (largest radix first or last);
 *   the mode (KDE_BATCH_PERSISTENT with either queue order, KDE_BATCH_STAGED);
 *   the threads per line (32, 64, 128; the same for rows and columns in the
 *     persistent mode, every pair in the staged mode),
 * skipping settings whose workspace exceeds workspace_bytes, and keeps the
 * fastest in the plan (re-planning the problems); *best_ms (may be NULL)
 * receives its time.  Each timed run starts with cold caches when the
 * workspace is at least 64 MB: up to 256 MB of it (scratch) is overwritten
 * before the run, outside its timing, so that the choice holds for batches
 * that arrive with new data.  Set-up, not part of an evaluation.  The padded
 * lengths change the plan's workspace size: query it again after tuning. */
enum { KDE_BATCH_PAD_SMALLEST = 0, KDE_BATCH_PAD_FEWEST_STAGES = 1 };
kde_status kde_batch_tune(kde_batch_plan plan, const void* X, void* density, void* workspace,
                          size_t workspace_bytes, kde_stream_t stream, int reps, float* best_ms);
kde_status kde_batch_eval(kde_batch_plan plan, const void* X, void* density, void* workspace,
                          size_t workspace_bytes, kde_stream_t stream);
enum { KDE_BATCH_PERSISTENT = 0, KDE_BATCH_STAGED = 1 };
/* Order of the persistent queue: every problem's items stage by stage
 * (KDE_BATCH_QUEUE_STAGES) or problem by problem, the problems with the
 * most work first (KDE_BATCH_QUEUE_PROBLEMS, the default: a problem's later
 * stages then run while other problems are still being binned). */
enum { KDE_BATCH_QUEUE_STAGES = 0, KDE_BATCH_QUEUE_PROBLEMS = 1 };
kde_status kde_batch_set_queue_order(kde_batch_plan plan, int order);
kde_status kde_batch_set_mode(kde_batch_plan plan, int mode);
kde_status kde_batch_get_mode(kde_batch_plan plan, int* mode);
/* Synchronises the stream, reads and clears the persistent kernel's status:
 * KDE_ERR_TIMEOUT if one of its waits gave up since the last check (the
 * output of that evaluation is invalid), else KDE_OK. */
kde_status kde_batch_check(kde_batch_plan plan, kde_stream_t stream);
/* Diagnostic of the persistent kernel's waits (no counterpart in the paper):
 * each wait gives up after `polls` polls of about 256 ns (default 2^22), and
 * completions of stage `withhold_stage` (0 zeroing, 1 kernel rows, 2
 * binning, 3 kernel spectrum, 4 count rows, 5 middle axis, 6 output rows;
 * -1 none, the default) are never signalled, so the waits of the stages
 * after it run out.  Nothing faults or hangs: the blocks leave and the next
 * launch starts from a clean queue. */
kde_status kde_batch_set_wait(kde_batch_plan plan, uint32_t polls, int withhold_stage);
kde_status kde_batch_plan_destroy(kde_batch_plan plan);

/* kde_fft_eval without a workspace argument, for callers that cannot
 * allocate device memory where they evaluate (for example code whose
 * allocations all belong to a host framework, or a loop that must never enter
 * an allocator).  The paper has no counterpart; this is an interface
 * convenience.  Scratch comes from one fixed array of KDE_NOALLOC_SCRATCH_BYTES
 * inside the library, reserved on every device that loads the library until
 * the process exits.  The call allocates nothing.  Plans whose
 * workspace_bytes exceed KDE_NOALLOC_SCRATCH_BYTES are rejected with
 * KDE_ERR_WORKSPACE.  The first call on a device looks up the array's device
 * address (once per device, with that device current); make that first call
 * before any stream capture.  All calls share the array and nothing in it
 * needs to start at zero (each pass writes what the next one reads), but
 * calls whose work overlaps on the GPU (different streams, or different
 * host threads, without ordering between them) race on it. */
#define KDE_NOALLOC_SCRATCH_BYTES (8u << 20)
kde_status kde_fft_eval_noalloc(kde_plan plan, const int64_t* counts, const void* Kspec,
                                void* density, kde_stream_t stream);
/* The size of that fixed array as the library was built (bindings read it
 * here rather than repeating the constant).  The looked-up device address
 * is kept per device for the life of the process; it is no longer valid
 * after cudaDeviceReset, so do not use this entry point after resetting a
 * device in the same process. */
size_t kde_noalloc_scratch_bytes(void);

/* Device-side status of a plan.  Kernels that wait on a barrier inside the
 * GPU (the tensor-core first pass) bound every wait; a wait that gives up
 * records that in a status word the plan owns and the kernel returns
 * without finishing its work, so the call's output is then invalid.
 * kde_plan_check synchronises the stream, reads and clears that word and
 * returns KDE_ERR_TIMEOUT if any wait gave up since the previous check
 * (KDE_OK otherwise). */
kde_status kde_plan_check(kde_plan plan, kde_stream_t stream);

/* Binning's dropped samples as a status (Sec. 3 requires the grid to cover
 * the data): synchronises the stream, copies the device counter n_outside
 * filled by kde_bin into *count (host, may be NULL) and returns
 * KDE_ERR_OUT_OF_RANGE if it is nonzero, KDE_OK if it is zero. */
kde_status kde_outside_check(const int64_t* n_outside, kde_stream_t stream, int64_t* count);

/* Debug builds (no counterpart in the paper): compiled with KDE_DEBUG the
 * kernels check their indices (counts, tiles, spectra, output rows) and
 * record the first failure in a device word instead of accessing out of
 * range.  *enabled (host, may be NULL) receives 1 for such a build, 0 for a
 * release build; code (host, may be NULL) receives 0 or the failure's code
 * (which check), after synchronising the device, and the words are cleared.
 * With code NULL the call touches no device. */
kde_status kde_debug_status(int* enabled, int* code);

/* Diagnostics. */
const char* kde_status_string(kde_status s);
const char* kde_last_error(void);
/* Number of CUDA kernels this library has launched in this process. */
int64_t kde_launch_count(void);
/* Per-kernel timing with CUDA events on the launching stream.  Enabling
 * clears earlier records.  kde_profile_count/entry aggregate by kernel name
 * and synchronise on the recorded events. */
kde_status kde_profile_enable(int on);
int kde_profile_count(void);
kde_status kde_profile_entry(int i, const char** name, double* total_ms, int64_t* launches);
/* Check of the bounded wait the tensor-core kernels use on their mbarriers
 * (a diagnostic; the paper has no counterpart): one block of 32 threads
 * initialises an mbarrier expecting one arrival, arrives on it if `arrive`
 * is nonzero, and waits for it with at most `limit` polls.  out (device,
 * 2 int64, caller-owned) receives 0 if the wait completed or 1 if it gave
 * up, then the cycles the wait took.  With arrive = 0 nothing ever completes
 * the phase: the kernel must still end, reporting 1.  KDE_ERR_INVALID_ARG
 * for out = NULL or limit = 0. */
kde_status kde_wait_probe(int arrive, uint32_t limit, long long* out, kde_stream_t stream);

/* ---- Learned bandwidth proposal --------------------------------------------
 * The paper points to fast bandwidth selection with the same FFT machinery
 * (Sec. 1, Sec. 5) but gives no method; the network below is not from the
 * paper.  Its inputs are features of a 2-D sample: the samples standardised
 * per axis, binned (kde_bin) on a fixed M x M grid of the standardised
 * coordinates, downsampled to 32 x 32 block masses, plus moments.  Its
 * outputs are a log-Cholesky proposal for H in standardised coordinates,
 * which the caller scores with kde_lscv. */

#define KDE_FEAT_DIM 1088 /* 32 x 32 block features + 64 moment slots */

/* One block reduction over n >= 2 samples (X: n x 2 FP32, device):
 * Z = (X - mean) / sd per axis (FP32, device, n x 2) and moments[8] (FP64,
 * device) = mean0, mean1, sd0, sd1, correlation, skewness0, skewness1,
 * mean excess kurtosis of the two axes (population moments).  The sums are
 * FP32 trees, so the moments carry FP32-level relative error (about 1e-6). */
kde_status kde_standardize2(const float* X, int64_t n, float* Z, double* moments,
                            kde_stream_t stream);
/* feat[KDE_FEAT_DIM] (FP32, device) from counts (M x M int64 from kde_bin,
 * M a multiple of 32) of n samples and the moments above: feat[32 by + bx]
 * = 8 sqrt(mass of block (by, bx) / n), feat[1024 ..] = correlation, the two
 * skewnesses, excess kurtosis, log10(n)/4, 1, then zeros. */
kde_status kde_features2(const int64_t* counts, int M, int64_t n, const double* moments,
                         float* feat, kde_stream_t stream);
/* The whole per-dataset preparation of the learned and plain selections for
 * nsets datasets in one call (<= 65535; kde_standardize2, kde_bin of the
 * standardised samples on the plan's grid, kde_features2 and
 * kde_autocorrelation of each, with the same arithmetic, in batched
 * launches).  plan: d = 2, an M x M grid with M a multiple of 32.
 * X: concatenated samples (FP32, device), dataset s in rows
 * [offsets[s], offsets[s+1]) (offsets: host, nsets + 1 entries, offsets[0]
 * = 0, every dataset at least 2 samples).  Outputs (device): counts
 * nsets x M x M (int64, units of 2^-32; samples outside the grid are
 * dropped and still count in n), moments nsets x 8 (as kde_standardize2),
 * feat nsets x KDE_FEAT_DIM, R nsets x P_0 x P_1 (the plan's precision, as
 * kde_autocorrelation).  workspace: at least
 * kde_prepare2_batch_workspace_bytes(plan, nsets, offsets[nsets]), 256-byte
 * aligned (it holds the standardised samples and the transforms'
 * intermediates).  offsets are copied from pageable memory, so the call is
 * not for CUDA-graph capture. */
kde_status kde_prepare2_batch(kde_plan plan, int nsets, const float* X, const int64_t* offsets,
                              int64_t* counts, double* moments, float* feat, void* R,
                              void* workspace, size_t workspace_bytes, kde_stream_t stream);
kde_status kde_prepare2_batch_workspace_bytes(kde_plan plan, int nsets, int64_t n_total,
                                              size_t* bytes);

/* Three-layer perceptron y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with
 * BF16 operands and FP32 accumulation on the tensor cores (tcgen05),
 * FP32 master parameters and Adam (beta 0.9, 0.999, eps 1e-8).  Sizes:
 * in_dim % 64 == 0, hidden % 128 == 0, 1 <= out_dim <= 16, batches of at
 * most max_batch rows.  Parameters are laid out flat as W1 (hidden x in_dim,
 * row-major), b1, W2 (hidden x hidden), b2, W3 (out_dim x hidden), b3 and
 * start He-normal (biases zero) from the seeded generator.  X (B x in_dim),
 * T and Y (B x out_dim), loss (one float) and grads are device pointers;
 * the parameter/state copies are host pointers and synchronise.  The loss
 * is (1/B) sum over rows and outputs of (y - t)^2.  create allocates (set-up,
 * not per step).  kde_mlp_status synchronises and reports 1 if a wait for
 * the tensor cores gave up (the results of that call are then invalid). */
typedef struct kde_mlp_s* kde_mlp;
kde_status kde_mlp_create(int in_dim, int hidden, int out_dim, int max_batch, uint64_t seed,
                          kde_mlp* out);
kde_status kde_mlp_destroy(kde_mlp mlp);
kde_status kde_mlp_param_count(kde_mlp mlp, int64_t* count);
kde_status kde_mlp_get_params(kde_mlp mlp, float* host, int64_t count);
kde_status kde_mlp_set_params(kde_mlp mlp, const float* host, int64_t count);
kde_status kde_mlp_get_state(kde_mlp mlp, float* adam_m, float* adam_v, int64_t* step);
kde_status kde_mlp_set_state(kde_mlp mlp, const float* adam_m, const float* adam_v, int64_t step);
kde_status kde_mlp_forward(kde_mlp mlp, const float* X, int B, float* Y, kde_stream_t stream);
kde_status kde_mlp_loss_grad(kde_mlp mlp, const float* X, const float* T, int B, float* loss,
                             float* grads, kde_stream_t stream);
kde_status kde_mlp_train_step(kde_mlp mlp, const float* X, const float* T, int B, float lr,
                              float* loss, kde_stream_t stream);
kde_status kde_mlp_status(kde_mlp mlp, int* flag);
/* The same flag copied, in stream order and without synchronising, into
 * *dst (one int, device or page-locked host memory), for callers that read
 * it together with other results. */
kde_status kde_mlp_status_copy(kde_mlp mlp, int* dst, kde_stream_t stream);

/* The tensor-core matrix product behind the network, exposed for testing:
 * C[M x N] (FP32, row stride ldc) = A[M x K] B[N x K]^T with A and B BF16
 * row-major (row strides lda, ldb elements), M % 128 == 0, N % 16 == 0,
 * K % 64 == 0, strides multiples of 8, 16-byte aligned bases.  *status
 * (device int) is set to 1 if a wait for the tensor cores gave up. */
kde_status kde_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                         float* C, int ldc, int* status, kde_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* KDE_GB300_H */
