// Two-phase FFT passes (FP32) for kde_kernel_grid and kde_fft_eval: the
// convolution of Eq. 10 in the wrapped, zero-padded form, with every line of
// padded length P = N1 N2 transformed as
//   phase A: thread n2 (0 <= n2 < N2) holds x[n2 + N2 n1], n1 < N1, takes
//            their N1-point DFT in registers, multiplies entry k1 by
//            e^{-2 pi i n2 k1 / P} and writes it to shared memory;
//   phase B: thread k1 (0 <= k1 < N1) reads those N2 values and takes their
//            N2-point DFT in registers, which gives X[k1 + N1 k2], k2 < N2.
// The inverse runs the same steps backwards (B then A, conjugate twiddles),
// so a forward transform, a pointwise product and the inverse need two
// exchanges through shared memory.  Input positions n2 + N2 n1 and output
// positions k1 + N1 k2 are contiguous across neighbouring threads, so lines
// are read from and written to global memory directly.
//
// Passes (row-major, last axis contiguous, Q = P_last/2 + 1):
//   rows:  two real rows ride in one complex line (x + i y), split into their
//          half spectra after phase B (counts, or the kernel grid generated
//          on the fly); the inverse rebuilds the pair from Hermitian symmetry
//          and writes the rows cropped;
//   cols:  B adjacent columns per block (column index fastest across
//          threads); modes forward, forward to the real kernel spectrum (two
//          Hermitian columns per line), forward * K * inverse with crop (the
//          leading axis), inverse with crop.
// Only lines that hold data are transformed and only lines that survive the
// crop are inverse-transformed; positions beyond the data are zero padding.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "fx3_kernels.cuh"
#include "fx_slab.cuh"

namespace kde {
namespace fx {
namespace {

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
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

Line line_of(const kde_plan_info& I, int k) {
  Line l;
  l.P = (int)I.P[k];
  l.N1 = I.split[k][0];
  l.N2 = I.split[k][1];
  l.N3 = I.split[k][2];
  l.magic1 = (unsigned)((1ull << 32) / (unsigned)l.N1 + 1ull);
  return l;
}

// Entries per k1 row of a line's exchange buffer (N2, or N2 N3).
int row_entries(const Line& l) { return l.N3 ? l.N2 * l.N3 : l.N2; }

// Threads each phase uses per line: two factors {N2, N1}; three
// {N2 N3, N1 N3, N1 N2}.
int phase_threads(const Line& l, int* t) {
  if (!l.N3) {
    t[0] = l.N2;
    t[1] = l.N1;
    return 2;
  }
  t[0] = l.N2 * l.N3;
  t[1] = l.N1 * l.N3;
  t[2] = l.N1 * l.N2;
  return 3;
}

int threads_per_line(const Line& l) {
  int t[3];
  const int np = phase_threads(l, t);
  return *std::max_element(t, t + np);
}

int max_threads(const Line& l) {
  if (l.N3) return kThreads3;
  return std::max(l.N1, l.N2) <= kSmallMax ? kThreadsSmall : kThreadsLarge;
}

// Lanes in use, averaged over the phases, of a block of B lines (the block
// has B x threads_per_line threads rounded up to whole warps).
double lane_use(int B, const Line& l) {
  int t[3];
  const int np = phase_threads(l, t);
  const double slots = (double)((B * threads_per_line(l) + 31) / 32 * 32);
  double u = 0.0;
  for (int i = 0; i < np; ++i) u += B * t[i] / slots;
  return u / np;
}

// Lines per block for nlines lines: the block count should cover the SMs,
// and whole warps should be busy; score = min(1, blocks / SMs) x lane use.
int pick_lines(int64_t nlines, const Line& l, bool pow2) {
  const int tpl = threads_per_line(l);
  int best = 1;
  double best_s = -1.0;
  for (int B = 1; B * tpl <= max_threads(l) && B <= 64; B = pow2 ? 2 * B : B + 1) {
    const int64_t blocks = (nlines + B - 1) / B;
    const double cover = std::min(1.0, (double)blocks / (double)num_sms());
    const double s = cover * lane_use(B, l);
    if (s > best_s + 1e-9) {
      best_s = s;
      best = B;
    }
  }
  return best;
}

kde_status done(cudaError_t e, const char* name) {
  return e == cudaSuccess ? KDE_OK : cuda_fail(e, name);
}

const float2* twiddles(const kde_plan_s* plan, int k) {
  return reinterpret_cast<const float2*>((const char*)plan->tw_dev + plan->tw_offset[k]);
}

// Row pass: SRC_COUNTS (counts rows -> half spectra), SRC_KGEN (kernel-grid
// rows -> half spectra) or the inverse (half spectra -> rows, cropped).
// Batched bandwidths of one launch (grid.y = bandwidth): per-bandwidth
// kernel-grid parameters and supports on the device, element offsets between
// consecutive bandwidths of each array.
struct Batch {
  int nh = 1;
  const KGen<float>* gens = nullptr;
  const int* L0 = nullptr;
  int64_t slab_in = 0, slab_out = 0, slab_real = 0, slab_K = 0;
};

kde_status rows_pass(const kde_plan_s* plan, int kind, int64_t nrows, const long long* counts,
                     int Min, int64_t in_stride, const KGen<float>* g, float2* out,
                     const float2* in, float* out_real, int Mout, cudaStream_t st,
                     const Batch& bt = Batch()) {
  const kde_plan_info& I = plan->info;
  const int dl = I.d - 1;
  RowsArgs a{};
  a.nrows = nrows;
  a.Min = Min;
  a.in_stride = in_stride;
  a.Q = (int)I.Q;
  a.Mout = Mout;
  a.ln = line_of(I, dl);
  a.out = out;
  a.in = in;
  a.out_real = out_real;
  a.tw = twiddles(plan, dl);
  a.gens = bt.gens;
  a.slab_out = bt.slab_out;
  a.slab_in = bt.slab_in;
  a.slab_real = bt.slab_real;
  a.SK = row_entries(a.ln) | 1;
  const int64_t pairs = (nrows + 1) / 2;
  a.B = pick_lines(pairs, a.ln, false);
  const int threads = (a.B * threads_per_line(a.ln) + 31) / 32 * 32;
  // exchange buffers, plus the staged kernel values of the kernel-grid rows
  const size_t smem = ((size_t)a.B * a.ln.N1 * a.SK + (kind == SRC_KGEN ? (size_t)a.B * a.ln.P : 0)) *
                      sizeof(float2);
  if (smem > kSmemMax) return fail(KDE_ERR_UNSUPPORTED, "two-phase row block too large");
  const Launch l{a.ln.N1, a.ln.N2, a.ln.N3, dim3((unsigned)((pairs + a.B - 1) / a.B), (unsigned)bt.nh),
                 threads, smem, st};
  if (kind == 2) {
    LaunchScope ls("kde_fx_rows_c2r_kernel", st);
    return done(launch_rows_c2r(l, a), "kde_fx_rows_c2r_kernel");
  }
  if (kind == SRC_COUNTS) {
    LaunchScope ls("kde_fx_rows_r2c_counts_kernel", st);
    return done(launch_rows_counts(l, a, counts), "kde_fx_rows_r2c_counts_kernel");
  }
  LaunchScope ls("kde_fx_rows_r2c_kgen_kernel", st);
  return done(launch_rows_kgen(l, a, *g), "kde_fx_rows_r2c_kgen_kernel");
}

// Column pass along axis k over S columns of O slabs.
template <int MODE>
kde_status cols_pass(const kde_plan_s* plan, int k, const char* name, const float2* in,
                     float2* out, float* out_real, const float* K, int64_t S, int64_t O, int Nin,
                     int Nout, int Lw, cudaStream_t st, const Batch* bt = nullptr,
                     float s_pre = 0.f, float s_post = 0.f, unsigned long long* clear = nullptr,
                     int64_t clear_n = 0) {
  const kde_plan_info& I = plan->info;
  ColsArgs a{};
  a.s_pre = s_pre;
  a.s_post = s_post;
  a.clear = clear;
  a.clear_n = clear_n;
  if (bt) {  // slabs are bandwidths
    O = bt->nh;
    a.h_L0 = bt->L0;
    a.slab_in = bt->slab_in;
    a.slab_out = bt->slab_out;
    a.slab_real = bt->slab_real;
    a.slab_K = bt->slab_K;
  } else {   // outer slabs of a 3-D pass: [O][Nin][S] in, [O][Nout or P][S] out
    a.slab_in = (int64_t)Nin * S;
    a.slab_out = (int64_t)(MODE == COL_FWD ? (int)I.P[k] : Nout) * S;
  }
  a.in = in;
  a.out = out;
  a.out_real = out_real;
  a.K = K;
  a.S = S;
  a.Nin = Nin;
  a.Nout = Nout;
  a.Lw = Lw;
  a.ln = line_of(I, k);
  a.tw = twiddles(plan, k);
  const int64_t lines = (MODE == COL_FWD_REAL ? (S + 1) / 2 : S);
  // lines per block over all slabs: at least 4 adjacent columns (a 32-byte
  // sector per row; fewer make every load a partial sector), at most 16
  int B = std::max(4, pick_lines(lines * O, a.ln, true));
  while (B * threads_per_line(a.ln) > max_threads(a.ln)) B /= 2;
  while (B > 1 && B > lines) B /= 2;
  B = std::min(B, 16);
  a.B = B;
  a.lgB = 0;
  while ((1 << a.lgB) < B) ++a.lgB;
  a.SK = B * row_entries(a.ln);
  if (B < 16)
    while (a.SK % 16 != B % 16) ++a.SK;   // conflict-free reads across k1
  const int threads = (B * threads_per_line(a.ln) + 31) / 32 * 32;
  const size_t smem = (size_t)a.ln.N1 * a.SK * sizeof(float2);
  if (smem > kSmemMax) return fail(KDE_ERR_UNSUPPORTED, "two-phase column block too large");
  const Launch l{a.ln.N1, a.ln.N2, a.ln.N3, dim3((unsigned)((lines + B - 1) / B), (unsigned)O), threads, smem, st};
  LaunchScope ls(name, st);
  cudaError_t e;
  switch (MODE) {
    case COL_FWD: e = launch_cols_fwd(l, a); break;
    case COL_FWD_REAL: e = launch_cols_real(l, a); break;
    case COL_MID: e = launch_cols_mid(l, a); break;
    case COL_AUTO: e = launch_cols_auto(l, a); break;
    default: e = launch_cols_inv(l, a); break;
  }
  return done(e, name);
}

// Slab pass of a 3-D plan (fwd: counts -> spec [M0][P1][Q]; else spec ->
// density [M0][M1][M2]): one cluster of kSlabC blocks per slab of axis 0.
kde_status slab_pass(const kde_plan_s* plan, bool fwd, const long long* counts, float2* spec,
                     float* density, cudaStream_t st) {
  const kde_plan_info& I = plan->info;
  const fxp::SlabGeo g = fxp::slab_geometry(I.M[1], I.Q, I.split[2], I.split[1]);
  if (!g.ok) return fail(KDE_ERR_UNSUPPORTED, "slab passes do not fit this plan");
  SlabArgs a{};
  a.counts = counts;
  a.spec = spec;
  a.out_real = density;
  a.M1 = (int)I.M[1];
  a.M2 = (int)I.M[2];
  a.Q = (int)I.Q;
  a.lr = line_of(I, 2);
  a.lc = line_of(I, 1);
  a.twr = twiddles(plan, 2);
  a.twc = twiddles(plan, 1);
  a.RP = g.RP;
  a.W = g.W;
  a.SKr = g.SKr;
  a.SKc = g.SKc;
  a.ex_elems = g.ex_elems;
  a.status = plan->status_dev;
  const Launch l{a.lr.N1, a.lr.N2, 0, dim3((unsigned)(I.M[0] * kSlabC)), g.threads,
                 (size_t)(fwd ? g.smem_fwd : g.smem_inv), st};
  if (fwd) {
    LaunchScope ls("kde_fx_slab_fwd_kernel", st);
    return done(launch_slab_fwd(l, a), "kde_fx_slab_fwd_kernel");
  }
  LaunchScope ls("kde_fx_slab_inv_kernel", st);
  return done(launch_slab_inv(l, a), "kde_fx_slab_inv_kernel");
}

}  // namespace
}  // namespace fx

// Kernel grid and its real spectrum, two-phase engine (FP32, d = 2 or 3).
// Layout of Kspec: row-major [P_0][P_1 ... P_{d-2}][Q].
kde_status fx_kernel_grid(kde_plan_s* plan, const KGen<float>& gen, void* Kspec, void* ws,
                          cudaStream_t st) {
  using namespace fx;
  const kde_plan_info& I = plan->info;
  const int d = I.d;
  float2* t1 = (float2*)ws;
  int64_t rows = 1;
  for (int k = 0; k < d - 1; ++k) rows *= 2 * I.L[k] + 1;
  kde_status s = rows_pass(plan, SRC_KGEN, rows, nullptr, 0, 0, &gen, t1, nullptr, nullptr, 0, st);
  if (s != KDE_OK) return s;
  if (d == 2)
    return cols_pass<COL_FWD_REAL>(plan, 0, "kde_fx_cols_kgen_real_kernel", t1, nullptr,
                                   (float*)Kspec, nullptr, I.Q, 1, (int)(2 * I.L[0] + 1), 0,
                                   (int)I.L[0], st);
  // d == 3: axis 1 (wrapped lags) into t2, then axis 0 to the real spectrum
  float2* t2 = t1 + rows * I.Q;
  s = cols_pass<COL_FWD>(plan, 1, "kde_fx_cols_kgen_kernel", t1, t2, nullptr, nullptr, I.Q,
                         2 * I.L[0] + 1, (int)(2 * I.L[1] + 1), (int)I.P[1], (int)I.L[1], st);
  if (s != KDE_OK) return s;
  return cols_pass<COL_FWD_REAL>(plan, 0, "kde_fx_cols_kgen_real_kernel", t2, nullptr,
                                 (float*)Kspec, nullptr, I.P[1] * I.Q, 1, (int)(2 * I.L[0] + 1), 0,
                                 (int)I.L[0], st);
}

// Density from counts and the kernel spectrum, two-phase engine.  With
// clear (the counts), the second pass also sets the counts to zero once the
// first has read them.
kde_status fx_fft_eval(kde_plan_s* plan, const long long* counts, const float* Kspec,
                       float* density, void* ws, cudaStream_t st, unsigned long long* clear) {
  using namespace fx;
  const kde_plan_info& I = plan->info;
  const int d = I.d, dl = d - 1;
  float2* A = (float2*)ws;  // [M_0 .. M_{d-2}][Q]
  int64_t rows = 1;
  for (int k = 0; k < dl; ++k) rows *= I.M[k];
  const int64_t cells = rows * I.M[dl];
  kde_status s;
  if (I.slab_passes) {  // d == 3: axes 2 and 1 slab by slab, axis 0 between
    float2* Bf = A + rows * I.Q;  // [M_0][P_1][Q]
    s = slab_pass(plan, true, counts, Bf, nullptr, st);
    if (s != KDE_OK) return s;
    s = cols_pass<COL_MID>(plan, 0, "kde_fx_cols_mid_kernel", Bf, Bf, nullptr, Kspec,
                           I.P[1] * I.Q, 1, (int)I.M[0], (int)I.M[0], -1, st, nullptr, 0.f, 0.f,
                           clear, clear ? cells : 0);
    if (s != KDE_OK) return s;
    return slab_pass(plan, false, nullptr, Bf, density, st);
  }
  if (plan->dft_tc)
    s = dft_tc_rows(plan, counts, rows, A, st);
  else
    s = rows_pass(plan, SRC_COUNTS, rows, counts, (int)I.M[dl], I.M[dl], nullptr, A, nullptr,
                  nullptr, 0, st);
  if (s != KDE_OK) return s;
  if (d == 2) {
    s = cols_pass<COL_MID>(plan, 0, "kde_fx_cols_mid_kernel", A, A, nullptr, Kspec, I.Q, 1,
                           (int)I.M[0], (int)I.M[0], -1, st, nullptr, 0.f, 0.f, clear,
                           clear ? cells : 0);
  } else {
    float2* Bf = A + rows * I.Q;  // [M_0][P_1][Q]
    s = cols_pass<COL_FWD>(plan, 1, "kde_fx_cols_fwd_kernel", A, Bf, nullptr, nullptr, I.Q, I.M[0],
                           (int)I.M[1], (int)I.P[1], -1, st, nullptr, 0.f, 0.f, clear,
                           clear ? cells : 0);
    if (s != KDE_OK) return s;
    s = cols_pass<COL_MID>(plan, 0, "kde_fx_cols_mid_kernel", Bf, Bf, nullptr, Kspec,
                           I.P[1] * I.Q, 1, (int)I.M[0], (int)I.M[0], -1, st);
    if (s != KDE_OK) return s;
    s = cols_pass<COL_INV>(plan, 1, "kde_fx_cols_inv_kernel", Bf, A, nullptr, nullptr, I.Q, I.M[0],
                           (int)I.P[1], (int)I.M[1], -1, st);
  }
  if (s != KDE_OK) return s;
  return rows_pass(plan, 2, rows, nullptr, 0, 0, nullptr, nullptr, A, density, (int)I.M[dl], st);
}

}  // namespace kde

namespace kde {

// Densities for nh bandwidths of a 2-D plan that share the counts' half
// spectra A (Eq. 10 with C = F(c) reused; only K changes with H): per
// bandwidth the kernel-grid rows, its real spectrum, the middle axis
// (forward, times K, inverse) and the output rows, each pass one launch over
// all nh bandwidths.  gens and L0 (device) hold each bandwidth's kernel-grid
// parameters and support along axis 0; Lmax0 bounds the supports.
kde_status fx_eval_batch2(kde_plan_s* plan, const float2* A, int nh, const KGen<float>* gens,
                          const int* L0, int Lmax0, float2* t1, float* Kb, float2* Sb,
                          float* density, cudaStream_t st) {
  using namespace fx;
  const kde_plan_info& I = plan->info;
  const int64_t Q = I.Q, M0 = I.M[0], M1 = I.M[1], P0 = I.P[0];
  const int64_t rows_max = 2 * (int64_t)Lmax0 + 1;
  Batch b;
  b.nh = nh;
  b.gens = gens;
  b.L0 = L0;
  b.slab_out = rows_max * Q;
  KGen<float> g0 = {};
  kde_status s = rows_pass(plan, SRC_KGEN, rows_max, nullptr, 0, 0, &g0, t1, nullptr, nullptr, 0,
                           st, b);
  if (s != KDE_OK) return s;
  b = Batch();
  b.nh = nh;
  b.L0 = L0;
  b.slab_in = rows_max * Q;
  b.slab_real = P0 * Q;
  s = cols_pass<COL_FWD_REAL>(plan, 0, "kde_fx_cols_kgen_real_kernel", t1, nullptr, Kb, nullptr,
                              Q, 1, (int)rows_max, 0, Lmax0, st, &b);
  if (s != KDE_OK) return s;
  b = Batch();
  b.nh = nh;
  b.slab_in = 0;          // every bandwidth reads the same count spectra
  b.slab_out = M0 * Q;
  b.slab_K = P0 * Q;
  s = cols_pass<COL_MID>(plan, 0, "kde_fx_cols_mid_kernel", A, Sb, nullptr, Kb, Q, 1, (int)M0,
                         (int)M0, -1, st, &b);
  if (s != KDE_OK) return s;
  b = Batch();
  b.nh = nh;
  b.slab_in = M0 * Q;
  b.slab_real = M0 * M1;
  return rows_pass(plan, 2, M0, nullptr, 0, 0, nullptr, nullptr, Sb, density, (int)M1, st, b);
}

// The counts' autocorrelation R = F^{-1}(|F(c)|^2) of nsets grids (2-D,
// counts [nsets][M_0][M_1] -> R [nsets][P_0][P_1]): rows of every grid to
// half spectra A, axis 0 forward, |2^-32 z|^2 / (P_0 P_1), inverse (all P_0
// rows kept) into B, then full rows.  A: nsets M_0 Q, B: nsets P_0 Q complex.
kde_status fx_autocorr(kde_plan_s* plan, const long long* counts, float* R, float2* A, float2* B,
                       int64_t nsets, cudaStream_t st) {
  using namespace fx;
  const kde_plan_info& I = plan->info;
  kde_status s = rows_pass(plan, SRC_COUNTS, nsets * I.M[0], counts, (int)I.M[1], I.M[1], nullptr,
                           A, nullptr, nullptr, 0, st);
  if (s != KDE_OK) return s;
  s = cols_pass<COL_AUTO>(plan, 0, "kde_fx_cols_auto_kernel", A, B, nullptr, nullptr, I.Q, nsets,
                         (int)I.M[0], (int)I.P[0], -1, st, nullptr, 2.3283064365386963e-10f,
                         (float)(1.0 / ((double)I.P[0] * (double)I.P[1])));
  if (s != KDE_OK) return s;
  return rows_pass(plan, 2, nsets * I.P[0], nullptr, 0, 0, nullptr, nullptr, B, R, (int)I.P[1], st);
}

// The counts' half spectra (first pass of the evaluation) into A.
kde_status fx_count_spectra(kde_plan_s* plan, const long long* counts, float2* A, cudaStream_t st) {
  using namespace fx;
  const kde_plan_info& I = plan->info;
  const int dl = I.d - 1;
  int64_t rows = 1;
  for (int k = 0; k < dl; ++k) rows *= I.M[k];
  if (plan->dft_tc) return dft_tc_rows(plan, counts, rows, A, st);
  return rows_pass(plan, SRC_COUNTS, rows, counts, (int)I.M[dl], I.M[dl], nullptr, A, nullptr,
                   nullptr, 0, st);
}

}  // namespace kde
