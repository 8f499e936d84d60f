// Slab passes of the two-phase engine for 3-D plans: the last two axes of
// one slab i of the leading axis (counts[i] is M1 x M2) transformed by one
// thread-block cluster, with the intermediate half spectra moved between the
// cluster's blocks through distributed shared memory instead of a round trip
// through global memory (Eq. 10, the same transforms as the row and column
// passes, in the same order and with the same arithmetic).
//
// Forward (counts[i] -> spec[i], [P1][Q]): block c of the kSlabC blocks
//   1. takes the row pairs b < RP, rows r0 = 2 (c RP + b), r0 + 1: the real
//      rows of length M2 zero-padded to P2 ride as x + i y in one complex
//      line, phase A (N1r-point DFTs) and phase B (N2r-point DFTs) as in the
//      row pass;
//   2. splits each line into the two half spectra X_k, Y_k, k < Q, and
//      stores entry k of row r into the buffer of block k / W (the block
//      that owns half-spectrum column k), at [r][k mod W];
//   3. after a cluster barrier holds all M1 rows of its W columns and takes
//      their P1-point transforms (zero beyond M1), phase A then phase B,
//      storing spec[i][k1 + N1c k2][c W + w].
// Inverse (spec[i] -> density[i], M1 x M2): block c takes the inverse
//   transforms of its W columns (phase B from global memory, then phase A),
//   keeps rows n < M1 (the crop) and stores entry (n, k) into the buffer of
//   the block that owns row n, at [n - 2 RP owner][k]; after a cluster
//   barrier each block rebuilds its row pairs' full lines from the half
//   spectra (Hermitian symmetry above Q) and takes their inverse row
//   transforms, storing the rows cropped to M2.
//
// Synchronisation: every block of a cluster is known to be running, and its
// mbarrier initialised, once a first cluster barrier completes (arrived at
// the kernel's start, waited on before the first remote store).  The remote
// stores are st.async operations that count their bytes on the receiving
// block's mbarrier, which expects exactly what the cluster sends it; a block
// waits (bounded) on its own mbarrier before it reads its cluster buffer.  A
// second cluster barrier, arrived after a block's stores are issued and
// waited on at its end, keeps every block resident until all stores to it
// have been issued.  Shared memory: the mbarrier (16 bytes), an exchange
// region (the row phases' lines, entry (b, k1, n2) at b N1r SKr + k1 SKr +
// n2, or the column phases' lines, entry (w, k1, n2) at w + n2 W + k1 SKc),
// then the cluster buffer ([M1][W] forward, [2 RP][Q] inverse).
#pragma once

#include "fx_kernels.cuh"
#include "tc_wait.cuh"

namespace kde {
namespace fx {

inline constexpr int kSlabC = fxp::kSlabC;                // blocks per cluster (portable size)
inline constexpr int kSlabThreads = fxp::kSlabMaxThreads;  // block limit

struct SlabArgs {
  const long long* counts;  // forward: [M0][M1][M2]
  float2* spec;             // forward out, inverse in: [M0][P1][Q]
  float* out_real;          // inverse: [M0][M1][M2]
  int M1, M2, Q;
  Line lr;                  // axis 2 (rows), P2 = N1 N2
  Line lc;                  // axis 1 (columns), P1 = N1 N2
  const float2* twr;        // e^{-2 pi i m / P2}
  const float2* twc;        // e^{-2 pi i m / P1}
  int RP;                   // row pairs per block
  int W;                    // half-spectrum columns per block
  int SKr, SKc;             // exchange strides (see above)
  int ex_elems;             // float2 entries of the exchange region
  int* status;              // the plan's status word (set if a wait gives up)
};

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address a (this block's shared window) in block rank's window.
__device__ __forceinline__ unsigned cluster_addr_u32(unsigned a, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ unsigned cluster_addr(const void* p, unsigned rank) {
  return cluster_addr_u32((unsigned)__cvta_generic_to_shared(p), rank);
}
// The exchange: each block's mbarrier (the first 16 bytes of its shared
// memory) expects exactly the bytes the cluster sends it, and every remote
// store is an st.async that counts its 8 bytes on the receiver's barrier, so
// a block waits only for its own data and no fence is needed on the sending
// side.  The wait is bounded (kWaitLimit polls, about a second): if it gives
// up, the plan's status word is set and the block carries on.
__device__ __forceinline__ void mbar_init_cluster(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void st_async(unsigned addr, float2 v, unsigned bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr),
               "f"(v.x), "f"(v.y), "r"(bar)
               : "memory");
}
__device__ __forceinline__ bool mbar_wait_cluster(unsigned bar, unsigned limit) {
  unsigned done = 0;
  for (unsigned it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar)
        : "memory");
  }
  return done != 0;
}

// ---- forward -------------------------------------------------------------

// Row phase A: thread (b, n2) loads counts rows r0, r0 + 1 at n2 + N2 n1.
template <int N1>
__device__ __forceinline__ void slab_rows_a(const SlabArgs& a, const long long* __restrict__ counts,
                                            int c, float2* ex) {
  const int N2 = a.lr.N2;
  for (int t = threadIdx.x; t < a.RP * N2; t += blockDim.x) {
    const int b = t / N2, n2 = t - b * N2;
    const int r0 = 2 * (c * a.RP + b);
    const bool one = r0 < a.M1, two = r0 + 1 < a.M1;
    const long long* c0 = counts + (int64_t)r0 * a.M2;
    long long v0[N1], v1[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const int pos = n2 + N2 * n1;
      v0[n1] = (one && pos < a.M2) ? __ldg(c0 + pos) : 0;
      v1[n1] = (two && pos < a.M2) ? __ldg(c0 + a.M2 + pos) : 0;
    }
    float2 x[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1)
      x[n1] = make_float2(count_value<float>(v0[n1]), count_value<float>(v1[n1]));
    a_fwd_store<N1>(x, n2, a.twr, ex + b * (N1 * a.SKr) + n2, a.SKr);
  }
}

// Row phase B: thread (b, k1), Z[k1 + N1 k2] back into the slots it read.
template <int N2>
__device__ __forceinline__ void slab_rows_b(const SlabArgs& a, float2* ex) {
  const int N1 = a.lr.N1;
  for (int t = threadIdx.x; t < a.RP * N1; t += blockDim.x) {
    const int b = t / N1, k1 = t - b * N1;
    float2* src = ex + b * (N1 * a.SKr) + k1 * a.SKr;
    float2 y[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) y[n2] = src[n2];
    dft<N2>(y);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) src[k2] = y[k2];
  }
}

// X = F(x), Y = F(y) from Z = F(x + i y); entry k of row r to block k / W.
__device__ __forceinline__ void slab_rows_scatter(const SlabArgs& a, int c, const float2* ex,
                                                  const float2* cb, unsigned bar) {
  const int N1 = a.lr.N1, P = a.lr.P;
  for (int idx = threadIdx.x; idx < a.RP * a.Q; idx += blockDim.x) {
    const int b = idx / a.Q, k = idx - b * a.Q;
    const int r0 = 2 * (c * a.RP + b);
    if (r0 >= a.M1) break;  // later idx have larger b
    const float2* z = ex + b * (N1 * a.SKr);
    const int km = k == 0 ? 0 : P - k;
    const int q = (int)__umulhi((unsigned)k, a.lr.magic1);
    const int qm = (int)__umulhi((unsigned)km, a.lr.magic1);
    const float2 zk = z[(k - q * N1) * a.SKr + q];
    const float2 zm = z[(km - qm * N1) * a.SKr + qm];
    const int owner = k / a.W, w = k - owner * a.W;
    if (!KDE_DCHECK(owner < kSlabC && r0 < a.M1, KDE_DBG_SLAB)) continue;
    const unsigned dst = cluster_addr(cb, (unsigned)owner) + (unsigned)(r0 * a.W + w) * 8u;
    const unsigned rbar = cluster_addr_u32(bar, (unsigned)owner);
    st_async(dst, make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y)), rbar);
    if (r0 + 1 < a.M1)
      st_async(dst + (unsigned)a.W * 8u, make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x)), rbar);
  }
}

// Column phase A: thread (w, n2) takes rows n2 + N2 n1 (< M1) of column w.
template <int N1>
__device__ __forceinline__ void slab_cols_a(const SlabArgs& a, const float2* cb, float2* ex) {
  const int N2 = a.lc.N2;
  for (int t = threadIdx.x; t < a.W * N2; t += blockDim.x) {
    const int n2 = t / a.W, w = t - n2 * a.W;
    float2 x[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const int pos = n2 + N2 * n1;
      x[n1] = pos < a.M1 ? cb[pos * a.W + w] : make_float2(0.f, 0.f);
    }
    a_fwd_store<N1>(x, n2, a.twc, ex + w + n2 * a.W, a.SKc);
  }
}

// Column phase B: thread (w, k1), X[k1 + N1 k2] to spec[i][k1 + N1 k2][c W + w].
template <int N2>
__device__ __forceinline__ void slab_cols_b(const SlabArgs& a, int c, int64_t i, const float2* ex) {
  const int N1 = a.lc.N1;
  for (int t = threadIdx.x; t < a.W * N1; t += blockDim.x) {
    const int k1 = t / a.W, w = t - k1 * a.W;
    const float2* src = ex + w + k1 * a.SKc;
    float2 y[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) y[n2] = src[n2 * a.W];
    dft<N2>(y);
    const int col = c * a.W + w;
    if (col >= a.Q) continue;
    float2* out = a.spec + i * (int64_t)a.lc.P * a.Q + col;
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2)
      if (KDE_DCHECK(k1 + N1 * k2 < a.lc.P, KDE_DBG_SLAB)) out[(int64_t)(k1 + N1 * k2) * a.Q] = y[k2];
  }
}

template <int CLS, int N1T, int N2T>
__global__ void __launch_bounds__(kSlabThreads, 2) kde_fx_slab_fwd_kernel(SlabArgs a) {
  pdl_trigger();
  extern __shared__ float2 fx_sm[];
  const unsigned bar = (unsigned)__cvta_generic_to_shared(fx_sm);
  float2* ex = fx_sm + 2;
  float2* cb = ex + a.ex_elems;
  const int c = (int)cluster_rank();
  const int64_t i = blockIdx.x / kSlabC;
  if (threadIdx.x == 0) mbar_init_cluster(bar);
  cluster_arrive_relaxed();
  pdl_wait();
  const long long* counts = a.counts + i * (int64_t)a.M1 * a.M2;
  size_call<N1T, CLS>(a.lr.N1, [&](auto N) { slab_rows_a<decltype(N)::value>(a, counts, c, ex); });
  __syncthreads();
  size_call<N2T, CLS>(a.lr.N2, [&](auto N) { slab_rows_b<decltype(N)::value>(a, ex); });
  __syncthreads();
  if (threadIdx.x == 0) {  // all M1 rows of this block's columns
    const int wc = min(a.W, max(0, a.Q - c * a.W));
    mbar_expect(bar, (unsigned)(a.M1 * wc) * 8u);
  }
  cluster_wait();  // every block of the cluster is running, its barrier initialised
  slab_rows_scatter(a, c, ex, cb, bar);
  cluster_arrive_relaxed();  // this block's stores are issued
  if (!mbar_wait_cluster(bar, kWaitLimit) && threadIdx.x == 0) atomicExch(a.status, 1);
  size_call<N1T, CLS>(a.lc.N1, [&](auto N) { slab_cols_a<decltype(N)::value>(a, cb, ex); });
  __syncthreads();
  size_call<N2T, CLS>(a.lc.N2, [&](auto N) { slab_cols_b<decltype(N)::value>(a, c, i, ex); });
  cluster_wait();  // no block leaves while stores to it may be outstanding
}

// ---- inverse -------------------------------------------------------------

// Column inverse phase B: thread (w, k1) reads X[k1 + N1 k2] of column c W + w.
template <int N2>
__device__ __forceinline__ void slab_icols_b(const SlabArgs& a, int c, int64_t i, float2* ex) {
  const int N1 = a.lc.N1;
  for (int t = threadIdx.x; t < a.W * N1; t += blockDim.x) {
    const int k1 = t / a.W, w = t - k1 * a.W;
    const int col = c * a.W + w;
    const bool v = col < a.Q;
    const float2* in = a.spec + i * (int64_t)a.lc.P * a.Q + col;
    float2 y[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2)
      y[k2] = v ? __ldg(in + (int64_t)(k1 + N1 * k2) * a.Q) : make_float2(0.f, 0.f);
    b_inv_store<N2>(y, k1, a.twc, ex + w + k1 * a.SKc, a.W);
  }
}

// Column inverse phase A: thread (w, n2), rows n2 + N2 n1 < M1 to their
// owners' buffers.
template <int N1>
__device__ __forceinline__ void slab_icols_a(const SlabArgs& a, int c, const float2* ex,
                                             const float2* hb, unsigned bar) {
  const int N2 = a.lc.N2;
  for (int t = threadIdx.x; t < a.W * N2; t += blockDim.x) {
    const int n2 = t / a.W, w = t - n2 * a.W;
    const int col = c * a.W + w;
    const float2* src = ex + w + n2 * a.W;
    float2 x[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) x[k1] = src[k1 * a.SKc];
    idft<N1>(x);
    if (col >= a.Q) continue;
    const int rows = 2 * a.RP;
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const int pos = n2 + N2 * n1;
      if (pos >= a.M1) continue;
      const int owner = pos / rows, r = pos - owner * rows;
      if (!KDE_DCHECK(owner < kSlabC, KDE_DBG_SLAB)) continue;
      st_async(cluster_addr(hb, (unsigned)owner) + (unsigned)(r * a.Q + col) * 8u, x[n1],
               cluster_addr_u32(bar, (unsigned)owner));
    }
  }
}

// Row inverse phase B: thread (b, k1), full line Z = X + i Y rebuilt from the
// pair's half spectra in this block's buffer, inverse N2-point DFT.
template <int N2>
__device__ __forceinline__ void slab_irows_b(const SlabArgs& a, int c, const float2* hb, float2* ex) {
  const int N1 = a.lr.N1, P = a.lr.P;
  for (int t = threadIdx.x; t < a.RP * N1; t += blockDim.x) {
    const int b = t / N1, k1 = t - b * N1;
    const int r0 = 2 * (c * a.RP + b);
    const bool two = r0 + 1 < a.M1;
    const float2* x0 = hb + 2 * b * a.Q;
    const float2* x1 = x0 + a.Q;
    float2 y[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const int k = k1 + N1 * k2;
      const bool lo = k < a.Q;
      const int kk = lo ? k : P - k;
      const float2 X = x0[kk];
      const float2 Y = two ? x1[kk] : make_float2(0.f, 0.f);
      y[k2] = lo ? make_float2(X.x - Y.y, X.y + Y.x) : make_float2(X.x + Y.y, Y.x - X.y);
    }
    b_inv_store<N2>(y, k1, a.twr, ex + b * (N1 * a.SKr) + k1 * a.SKr, 1);
  }
}

// Row inverse phase A: thread (b, n2), rows r0, r0 + 1 cropped to M2.
template <int N1>
__device__ __forceinline__ void slab_irows_a(const SlabArgs& a, int c, int64_t i, const float2* ex) {
  const int N2 = a.lr.N2;
  for (int t = threadIdx.x; t < a.RP * N2; t += blockDim.x) {
    const int b = t / N2, n2 = t - b * N2;
    const int r0 = 2 * (c * a.RP + b);
    if (r0 >= a.M1) continue;
    const bool two = r0 + 1 < a.M1;
    const float2* src = ex + b * (N1 * a.SKr) + n2;
    float2 x[N1];
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) x[k1] = src[k1 * a.SKr];
    idft<N1>(x);
    float* o0 = a.out_real + (i * a.M1 + r0) * (int64_t)a.M2;
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      const int pos = n2 + N2 * n1;
      if (pos < a.M2) {
        o0[pos] = x[n1].x;
        if (two) o0[a.M2 + pos] = x[n1].y;
      }
    }
  }
}

template <int CLS, int N1T, int N2T>
__global__ void __launch_bounds__(kSlabThreads, 2) kde_fx_slab_inv_kernel(SlabArgs a) {
  pdl_trigger();
  extern __shared__ float2 fx_sm[];
  const unsigned bar = (unsigned)__cvta_generic_to_shared(fx_sm);
  float2* ex = fx_sm + 2;
  float2* hb = ex + a.ex_elems;
  const int c = (int)cluster_rank();
  const int64_t i = blockIdx.x / kSlabC;
  if (threadIdx.x == 0) mbar_init_cluster(bar);
  cluster_arrive_relaxed();
  pdl_wait();
  size_call<N2T, CLS>(a.lc.N2, [&](auto N) { slab_icols_b<decltype(N)::value>(a, c, i, ex); });
  __syncthreads();
  if (threadIdx.x == 0) {  // all Q columns of this block's kept rows
    const int nr = min(2 * a.RP, max(0, a.M1 - 2 * a.RP * c));
    mbar_expect(bar, (unsigned)(nr * a.Q) * 8u);
  }
  cluster_wait();  // every block of the cluster is running, its barrier initialised
  size_call<N1T, CLS>(a.lc.N1, [&](auto N) { slab_icols_a<decltype(N)::value>(a, c, ex, hb, bar); });
  cluster_arrive_relaxed();  // this block's stores are issued
  if (!mbar_wait_cluster(bar, kWaitLimit) && threadIdx.x == 0) atomicExch(a.status, 1);
  size_call<N2T, CLS>(a.lr.N2, [&](auto N) { slab_irows_b<decltype(N)::value>(a, c, hb, ex); });
  __syncthreads();
  size_call<N1T, CLS>(a.lr.N1, [&](auto N) { slab_irows_a<decltype(N)::value>(a, c, i, ex); });
  cluster_wait();  // no block leaves while stores to it may be outstanding
}

// Launch with a cluster of kSlabC blocks along x, as a programmatic
// dependent of the kernel before it on the stream.
template <typename Kern>
cudaError_t launch_slab(Kern* fn, const Launch& l, const SlabArgs& a) {
  cudaError_t e = allow_smem(fn);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = l.grid;
  cfg.blockDim = dim3(l.threads);
  cfg.dynamicSmemBytes = l.smem;
  cfg.stream = l.st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kSlabC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  e = cudaLaunchKernelEx(&cfg, fn, a);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t launch_slab_fwd(const Launch& l, const SlabArgs& a);
cudaError_t launch_slab_inv(const Launch& l, const SlabArgs& a);

}  // namespace fx
}  // namespace kde
