// Line splits of the two-phase engine that have kernels compiled for exactly
// that split (straight-line code for its DFT sizes only, which keeps each
// kernel's instructions cached).  Lengths up to 400 run on two factors: the
// listed pairs, or generic kernels for any split with N1, N2 <= 20.  Longer
// lines take the smallest listed three-factor length.  Plain C++, shared by
// the planner and the launchers.
#pragma once

#define KDE_FX_PAIRS(X) X(16, 16) X(14, 20) X(16, 20) X(18, 20) X(20, 20)

// Three-factor splits P = N1 N2 N3 for lines longer than 400 (three-phase
// kernels, each compiled for its split), spaced by at most 12%.
#define KDE_FX_TRIPLES(X)                                                                     \
  X(7, 8, 8) X(6, 8, 10) X(8, 8, 8) X(7, 8, 10) X(8, 8, 9) X(8, 8, 10) X(7, 8, 12) X(8, 9, 10) \
  X(8, 8, 12) X(8, 10, 10) X(8, 9, 12) X(9, 10, 10) X(8, 10, 12) X(8, 8, 16) X(9, 10, 12)      \
  X(8, 12, 12) X(10, 10, 12) X(8, 10, 16) X(9, 12, 12) X(10, 12, 12) X(10, 10, 16)             \
  X(12, 12, 12) X(10, 12, 16) X(8, 16, 16)

namespace kde {
namespace fxp {

struct Pair {
  int N1, N2;
};

struct Triple {
  int N1, N2, N3;
};

#define KDE_FX_PAIR_ENTRY(a, b) Pair{a, b},
inline constexpr Pair kPairs[] = {KDE_FX_PAIRS(KDE_FX_PAIR_ENTRY)};
#undef KDE_FX_PAIR_ENTRY
inline constexpr int kNumPairs = sizeof(kPairs) / sizeof(kPairs[0]);
#define KDE_FX_TRIPLE_ENTRY(a, b, c) Triple{a, b, c},
inline constexpr Triple kTriples[] = {KDE_FX_TRIPLES(KDE_FX_TRIPLE_ENTRY)};
#undef KDE_FX_TRIPLE_ENTRY
inline constexpr int kNumTriples = sizeof(kTriples) / sizeof(kTriples[0]);
inline constexpr int kGenericMax = 20;     // generic kernels: N1, N2 <= 20
inline constexpr int kGenericMaxP = 400;

// Slab passes (3-D): the last two axes of one slab on a cluster of kSlabC
// blocks.  Block c takes row pairs [c RP, (c + 1) RP) of the slab's M1 rows
// and half-spectrum columns [c W, (c + 1) W) of Q; its shared memory is an
// mbarrier (16 bytes), an exchange region of ex_elems complex entries (RP
// lines of N1r x SKr for the rows, N1c x SKc for the columns, SKc = W
// (mod 16) so that phase-B reads across k1 are conflict-free) and a cluster
// buffer ([M1][W] forward, [2 RP][Q] inverse).  Blocks have up to kSlabMaxThreads threads, each
// looping over its tasks of a phase (row pairs x N, columns x N).  sr, sc:
// the splits {N1, N2, N3} of axes 2 and 1.
inline constexpr int kSlabC = 8;
inline constexpr int kSlabMaxThreads = 384;
inline constexpr long long kSlabMaxSmem = 113 * 1024;  // two blocks per SM

struct SlabGeo {
  int RP, W, SKr, SKc, ex_elems, threads;
  long long smem_fwd, smem_inv;
  bool ok;
};

inline SlabGeo slab_geometry(long long M1, long long Q, const int* sr, const int* sc) {
  SlabGeo g{};
  if (sr[2] || sc[2] || sr[0] < 2 || sc[0] < 2) return g;
  if (sr[0] > kGenericMax || sr[1] > kGenericMax || sc[0] > kGenericMax || sc[1] > kGenericMax)
    return g;
  g.RP = (int)(((M1 + 1) / 2 + kSlabC - 1) / kSlabC);
  g.W = (int)((Q + kSlabC - 1) / kSlabC);
  g.SKr = sr[1] | 1;
  int skc = g.W * sc[1];
  while (skc % 16 != g.W % 16) ++skc;
  g.SKc = skc;
  const long long exr = (long long)g.RP * sr[0] * g.SKr, exc = (long long)sc[0] * g.SKc;
  g.ex_elems = (int)(exr > exc ? exr : exc);
  const int tr = g.RP * (sr[0] > sr[1] ? sr[0] : sr[1]);
  const int tc = g.W * (sc[0] > sc[1] ? sc[0] : sc[1]);
  g.threads = ((tr > tc ? tr : tc) + 31) / 32 * 32;  // threads loop over the tasks above this
  if (g.threads > kSlabMaxThreads) g.threads = kSlabMaxThreads;
  g.smem_fwd = 16 + (g.ex_elems + M1 * g.W) * 8;  // mbarrier, exchange, cluster buffer
  g.smem_inv = 16 + (g.ex_elems + 2LL * g.RP * Q) * 8;
  g.ok = g.smem_fwd <= kSlabMaxSmem && g.smem_inv <= kSlabMaxSmem;
  return g;
}

}  // namespace fxp
}  // namespace kde
