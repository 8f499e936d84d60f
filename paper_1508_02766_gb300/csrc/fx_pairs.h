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

}  // namespace fxp
}  // namespace kde
