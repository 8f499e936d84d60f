// Line splits P = N1 x N2 of the two-phase engine that have kernels compiled
// for exactly that split (straight-line code for two DFT sizes only, which
// keeps each kernel's instructions cached).  Lengths up to 400 also run on
// generic kernels for any split with N1, N2 <= 20; above 400 the planner takes
// the smallest length from this list (spaced by at most 12%).  Plain C++,
// shared by the planner and the launchers.
#pragma once

#define KDE_FX_PAIRS(X)                                                                    \
  X(16, 16) X(14, 20) X(16, 20) X(18, 20) X(20, 20) X(16, 28) X(20, 24) X(16, 32) X(20, 28) \
  X(24, 24) X(20, 32) X(24, 28) X(24, 30) X(24, 32) X(25, 32) X(24, 36) X(30, 30) X(30, 32) \
  X(32, 32) X(30, 36) X(32, 36) X(30, 40) X(32, 40) X(36, 36) X(36, 40) X(40, 40)

namespace kde {
namespace fxp {

struct Pair {
  int N1, N2;
};

#define KDE_FX_PAIR_ENTRY(a, b) Pair{a, b},
inline constexpr Pair kPairs[] = {KDE_FX_PAIRS(KDE_FX_PAIR_ENTRY)};
#undef KDE_FX_PAIR_ENTRY
inline constexpr int kNumPairs = sizeof(kPairs) / sizeof(kPairs[0]);
inline constexpr int kGenericMax = 20;     // generic kernels: N1, N2 <= 20
inline constexpr int kGenericMaxP = 400;

}  // namespace fxp
}  // namespace kde
