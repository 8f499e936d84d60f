// Bounds-checked debug builds (compile with -DKDE_DEBUG; build(debug=True)
// makes libkde_gb300_debug.so).  KDE_DCHECK(cond, code) is true when cond
// holds; when it does not, a debug build records code in this translation
// unit's device word (the first failure wins) and the caller skips the
// access, so an out-of-range index is reported instead of faulting.  A
// release build compiles every check to true.  kde_debug_status reads (and
// clears) the words of all translation units.
#pragma once

#include <cuda_runtime.h>

#ifdef KDE_DEBUG
#define KDE_DEBUG_ENABLED 1
static __device__ int kde_debug_word;
#define KDE_DCHECK(cond, code) ((cond) ? true : (atomicCAS(&kde_debug_word, 0, (code)), false))
#define KDE_DEBUG_READER(name)                                            \
  namespace kde {                                                         \
  int debug_read_##name() {                                               \
    int v = 0, z = 0;                                                     \
    if (cudaMemcpyFromSymbol(&v, kde_debug_word, sizeof(int)) != cudaSuccess) return -1; \
    if (v) cudaMemcpyToSymbol(kde_debug_word, &z, sizeof(int));           \
    return v;                                                             \
  }                                                                       \
  }
#else
#define KDE_DEBUG_ENABLED 0
#define KDE_DCHECK(cond, code) true
#define KDE_DEBUG_READER(name) \
  namespace kde {              \
  int debug_read_##name() { return 0; } \
  }
#endif

// Codes recorded by the checks (which kernel found an index out of range).
enum {
  KDE_DBG_BIN_DIRECT = 1,
  KDE_DBG_BIN_ACCUM = 2,
  KDE_DBG_BIN_SCATTER = 3,
  KDE_DBG_ROWS_STORE = 4,
  KDE_DBG_COLS_STORE = 5,
  KDE_DBG_COLS_LOAD = 6,
  KDE_DBG_STOCKHAM = 7,
  KDE_DBG_SLAB = 8
};
