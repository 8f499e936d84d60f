"""Plain FP64 CPU oracle for binned FFT kernel density estimation with an
unconstrained bandwidth matrix (Gramacki & Gramacki, arXiv 1508.02766).

TEST INFRASTRUCTURE ONLY.  This module is the independent reference the CUDA
path is checked against: only the test suite, the package's smoke check and the benchmark's CPU
baseline may import it.  It shares no code, tables or helpers with the CUDA
library and never imports it.

It is slow on purpose.  Every function states the passage it follows and does
what that passage says, in its order, with no blocking or fusion:

* ``scaled_gaussian``      -- K_H of Eq. 1 with the standard normal kernel.
* ``binwidths``            -- Eq. 4.
* ``support_L``            -- Eq. 15 (corrected range) and the per-axis range.
* ``bin_linear``           -- linear binning (Sec. 2, first step) under the
                              exact integer rounding spec stated below.
* ``kernel_weights``       -- k_l of Eq. 6 on the lags |l_k| <= L_k.
* ``binned_direct``        -- the truncated binned estimator, Eq. 7 (O2).
* ``binned_direct_at``     -- the same at chosen grid nodes.
* ``fft_corrected``        -- Eq. 10 with the corrected layouts Eq. 12-14 (O3).
* ``fft_wand``             -- Eq. 10 with Wand's layouts Eq. 8, 9, 11 (O3).
* ``direct_kde``           -- the unbinned estimator, Eq. 1 (O1).

Readings of passages the paper leaves open (each pinned by a test):

* Eq. 12 prints lags +-M_k, but Eq. 5 sums over +-(M_k-1) and the crop of
  Eq. 14 with c_{1,1} at row M_1 is consistent only with lags +-(M_k-1);
  after Eq. 15 the lags run over +-L_k.  The count offset stays M_k - 1
  (Eq. 13) and the crop starts at 0-based index L_k + M_k - 1, which is
  Eq. 14's (2M_k-1) (1-based) when L_k = M_k - 1.
* Eq. 8 repeats the index-M_k row/column; Wand's layout is read as k_{|l|}
  at the wrapped position l mod P_k for |l_k| <= L_k.
* Eq. 15's |lambda| is the largest eigenvalue of H; tau defaults to 3.7 for
  every d; the per-axis ("Wand") range is ceil(tau sqrt(H_kk) / delta_k).
* Binning rounding spec (the paper gives none; Sec. 3 footnote only requires
  the counts to sum to n):  per axis, t = (x - lo) * s in the dtype of X with
  s = (M-1)/(hi-lo) computed in FP64 then rounded to that dtype, lo rounded to
  that dtype, no fused multiply-add.  A sample with t < 0, t > M-1 or NaN on
  any axis is dropped and counted.  i = floor(t), f = t - i; a sample at
  t = M-1 goes to i = M-2, f = 1.  Q = round-half-even(f * 2^32) in FP64.
  The unit mass W = 2^32 is split axis by axis (axis 0 first): each part w
  gives w_hi = floor((w*Q + 2^31) / 2^32) to node i+1 and w - w_hi to node i.
  The 2^d corner weights are integers summing to exactly 2^32; counts are
  int64 in units of 2^-32.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

TWO32 = 1 << 32


# ----------------------------------------------------------------------------
# Eq. 1: the scaled kernel K_H(u) = |H|^{-1/2} K(H^{-1/2} u), K standard normal.
# ----------------------------------------------------------------------------
def scaled_gaussian(U, H):
    """K_H(u) for each row u of U (Eq. 1, standard multivariate normal K).

    K(H^{-1/2} u) = (2 pi)^{-d/2} exp(-u^T H^{-1} u / 2), times |H|^{-1/2}.
    """
    H = np.asarray(H, dtype=np.float64)
    U = np.atleast_2d(np.asarray(U, dtype=np.float64))
    d = H.shape[0]
    Hinv = np.linalg.inv(H)
    quad = np.einsum("ni,ij,nj->n", U, Hinv, U)
    return (2.0 * np.pi) ** (-d / 2.0) * np.linalg.det(H) ** -0.5 * np.exp(-0.5 * quad)


# ----------------------------------------------------------------------------
# Eq. 3-4: grid nodes and binwidths.
# ----------------------------------------------------------------------------
def binwidths(lo, hi, M):
    """delta_k = (g_{k M_k} - g_{k 1}) / (M_k - 1)   (Eq. 4)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    M = np.asarray(M, dtype=np.int64)
    return (hi - lo) / (M - 1)


def grid_axes(lo, hi, M):
    """g_{k j} = g_{k 1} + (j-1) delta_k, j = 1..M_k (Eq. 3 with Eq. 4)."""
    delta = binwidths(lo, hi, M)
    return [lo[k] + delta[k] * np.arange(M[k]) for k in range(len(M))]


# ----------------------------------------------------------------------------
# Eq. 15: effective support.
# ----------------------------------------------------------------------------
def support_L(H, lo, hi, M, tau=3.7, range_mode="corrected"):
    """L_k = min(M_k - 1, ceil(tau sqrt(|lambda|) / delta_k))   (Eq. 15).

    lambda is the largest eigenvalue of H.  range_mode="per_axis" gives the
    axis-aligned range ceil(tau sqrt(H_kk) / delta_k) used for comparison.
    """
    H = np.asarray(H, dtype=np.float64)
    delta = binwidths(lo, hi, M)
    if range_mode == "corrected":
        lam = float(np.max(np.linalg.eigvalsh(H)))
        half = np.full(len(M), tau * math.sqrt(abs(lam)))
    elif range_mode == "per_axis":
        half = tau * np.sqrt(np.diag(H))
    else:
        raise ValueError(range_mode)
    L = [min(int(M[k]) - 1, int(math.ceil(half[k] / delta[k]))) for k in range(len(M))]
    return tuple(L)


# ----------------------------------------------------------------------------
# Linear binning (Sec. 2, first step) under the exact rounding spec above.
# ----------------------------------------------------------------------------
def _mulhi_round(w, Q):
    """floor((w*Q + 2^31) / 2^32) for uint64 arrays 0 <= w, Q <= 2^32, exactly.

    w*Q can reach 2^64, so Q is split as Qh*2^16 + Ql:
    (w*Q + 2^31) >> 32 = ((w*Qh) + ((w*Ql + 2^31) >> 16)) >> 16.
    """
    w = w.astype(np.uint64)
    Q = Q.astype(np.uint64)
    Qh = Q >> np.uint64(16)
    Ql = Q & np.uint64(0xFFFF)
    A = w * Qh
    B = w * Ql + np.uint64(1 << 31)
    return (A + (B >> np.uint64(16))) >> np.uint64(16)


def bin_positions(X, lo, hi, M):
    """Per-sample node index i (n x d), fixed-point fraction Q, inside mask."""
    X = np.asarray(X)
    dt = X.dtype.type
    if X.dtype not in (np.float32, np.float64):
        raise TypeError("X must be float32 or float64")
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    M = np.asarray(M, dtype=np.int64)
    s = (M - 1).astype(np.float64) / (hi - lo)
    lo_t = lo.astype(dt)
    s_t = s.astype(dt)
    with np.errstate(invalid="ignore"):
        t = (X - lo_t) * s_t                      # two rounded ops in X's dtype
        inside = np.all((t >= 0) & (t <= (M - 1).astype(dt)), axis=1)
    t = t[inside]
    i = np.floor(t).astype(np.int64)
    f = t - i.astype(dt)                          # exact
    top = i == (M - 1)
    i = np.where(top, M - 2, i)
    f = np.where(top, dt(1.0), f)
    Q = np.rint(f.astype(np.float64) * float(TWO32)).astype(np.uint64)
    return i, Q, inside


def corner_weights(Q):
    """Integer weights of the 2^d corners, axis 0 split first (rounding spec).

    Returns (n x 2^d) uint64; corner c has offset bit (c >> (d-1-k)) & 1 on axis k.
    """
    n, d = Q.shape
    parts = np.full((n, 1), TWO32, dtype=np.uint64)
    for k in range(d):
        w_hi = _mulhi_round(parts, Q[:, k:k + 1])
        w_lo = parts - w_hi
        parts = np.stack([w_lo, w_hi], axis=2).reshape(n, -1)
    return parts


def bin_linear(X, lo, hi, M):
    """Linear binning: counts c_l (int64, units of 2^-32) and the number of
    samples dropped as outside [lo, hi].  sum(counts) == (n - n_out) * 2^32."""
    M = tuple(int(m) for m in M)
    d = len(M)
    i, Q, inside = bin_positions(X, lo, hi, M)
    w = corner_weights(Q)
    strides = np.array([int(np.prod(M[k + 1:])) for k in range(d)], dtype=np.int64)
    counts = np.zeros(int(np.prod(M)), dtype=np.int64)
    for c in range(1 << d):
        off = np.array([(c >> (d - 1 - k)) & 1 for k in range(d)], dtype=np.int64)
        flat = (i + off) @ strides
        np.add.at(counts, flat, w[:, c].astype(np.int64))
    return counts.reshape(M), int(np.count_nonzero(~inside))


def counts_to_c(counts):
    """Grid counts c_l in sample units (FP64)."""
    return counts.astype(np.float64) * 2.0 ** -32


# ----------------------------------------------------------------------------
# Eq. 6: kernel weights on the lag lattice.
# ----------------------------------------------------------------------------
def kernel_weights(H, lo, hi, M, L, n, layout="corrected"):
    """k_l = (1/n) K_H(delta_1 l_1, ..., delta_d l_d) for |l_k| <= L_k (Eq. 6).

    Returned as an array of shape (2L_1+1, ..., 2L_d+1), index l_k + L_k.
    layout="wand" gives what Wand's layout (Eq. 8) actually convolves with:
    k_{|l_1|, ..., |l_d|} at lag l.
    """
    delta = binwidths(lo, hi, M)
    axes = [np.arange(-Lk, Lk + 1) for Lk in L]
    lags = np.array(list(itertools.product(*axes)), dtype=np.float64)
    if layout == "wand":
        lags = np.abs(lags)
    elif layout != "corrected":
        raise ValueError(layout)
    k = scaled_gaussian(lags * delta, H) / n
    return k.reshape([2 * Lk + 1 for Lk in L])


# ----------------------------------------------------------------------------
# O2: Eq. 7, the truncated binned estimator, by direct summation.
# ----------------------------------------------------------------------------
def binned_direct(c, k, L):
    """f_j = sum_{|l_k| <= L_k} c_{j-l} k_l, c zero outside the grid (Eq. 7)."""
    c = np.asarray(c, dtype=np.float64)
    M = c.shape
    d = len(M)
    f = np.zeros(M)
    for lag in itertools.product(*[range(-Lk, Lk + 1) for Lk in L]):
        w = k[tuple(lk + Lk for lk, Lk in zip(lag, L))]
        dst, src = [], []
        for kk in range(d):
            a = max(0, lag[kk])               # j_k with 0 <= j_k - l_k < M_k
            b = min(M[kk], M[kk] + lag[kk])
            if a >= b:
                break
            dst.append(slice(a, b))
            src.append(slice(a - lag[kk], b - lag[kk]))
        else:
            f[tuple(dst)] += w * c[tuple(src)]
    return f


def binned_direct_at(c, k, L, nodes, chunk=512):
    """Eq. 7 at chosen nodes j (m x d, 0-based), by the same sum per node."""
    c = np.asarray(c, dtype=np.float64)
    d = c.ndim
    L = tuple(L)
    cpad = np.pad(c, [(Lk, Lk) for Lk in L])
    win = np.lib.stride_tricks.sliding_window_view(cpad, [2 * Lk + 1 for Lk in L])
    kflip = k[(slice(None, None, -1),) * d]   # window offset m <-> lag L - m
    nodes = np.asarray(nodes, dtype=np.int64)
    out = np.empty(len(nodes))
    for s in range(0, len(nodes), chunk):
        J = nodes[s:s + chunk]
        W = win[tuple(J[:, kk] for kk in range(d))]
        out[s:s + chunk] = np.tensordot(W, kflip, axes=d)
    return out


# ----------------------------------------------------------------------------
# Eq. 10: discrete convolution theorem with a plain DFT.
# ----------------------------------------------------------------------------
def dft_matrix(P, sign):
    """W[a, b] = exp(sign * 2 pi i (a b mod P) / P), the angle reduced exactly."""
    a = np.arange(P, dtype=np.int64)
    ang = 2.0 * np.pi * (np.outer(a, a) % P) / P
    return np.cos(ang) + 1j * sign * np.sin(ang)


def dftn(a, sign):
    """Separable multi-dimensional DFT (unnormalised), one axis at a time."""
    out = np.asarray(a, dtype=np.complex128)
    for ax in range(out.ndim):
        W = dft_matrix(out.shape[ax], sign)
        out = np.moveaxis(np.tensordot(W, out, axes=([1], [ax])), 0, ax)
    return out


def convolve_by_dft(c_pad, k_pad):
    """C = F(c), K = F(k), S = C K, s = F^{-1}(S) unnormalised (Eq. 10)."""
    C = dftn(c_pad, -1)
    K = dftn(k_pad, -1)
    S = C * K
    return dftn(S, +1)


def _next_pow2(x):
    p = 1
    while p < x:
        p *= 2
    return p


def fft_corrected(c, k, L, P=None):
    """O3, corrected algorithm: layouts Eq. 12-13, Eq. 10, crop Eq. 14.

    k_new holds every signed lag -L_k..L_k starting at index 0, c_new holds
    c_{1..M} starting at 0-based index M_k - 1 (c_{1,1} in row M_1), and the
    estimate is s[L_k + M_k - 1 : L_k + 2 M_k - 1] / prod(P) per axis.
    Without wrap-around P_k >= 2 M_k - 1 + L_k; default: the next power of 2.
    """
    c = np.asarray(c, dtype=np.float64)
    M = c.shape
    d = len(M)
    if P is None:
        P = tuple(_next_pow2(2 * M[kk] - 1 + L[kk]) for kk in range(d))
    for kk in range(d):
        if P[kk] < 2 * M[kk] - 1 + L[kk]:
            raise ValueError("P too small for the corrected layout")
    k_new = np.zeros(P)
    k_new[tuple(slice(0, 2 * Lk + 1) for Lk in L)] = k
    c_new = np.zeros(P)
    c_new[tuple(slice(M[kk] - 1, 2 * M[kk] - 1) for kk in range(d))] = c
    s = convolve_by_dft(c_new, k_new)
    crop = tuple(slice(L[kk] + M[kk] - 1, L[kk] + 2 * M[kk] - 1) for kk in range(d))
    return s[crop].real / float(np.prod(P)), s[crop].imag / float(np.prod(P))


def fft_wand(c, k_abs, L, P=None):
    """O3, Wand's algorithm: layouts Eq. 8-9, Eq. 10, crop Eq. 11.

    k_abs[a] = k_{a_1..a_d} for 0 <= a_k <= L_k (first quadrant only).  The
    kernel array holds k_{|l|} at wrapped position l mod P_k; counts start at
    the origin; the estimate is s[0:M_k] / prod(P).  P_k >= M_k + L_k.
    """
    c = np.asarray(c, dtype=np.float64)
    M = c.shape
    d = len(M)
    if P is None:
        P = tuple(_next_pow2(M[kk] + L[kk]) for kk in range(d))
    for kk in range(d):
        if P[kk] < M[kk] + L[kk]:
            raise ValueError("P too small for Wand's layout")
    k_w = np.zeros(P)
    for pos in itertools.product(*[list(range(0, Lk + 1)) + list(range(Pk - Lk, Pk))
                                   for Lk, Pk in zip(L, P)]):
        a = tuple(p if p <= Lk else Pk - p for p, Lk, Pk in zip(pos, L, P))
        k_w[pos] = k_abs[a]
    c_w = np.zeros(P)
    c_w[tuple(slice(0, m) for m in M)] = c
    s = convolve_by_dft(c_w, k_w)
    crop = tuple(slice(0, m) for m in M)
    return s[crop].real / float(np.prod(P)), s[crop].imag / float(np.prod(P))


# ----------------------------------------------------------------------------
# O1: Eq. 1, the unbinned estimator.
# ----------------------------------------------------------------------------
def direct_kde(X, H, points, chunk=256):
    """f(x) = (1/n) sum_i K_H(x - X_i) at each row x of points (Eq. 1)."""
    X = np.asarray(X, dtype=np.float64)
    points = np.atleast_2d(np.asarray(points, dtype=np.float64))
    H = np.asarray(H, dtype=np.float64)
    d = H.shape[0]
    Hinv = np.linalg.inv(H)
    norm = (2.0 * np.pi) ** (-d / 2.0) * np.linalg.det(H) ** -0.5
    out = np.empty(len(points))
    for s in range(0, len(points), chunk):
        D = points[s:s + chunk, None, :] - X[None, :, :]
        quad = np.einsum("pni,ij,pnj->pn", D, Hinv, D)
        out[s:s + chunk] = norm * np.exp(-0.5 * quad).mean(axis=1)
    return out


# ----------------------------------------------------------------------------
# The full plain pipeline: bin, weigh, sum (Sec. 2, steps one to three).
# ----------------------------------------------------------------------------
def binned_estimate(X, H, lo, hi, M, tau=3.7, range_mode="corrected",
                    layout="corrected", nodes=None):
    """Bin X, form k_l over the Eq. 15 support and evaluate Eq. 7.

    Returns (f, counts, L, n_out); f is the full grid or, if nodes is given,
    the values at those nodes.
    """
    counts, n_out = bin_linear(X, lo, hi, M)
    L = support_L(H, lo, hi, M, tau, range_mode)
    n = len(X)
    k = kernel_weights(H, lo, hi, M, L, n, layout)
    c = counts_to_c(counts)
    f = binned_direct(c, k, L) if nodes is None else binned_direct_at(c, k, L, nodes)
    return f, counts, L, n_out


# ----------------------------------------------------------------------------
# Bandwidth selection by least-squares cross-validation on the binned data.
# The paper states (Sec. 1 and Sec. 5) that the same FFT machinery computes
# the functionals needed for fast bandwidth selection; the criterion below is
# the textbook LSCV for a Gaussian kernel, with every double sum over samples
# replaced by the binned double sum the FFT evaluates (Eq. 2 / Eq. 7 form).
# ----------------------------------------------------------------------------
def binned_pair_sum(c, A, lo, hi, M, L):
    """S(A) = sum_j c_j sum_{|l_k| <= L_k} c_{j-l} K_A(delta o l): the binned
    counterpart of sum_{i,j} K_A(X_i - X_j)."""
    k = kernel_weights(A, lo, hi, M, L, n=1)
    return float(np.sum(np.asarray(c, dtype=np.float64) * binned_direct(c, k, L)))


def lscv_binned(counts, n, H, lo, hi, M, tau=3.7):
    """LSCV(H) = (1/n^2) S(2H) - 2 (S(H) - n K_H(0)) / (n (n-1)).

    The first term is the integral of the squared estimate (K_H * K_H =
    K_{2H} for Gaussian kernels); the second is the leave-one-out term, whose
    i = j pairs contribute n K_H(0) to S(H).  Each S uses the support L of
    its own matrix (Eq. 15).
    """
    H = np.asarray(H, dtype=np.float64)
    c = counts_to_c(counts)
    L2 = support_L(2.0 * H, lo, hi, M, tau)
    L1 = support_L(H, lo, hi, M, tau)
    S2 = binned_pair_sum(c, 2.0 * H, lo, hi, M, L2)
    S1 = binned_pair_sum(c, H, lo, hi, M, L1)
    K0 = float(scaled_gaussian(np.zeros((1, H.shape[0])), H)[0])
    return S2 / n**2 - 2.0 * (S1 - n * K0) / (n * (n - 1.0))


def lscv_exact(X, H):
    """The unbinned LSCV criterion by direct O(n^2) sums over the samples."""
    X = np.asarray(X, dtype=np.float64)
    H = np.asarray(H, dtype=np.float64)
    n = len(X)
    D = (X[:, None, :] - X[None, :, :]).reshape(-1, X.shape[1])
    S2 = float(np.sum(scaled_gaussian(D, 2.0 * H)))
    S1 = float(np.sum(scaled_gaussian(D, H)))
    K0 = float(scaled_gaussian(np.zeros((1, X.shape[1])), H)[0])
    return S2 / n**2 - 2.0 * (S1 - n * K0) / (n * (n - 1.0))


def binned_pair_sum_dft(c, A, lo, hi, M, L, P):
    """S(A) by Eq. 10 and Parseval: counts zero-padded to P at the origin,
    K_A(delta o l) at wrapped index l mod P (all signed lags), then
    (1/prod P) sum_w |C(w)|^2 K(w).  Equals binned_pair_sum when P_k >= M_k + L_k."""
    c = np.asarray(c, dtype=np.float64)
    d = c.ndim
    k = kernel_weights(A, lo, hi, M, L, n=1)
    kw = np.zeros(P)
    for lag in itertools.product(*[range(-Lk, Lk + 1) for Lk in L]):
        kw[tuple(l % Pk for l, Pk in zip(lag, P))] = k[tuple(l + Lk for l, Lk in zip(lag, L))]
    cp = np.zeros(P)
    cp[tuple(slice(0, m) for m in M)] = c
    C = dftn(cp, -1)
    K = dftn(kw, -1)
    return float(np.sum(np.abs(C) ** 2 * K.real)) / float(np.prod(P))
