"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-worked
values, closed forms, textbook or library formulas, invariants the paper
states, or brute force on tiny inputs.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.stats import multivariate_normal

from oracle import kde_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def random_spd(rng, d, scale):
    A = rng.standard_normal((d, d))
    return scale * (A @ A.T / d + 0.3 * np.eye(d))


# --------------------------------------------------------------------------
# Binning (Sec. 2 first step; Sec. 3 footnote)
# --------------------------------------------------------------------------
def test_mulhi_round_matches_big_integers():
    rng = np.random.default_rng(0)
    w = rng.integers(0, 1 << 32, size=20000, dtype=np.uint64)
    Q = rng.integers(0, 1 << 32, size=20000, dtype=np.uint64)
    edge = np.array([0, 1, (1 << 31), (1 << 32) - 1, 1 << 32], dtype=np.uint64)
    w = np.concatenate([w, np.repeat(edge, len(edge))])
    Q = np.concatenate([Q, np.tile(edge, len(edge))])
    got = O._mulhi_round(w, Q)
    want = [(int(a) * int(b) + (1 << 31)) >> 32 for a, b in zip(w, Q)]
    assert [int(x) for x in got] == want


def test_binning_worked_examples():
    with open(os.path.join(GOLDEN, "binning_worked.json")) as fh:
        cases = json.load(fh)["cases"]
    for case in cases:
        X = np.array(case["X"], dtype=case["dtype"])
        counts, n_out = O.bin_linear(X, case["lo"], case["hi"], case["M"])
        assert n_out == case["n_outside"]
        flat = counts.ravel()
        if "counts" in case:
            assert flat.tolist() == case["counts"]
        else:
            want = np.zeros_like(flat)
            for idx, v in case["counts_nonzero"].items():
                want[int(idx)] = v
            assert flat.tolist() == want.tolist()


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_binning_mass_is_exact(d, dtype):
    """P1: sum of counts equals (n - n_outside) * 2^32 exactly."""
    rng = np.random.default_rng(10 + d)
    n = 5000
    X = rng.uniform(-0.2, 1.2, size=(n, d)).astype(dtype)
    X[:7, 0] = np.nan
    X[7:12] = 1.0                                   # exactly at hi
    M = [7, 5, 4][:d]
    counts, n_out = O.bin_linear(X, [0.0] * d, [1.0] * d, M)
    inside = np.all((X >= 0) & (X <= 1), axis=1)    # spec is looser only by rounding
    assert n_out == n - int(counts.sum() >> 32)
    assert int(counts.sum()) == (n - n_out) * (1 << 32)
    assert abs(n_out - int(np.count_nonzero(~inside))) <= 2
    assert counts.min() >= 0


@pytest.mark.parametrize("d", [1, 2, 3])
def test_binning_weights_close_to_exact_products(d):
    """Each corner weight is within d units of 2^32 prod_k (1-f_k or f_k),
    with f taken exactly from the rounded position (brute force, Fractions)."""
    rng = np.random.default_rng(20 + d)
    X = rng.uniform(0, 1, size=(40, d))
    M = [6, 9, 5][:d]
    lo, hi = np.zeros(d), np.ones(d)
    for x in X:
        counts, _ = O.bin_linear(x[None, :], lo, hi, M)
        s = (np.array(M) - 1) / (hi - lo)
        t = [Fraction(float((x[k] - lo[k]) * s[k])) for k in range(d)]
        base = [int(math.floor(tk)) for tk in t]
        for off in itertools.product([0, 1], repeat=d):
            w = Fraction(1)
            for k in range(d):
                fk = t[k] - base[k]
                w *= fk if off[k] else (1 - fk)
            node = tuple(base[k] + off[k] for k in range(d))
            assert abs(int(counts[node]) - w * (1 << 32)) <= d


def test_binning_preserves_first_moment():
    """Linear binning keeps sum_l c_l g_l = sum_i X_i (up to 2^-32 quantisation)."""
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 2, size=(3000, 2))
    lo, hi, M = [-1.0, -1.0], [2.0, 2.0], [31, 17]
    counts, n_out = O.bin_linear(X, lo, hi, M)
    assert n_out == 0
    c = O.counts_to_c(counts)
    g0, g1 = O.grid_axes(np.array(lo), np.array(hi), M)
    m0 = (c.sum(axis=1) * g0).sum()
    m1 = (c.sum(axis=0) * g1).sum()
    assert abs(m0 - X[:, 0].sum()) < 1e-6
    assert abs(m1 - X[:, 1].sum()) < 1e-6


# --------------------------------------------------------------------------
# Eq. 1 and Eq. 15
# --------------------------------------------------------------------------
def test_scaled_gaussian_matches_bivariate_normal_formula():
    """K_H against the textbook correlated bivariate normal density."""
    s1, s2, rho = 0.3, 0.5, -0.8
    H = np.array([[s1 * s1, rho * s1 * s2], [rho * s1 * s2, s2 * s2]])
    rng = np.random.default_rng(4)
    U = rng.normal(size=(50, 2))
    z1, z2 = U[:, 0] / s1, U[:, 1] / s2
    want = np.exp(-(z1 * z1 - 2 * rho * z1 * z2 + z2 * z2) / (2 * (1 - rho * rho)))
    want /= 2 * np.pi * s1 * s2 * math.sqrt(1 - rho * rho)
    assert rel_max(O.scaled_gaussian(U, H), want) < 1e-13


def test_scaled_gaussian_3d_matches_scipy():
    rng = np.random.default_rng(5)
    H = random_spd(rng, 3, 0.2)
    U = rng.normal(size=(40, 3)) * 0.3
    want = multivariate_normal(mean=np.zeros(3), cov=H).pdf(U)
    assert rel_max(O.scaled_gaussian(U, H), want) < 1e-12


def test_support_L_hand_values():
    """Eq. 15 for H=[[.09,.07],[.07,.09]]: eigenvalues .16, .02 (a +- b), so
    tau sqrt(lambda) = 3.7*0.4 = 1.48; with delta = 0.1, L = ceil(14.8) = 15.
    Per-axis: 3.7*0.3/0.1 = 11.1 -> 12.  L is capped at M-1."""
    H = np.array([[0.09, 0.07], [0.07, 0.09]])
    lo, hi, M = [0.0, 0.0], [12.7, 12.7], [128, 128]
    assert O.support_L(H, lo, hi, M) == (15, 15)
    assert O.support_L(H, lo, hi, M, range_mode="per_axis") == (12, 12)
    assert O.support_L(H, [0.0, 0.0], [0.9, 12.7], [10, 128]) == (9, 15)


def test_support_L_isotropic_ranges_agree():
    """P9: for H = h^2 I both ranges give the same L."""
    for h in [0.05, 0.13, 0.4]:
        H = h * h * np.eye(3)
        lo, hi, M = [0, -1, 2], [3, 1, 7], [40, 50, 60]
        assert O.support_L(H, lo, hi, M) == O.support_L(H, lo, hi, M, range_mode="per_axis")


# --------------------------------------------------------------------------
# Eq. 10: the plain DFT
# --------------------------------------------------------------------------
@pytest.mark.parametrize("P", [1, 2, 7, 12, 30])
def test_dft_textbook_identities(P):
    """P10: F(delta) = 1, F(exp(2 pi i m n / P)) = P delta_{k m},
    F^{-1} F = P I, Parseval."""
    e0 = np.zeros(P)
    e0[0] = 1
    assert np.allclose(O.dftn(e0, -1), np.ones(P), atol=1e-15)
    for m in range(P):
        x = np.exp(2j * np.pi * m * np.arange(P) / P)
        want = np.zeros(P, complex)
        want[m] = P
        assert np.allclose(O.dftn(x, -1), want, atol=1e-12)
    rng = np.random.default_rng(P)
    a = rng.normal(size=(P, 3)) + 1j * rng.normal(size=(P, 3))
    back = O.dftn(O.dftn(a, -1), +1) / (P * 3)
    assert np.allclose(back, a, atol=1e-13)
    A = O.dftn(a, -1)
    assert abs(np.sum(abs(A) ** 2) - P * 3 * np.sum(abs(a) ** 2)) < 1e-9 * np.sum(abs(A) ** 2)


# --------------------------------------------------------------------------
# The estimator: Eq. 7 by direct sum (O2) versus Eq. 10-14 (O3)
# --------------------------------------------------------------------------
def _problem(rng, d, M, n=60, scale=0.05, full=True):
    X = rng.uniform(0.1, 0.9, size=(n, d))
    H = random_spd(rng, d, scale) if full else np.diag(rng.uniform(0.3, 1.0, d) * scale)
    lo, hi = np.zeros(d), np.ones(d)
    counts, n_out = O.bin_linear(X, lo, hi, M)
    assert n_out == 0
    return X, H, lo, hi, counts


@pytest.mark.parametrize("d,M", [(1, (9,)), (1, (2,)), (2, (5, 7)), (2, (3, 2)),
                                 (2, (8, 8)), (3, (4, 3, 5)), (3, (2, 2, 2))])
@pytest.mark.parametrize("Lmode", ["eq15", "full"])
def test_direct_sum_equals_corrected_fft(d, M, Lmode):
    """P2: Eq. 7 by direct summation equals the corrected FFT algorithm
    (Eq. 12-14) for full H, including L = M - 1 (Sec. 4.2 'identical')."""
    rng = np.random.default_rng(hash((d, M, Lmode)) % 2**32)
    X, H, lo, hi, counts = _problem(rng, d, M)
    L = O.support_L(H, lo, hi, M) if Lmode == "eq15" else tuple(m - 1 for m in M)
    k = O.kernel_weights(H, lo, hi, M, L, len(X))
    c = O.counts_to_c(counts)
    f2 = O.binned_direct(c, k, L)
    f3, f3_imag = O.fft_corrected(c, k, L)
    assert rel_max(f3, f2) < 1e-13
    assert np.max(np.abs(f3_imag)) < 1e-13 * np.max(np.abs(f2))


def test_literal_crop_is_eq14_when_L_is_M_minus_1():
    """With L = M-1 and c_{1,1} at row M (Eq. 13), the crop of Eq. 14 is rows
    (2M-1):(3M-2), 1-based: a single count at c_{j} comes out at f_j."""
    M, L = (4, 6), (3, 5)
    P = (16, 32)
    for j in [(0, 0), (3, 5), (1, 4)]:
        c = np.zeros(M)
        c[j] = 1.0
        k = np.zeros([2 * x + 1 for x in L])
        k[L] = 1.0                                  # only k_0
        f, _ = O.fft_corrected(c, k, L, P)
        assert np.allclose(f * np.prod(P) / np.prod(P), c, atol=1e-14)
        # 0-based crop start L + M - 1 = 2M - 2, i.e. 1-based 2M - 1 (Eq. 14)
        assert all(L[i] + M[i] - 1 == 2 * M[i] - 2 for i in range(2))


def test_corrected_fft_independent_of_P():
    rng = np.random.default_rng(7)
    M = (6, 5)
    X, H, lo, hi, counts = _problem(rng, 2, M)
    L = (5, 4)
    k = O.kernel_weights(H, lo, hi, M, L, len(X))
    c = O.counts_to_c(counts)
    a, _ = O.fft_corrected(c, k, L, P=(16, 14))
    b, _ = O.fft_corrected(c, k, L, P=(21, 30))
    assert rel_max(a, b) < 1e-13


def test_single_sample_reproduces_kernel_closed_form():
    """P3: one sample exactly at node j0 (n=1): f_j = K_H(delta (j - j0)) for
    |j - j0| <= L in every quadrant, 0 beyond, with an independent formula."""
    s1, s2, rho = 0.11, 0.07, 0.85
    H = np.array([[s1 * s1, rho * s1 * s2], [rho * s1 * s2, s2 * s2]])
    M = (41, 37)
    lo, hi = np.array([0.0, 0.0]), np.array([2.0, 1.8])      # delta = 0.05
    delta = (hi - lo) / (np.array(M) - 1)
    j0 = (20, 17)
    X = (lo + delta * np.array(j0))[None, :]
    counts, _ = O.bin_linear(X, lo, hi, M)
    assert counts[j0] == 1 << 32
    L = O.support_L(H, lo, hi, M)
    k = O.kernel_weights(H, lo, hi, M, L, 1)
    f = O.binned_direct(O.counts_to_c(counts), k, L)
    J = np.indices(M).reshape(2, -1).T
    off = J - np.array(j0)
    u = off * delta
    z1, z2 = u[:, 0] / s1, u[:, 1] / s2
    want = np.exp(-(z1 * z1 - 2 * rho * z1 * z2 + z2 * z2) / (2 * (1 - rho * rho)))
    want /= 2 * np.pi * s1 * s2 * math.sqrt(1 - rho * rho)
    inside = np.all(np.abs(off) <= np.array(L), axis=1)
    want[~inside] = 0.0
    assert rel_max(f.ravel(), want) < 1e-13
    f3, _ = O.fft_corrected(O.counts_to_c(counts), k, L)
    assert rel_max(f3.ravel(), want) < 1e-12


def test_density_mass_is_one():
    """P4: sum_j f_j prod(delta) = 1 for a sample at the grid centre when the
    lattice is fine (Poisson summation) and nothing is truncated (L = M-1)."""
    H = np.array([[0.04, 0.03], [0.03, 0.05]])
    M = (81, 81)
    lo, hi = np.array([-2.0, -2.0]), np.array([2.0, 2.0])     # delta = 0.05
    X = np.array([[0.0, 0.0]])
    counts, _ = O.bin_linear(X, lo, hi, M)
    L = (80, 80)
    k = O.kernel_weights(H, lo, hi, M, L, 1)
    f = O.binned_direct(O.counts_to_c(counts), k, L)
    delta = (hi - lo) / (np.array(M) - 1)
    assert abs(f.sum() * np.prod(delta) - 1.0) < 1e-10


def test_wand_layout_exact_for_diagonal_H():
    """P5: with diagonal H, Wand's layout (Eq. 8, 9, 11) gives the same
    estimate as the corrected one (Sec. 3, Figure 1(c))."""
    rng = np.random.default_rng(8)
    for d, M in [(2, (9, 7)), (3, (5, 4, 6))]:
        X, H, lo, hi, counts = _problem(rng, d, M, full=False)
        L = O.support_L(H, lo, hi, M)
        k = O.kernel_weights(H, lo, hi, M, L, len(X))
        k_abs = k[tuple(slice(Lk, None) for Lk in L)]
        c = O.counts_to_c(counts)
        fw, _ = O.fft_wand(c, k_abs, L)
        fc, _ = O.fft_corrected(c, k, L)
        assert rel_max(fw, fc) < 1e-13


def test_wand_layout_wrong_for_full_H_closed_form():
    """P6: for full H, Wand's layout convolves with k_{|l|}: a single sample
    at j0 gives K_H(a d1, b d2) at offset (-a, b) where the true value is
    K_H(-a d1, b d2).  For correlation .95 the error is O(1) of the peak."""
    H = np.array([[0.1025, 0.0975], [0.0975, 0.1025]])      # eig .2, .005
    M = (61, 61)
    lo, hi = np.array([-3.0, -3.0]), np.array([3.0, 3.0])   # delta = 0.1
    delta = 0.1
    j0 = (30, 30)
    X = np.array([[0.0, 0.0]])
    counts, _ = O.bin_linear(X, lo, hi, M)
    assert counts[j0] == 1 << 32
    L = O.support_L(H, lo, hi, M)
    k = O.kernel_weights(H, lo, hi, M, L, 1)
    k_abs = k[L[0]:, L[1]:]
    c = O.counts_to_c(counts)
    fw, _ = O.fft_wand(c, k_abs, L)
    fc, _ = O.fft_corrected(c, k, L)
    for a, b in [(3, 3), (1, 4), (5, 2)]:
        node = (j0[0] - a, j0[1] + b)
        want_w = O.scaled_gaussian([[a * delta, b * delta]], H)[0]
        want_c = O.scaled_gaussian([[-a * delta, b * delta]], H)[0]
        assert abs(fw[node] - want_w) < 1e-12 * want_w + 1e-300
        assert abs(fc[node] - want_c) < 1e-12 * max(want_c, 1e-300) + 1e-15
    assert np.max(np.abs(fw - fc)) / fc.max() > 0.5
    # Wand's result is symmetric under a reflection of one axis (Figure 1(b)
    # looks like the diagonal-H estimate): it lost the sign of the correlation.
    assert np.allclose(fw, fw[::-1, :], atol=1e-12 * fw.max())


def test_wand_layout_exact_in_one_dimension():
    """P7: the 1-D algorithm is correct (Sec. 4.1)."""
    rng = np.random.default_rng(9)
    X, H, lo, hi, counts = _problem(rng, 1, (33,), scale=0.01)
    L = O.support_L(H, lo, hi, (33,))
    k = O.kernel_weights(H, lo, hi, (33,), L, len(X))
    c = O.counts_to_c(counts)
    fw, _ = O.fft_wand(c, k[L[0]:], L)
    fc, _ = O.fft_corrected(c, k, L)
    assert rel_max(fw, fc) < 1e-13


def test_truncation_bound_and_corrected_range_wider():
    """P8: the largest kernel value left outside the box |l_k| <= L_k, relative
    to the peak, is at most max_k exp(-((L_k+1) delta_k)^2 / (2 H_kk)) (the
    minimum of u^T H^-1 u on the plane u_k = a is a^2 / H_kk); brute force on
    the lattice.  The per-axis range drops far more for correlated H."""
    H = np.array([[0.1025, 0.0975], [0.0975, 0.1025]])
    lo, hi, M = np.array([0.0, 0.0]), np.array([10.23, 10.23]), (1024, 1024)
    delta = O.binwidths(lo, hi, M)
    Hinv = np.linalg.inv(H)
    out = {}
    for mode in ["corrected", "per_axis"]:
        L = O.support_L(H, lo, hi, M, range_mode=mode)
        bound = max(math.exp(-((L[k] + 1) * delta[k]) ** 2 / (2 * H[k, k])) for k in range(2))
        R = 3 * max(L)
        g = np.arange(-R, R + 1)
        l1, l2 = np.meshgrid(g, g, indexing="ij")
        u1, u2 = l1 * delta[0], l2 * delta[1]
        q = Hinv[0, 0] * u1 * u1 + 2 * Hinv[0, 1] * u1 * u2 + Hinv[1, 1] * u2 * u2
        outside = (np.abs(l1) > L[0]) | (np.abs(l2) > L[1])
        worst = float(np.exp(-0.5 * q[outside]).max())
        assert worst <= bound * (1 + 1e-9)
        assert worst >= 0.5 * bound                 # the lattice nearly attains it
        out[mode] = worst
    assert out["corrected"] < 2e-6
    assert out["per_axis"] > 1e-4
    assert out["per_axis"] > 100 * out["corrected"]


def test_diagonal_H_ranges_agree_within_per_axis_bound():
    """P9: for diagonal H, L >= L^W elementwise and the two estimates differ by
    no more than the per-axis truncation allows."""
    rng = np.random.default_rng(11)
    M = (40, 50)
    X, _, lo, hi, counts = _problem(rng, 2, M, n=200)
    H = np.diag([0.002, 0.0005])
    La = O.support_L(H, lo, hi, M)
    Lw = O.support_L(H, lo, hi, M, range_mode="per_axis")
    assert all(a >= b for a, b in zip(La, Lw))
    c = O.counts_to_c(counts)
    fa = O.binned_direct(c, O.kernel_weights(H, lo, hi, M, La, 200), La)
    fw = O.binned_direct(c, O.kernel_weights(H, lo, hi, M, Lw, 200), Lw)
    assert rel_max(fw, fa) < 5e-3


def test_linearity_and_shift():
    """P11: Eq. 7 is linear in c and shift-equivariant away from the edges."""
    rng = np.random.default_rng(12)
    M = (30, 30)
    H = random_spd(rng, 2, 0.002)
    lo, hi = np.zeros(2), np.ones(2)
    L = O.support_L(H, lo, hi, M)
    k = O.kernel_weights(H, lo, hi, M, L, 10)
    c1 = np.zeros(M)
    c1[12:16, 10:14] = rng.uniform(size=(4, 4))
    c2 = rng.uniform(size=M)
    f1 = O.binned_direct(c1, k, L)
    f2 = O.binned_direct(c2, k, L)
    f12 = O.binned_direct(2 * c1 - 3 * c2, k, L)
    assert rel_max(f12, 2 * f1 - 3 * f2) < 1e-13
    cs = np.roll(c1, (3, -2), axis=(0, 1))
    fs = O.binned_direct(cs, k, L)
    assert rel_max(fs, np.roll(f1, (3, -2), axis=(0, 1))) < 1e-13


def test_binned_direct_at_matches_full_grid():
    rng = np.random.default_rng(13)
    for d, M in [(1, (50,)), (2, (20, 17)), (3, (9, 8, 7))]:
        X, H, lo, hi, counts = _problem(rng, d, M, n=300)
        L = O.support_L(H, lo, hi, M)
        k = O.kernel_weights(H, lo, hi, M, L, 300)
        c = O.counts_to_c(counts)
        full = O.binned_direct(c, k, L)
        nodes = np.stack([rng.integers(0, m, 100) for m in M], axis=1)
        at = O.binned_direct_at(c, k, L, nodes)
        assert np.allclose(at, full[tuple(nodes.T)], rtol=1e-13, atol=1e-13 * full.max())


# --------------------------------------------------------------------------
# O1: Eq. 1 directly; binning as an approximation of it
# --------------------------------------------------------------------------
def test_direct_kde_matches_scipy_mixture_mean():
    rng = np.random.default_rng(14)
    H = random_spd(rng, 2, 0.05)
    X = rng.normal(size=(200, 2))
    pts = rng.normal(size=(30, 2))
    want = np.mean([multivariate_normal(mean=x, cov=H).pdf(pts) for x in X], axis=0)
    assert rel_max(O.direct_kde(X, H, pts), want) < 1e-12


def test_binning_error_second_order():
    """P12: max |binned - direct| shrinks about 4x when the grid is refined 2x."""
    rng = np.random.default_rng(15)
    X = rng.normal(size=(400, 2)) * 0.4
    H = np.array([[0.04, 0.02], [0.02, 0.03]])
    lo, hi = np.array([-3.0, -3.0]), np.array([3.0, 3.0])
    errs = []
    for M in [(41, 41), (81, 81), (161, 161)]:
        f, counts, L, n_out = O.binned_estimate(X, H, lo, hi, M, tau=8.0)
        assert n_out == 0
        g = O.grid_axes(lo, hi, M)
        G = np.stack(np.meshgrid(*g, indexing="ij"), -1).reshape(-1, 2)
        idx = np.arange(0, len(G), 7)
        direct = O.direct_kde(X, H, G[idx])
        errs.append(np.max(np.abs(f.ravel()[idx] - direct)) / direct.max())
    assert errs[0] / errs[1] > 2.5 and errs[1] / errs[2] > 2.5


def test_wand_kernel_weights_direct_sum_equals_wand_layout():
    """The direct sum with Wand's weights k_{|l|} is what Eq. 8's wrap-around
    layout computes (the literal layout pins the 'wand' weights)."""
    rng = np.random.default_rng(16)
    for d, M in [(2, (9, 11)), (3, (5, 6, 4))]:
        X, H, lo, hi, counts = _problem(rng, d, M)
        L = O.support_L(H, lo, hi, M)
        kc = O.kernel_weights(H, lo, hi, M, L, len(X))
        kw = O.kernel_weights(H, lo, hi, M, L, len(X), layout="wand")
        c = O.counts_to_c(counts)
        fw, _ = O.fft_wand(c, kc[tuple(slice(Lk, None) for Lk in L)], L)
        assert rel_max(O.binned_direct(c, kw, L), fw) < 1e-13
        assert rel_max(O.binned_direct(c, kc, L), fw) > 1e-3


# --------------------------------------------------------------------------
# LSCV on binned data (the bandwidth-selection functional the paper points to)
# --------------------------------------------------------------------------
def test_lscv_binned_equals_exact_for_samples_on_nodes():
    """Samples exactly on grid nodes are binned without error; with the full
    support (L = M-1, via a large tau) the binned pair sums equal the sums
    over sample pairs, so binned LSCV = exact LSCV (brute-force double loop)."""
    rng = np.random.default_rng(50)
    M = (21, 17)
    lo, hi = np.array([0.0, 0.0]), np.array([2.0, 1.6])      # delta = 0.1
    nodes = np.stack([rng.integers(2, 19, 40), rng.integers(2, 15, 40)], axis=1)
    X = lo + 0.1 * nodes
    H = np.array([[0.02, 0.012], [0.012, 0.015]])
    counts, n_out = O.bin_linear(X, lo, hi, M)
    assert n_out == 0
    got = O.lscv_binned(counts, len(X), H, lo, hi, M, tau=100.0)
    want = O.lscv_exact(X, H)
    assert abs(got - want) < 1e-12 * abs(want)


def test_lscv_first_term_is_integral_of_square():
    """(1/n^2) sum_{i,j} K_{2H}(X_i - X_j) = integral of f^2 (Gaussian
    convolution), checked by quadrature of the estimate on a fine grid."""
    rng = np.random.default_rng(51)
    X = rng.normal(size=(7, 2)) * 0.3
    H = np.array([[0.05, 0.02], [0.02, 0.04]])
    g = np.linspace(-3, 3, 301)
    G = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
    f = O.direct_kde(X, H, G)
    integral = float(np.sum(f * f)) * (g[1] - g[0]) ** 2
    D = (X[:, None, :] - X[None, :, :]).reshape(-1, 2)
    closed = float(np.sum(O.scaled_gaussian(D, 2 * H))) / len(X) ** 2
    assert abs(integral - closed) < 1e-8 * closed


def test_lscv_leave_one_out_term():
    """The second term is (2/n) sum_i f_{-i}(X_i) with the leave-one-out
    estimate written out sample by sample."""
    rng = np.random.default_rng(52)
    X = rng.normal(size=(9, 2)) * 0.5
    H = np.array([[0.08, -0.03], [-0.03, 0.06]])
    n = len(X)
    loo = 0.0
    for i in range(n):
        others = np.delete(X, i, axis=0)
        loo += float(np.sum(O.scaled_gaussian(X[i] - others, H))) / (n - 1)
    D = (X[:, None, :] - X[None, :, :]).reshape(-1, 2)
    first = float(np.sum(O.scaled_gaussian(D, 2 * H))) / n**2
    assert abs(O.lscv_exact(X, H) - (first - 2.0 * loo / n)) < 1e-13


def test_lscv_binned_spectral_form():
    """S(A) = (1/prod P) sum_w |C(w)|^2 K_A(w) (Parseval on the zero-padded,
    wrapped arrays) -- the identity the batched GPU evaluation relies on --
    against the direct binned pair sum."""
    rng = np.random.default_rng(53)
    M = (24, 19)
    X = rng.uniform(0.2, 0.8, size=(300, 2))
    lo, hi = np.zeros(2), np.ones(2)
    counts, _ = O.bin_linear(X, lo, hi, M)
    c = O.counts_to_c(counts)
    A = np.array([[0.004, 0.002], [0.002, 0.003]])
    L = O.support_L(A, lo, hi, M)
    P = (M[0] + L[0] + 3, M[1] + L[1] + 5)
    k = O.kernel_weights(A, lo, hi, M, L, n=1)
    kw = np.zeros(P)
    for a in range(-L[0], L[0] + 1):
        for b in range(-L[1], L[1] + 1):
            kw[a % P[0], b % P[1]] = k[a + L[0], b + L[1]]
    cp = np.zeros(P)
    cp[: M[0], : M[1]] = c
    C = O.dftn(cp, -1)
    K = O.dftn(kw, -1)
    spectral = float(np.sum(np.abs(C) ** 2 * K.real)) / np.prod(P)
    direct = O.binned_pair_sum(c, A, lo, hi, M, L)
    assert abs(spectral - direct) < 1e-12 * abs(direct)
    assert np.max(np.abs(K.imag)) < 1e-12 * np.max(np.abs(K.real))


def test_lscv_supports_follow_eq15_per_matrix():
    """Each pair sum uses the support of its own matrix (Eq. 15 on H and on
    2H): with tau = 3.7 the criterion matches the untruncated one to within
    the tail of the Gaussian, far closer than if 2H were cut at H's support."""
    rng = np.random.default_rng(54)
    X = rng.normal(size=(400, 2)) * 0.4
    H = np.array([[0.03, 0.015], [0.015, 0.02]])
    lo, hi, M = np.array([-3.0, -3.0]), np.array([3.0, 3.0]), (61, 61)
    counts, _ = O.bin_linear(X, lo, hi, M)
    full = O.lscv_binned(counts, len(X), H, lo, hi, M, tau=100.0)
    eq15 = O.lscv_binned(counts, len(X), H, lo, hi, M, tau=3.7)
    c = O.counts_to_c(counts)
    L1 = O.support_L(H, lo, hi, M)
    S2_short = O.binned_pair_sum(c, 2 * H, lo, hi, M, L1)
    S2_full = O.binned_pair_sum(c, 2 * H, lo, hi, M, (60, 60))
    scale = S2_full / len(X) ** 2
    assert abs(eq15 - full) < 3e-6 * scale
    assert abs(S2_short - S2_full) / len(X) ** 2 > 3e-5 * scale


def test_pair_sum_dft_equals_direct():
    """The spectral pair sum (zero-padded, wrapped, Parseval) equals the direct
    binned pair sum for any padding P >= M + L, in 1-D and 2-D."""
    rng = np.random.default_rng(55)
    for d, M in [(1, (40,)), (2, (18, 23))]:
        X = rng.uniform(0.1, 0.9, size=(200, d))
        lo, hi = np.zeros(d), np.ones(d)
        counts, _ = O.bin_linear(X, lo, hi, M)
        c = O.counts_to_c(counts)
        A = random_spd(rng, d, 0.003)
        L = O.support_L(A, lo, hi, M)
        direct = O.binned_pair_sum(c, A, lo, hi, M, L)
        for extra in (0, 7):
            P = tuple(m + l + extra for m, l in zip(M, L))
            assert abs(O.binned_pair_sum_dft(c, A, lo, hi, M, L, P) - direct) < 1e-12 * abs(direct)
