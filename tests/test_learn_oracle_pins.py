"""Pins of the learned-proposal oracle (oracle/learn_oracle.py) against
things other than itself: finite differences, hand-worked values and scipy."""
import numpy as np
import pytest

from oracle import learn_oracle as LO


def _params(rng, in_dim, hidden, out_dim, scale=0.7):
    n = hidden * in_dim + hidden + hidden * hidden + hidden + out_dim * hidden + out_dim
    return rng.normal(0.0, scale, n)


def test_forward_hand_worked():
    # x = (1, -2); W1 = I, b1 = 0 -> z1 = (1, -2), a1 = (1, 0)
    # W2 = [[2, 1], [-1, 3]], b2 = (.5, .5) -> z2 = (2.5, -.5), a2 = (2.5, 0)
    # W3 = [[1, 1]], b3 = -1 -> y = 1.5
    p = np.array([1, 0, 0, 1, 0, 0, 2, 1, -1, 3, .5, .5, 1, 1, -1], dtype=np.float64)
    y, _ = LO.mlp_forward(p, np.array([[1.0, -2.0]]), 2, 2, 1)
    assert y.shape == (1, 1) and y[0, 0] == 1.5
    loss, g = LO.mlp_loss_grad(p, np.array([[1.0, -2.0]]), np.array([[0.5]]), 2, 2, 1)
    assert loss == 1.0
    # dy = 2; dW3 = dy a2 = (5, 0); db3 = 2; da2 = dy W3 = (2, 2); dz2 = (2, 0)
    # dW2 = dz2^T a1 = [[2, 0], [0, 0]]; db2 = (2, 0); da1 = dz2 W2 = (4, 2);
    # dz1 = (4, 0); dW1 = [[4, -8], [0, 0]]; db1 = (4, 0)
    assert np.array_equal(g, [4, -8, 0, 0, 4, 0, 2, 0, 0, 0, 2, 0, 5, 0, 2])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    in_dim, hidden, out_dim, B = 7, 6, 3, 5
    X = rng.normal(size=(B, in_dim))
    T = rng.normal(size=(B, out_dim))
    for _ in range(50):  # draw parameters with every unit away from the ReLU kink
        p = _params(rng, in_dim, hidden, out_dim)
        _, (X_, z1, a1, z2, a2) = LO.mlp_forward(p, X, in_dim, hidden, out_dim)
        if np.abs(z1).min() > 1e-3 and np.abs(z2).min() > 1e-3:
            break
    loss, g = LO.mlp_loss_grad(p, X, T, in_dim, hidden, out_dim)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = LO.mlp_loss_grad(p + e, X, T, in_dim, hidden, out_dim)
        lm, _ = LO.mlp_loss_grad(p - e, X, T, in_dim, hidden, out_dim)
        fd[i] = (lp - lm) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-6 * max(1.0, np.max(np.abs(g)))


def test_standardize_against_scipy():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(3)
    X = rng.gamma(2.0, size=(5000, 2)) @ np.array([[1.0, 0.3], [0.0, 2.0]])
    Z, mom = LO.standardize(X)
    assert np.allclose(mom[:2], X.mean(axis=0), rtol=1e-12)
    assert np.allclose(mom[2:4], X.std(axis=0), rtol=1e-12)
    assert abs(mom[4] - np.corrcoef(X.T)[0, 1]) < 1e-12
    assert np.allclose(mom[5:7], stats.skew(X, axis=0, bias=True), rtol=1e-10)
    assert abs(mom[7] - stats.kurtosis(X, axis=0, fisher=True, bias=True).mean()) < 1e-10
    assert np.allclose(Z.mean(axis=0), 0, atol=1e-12) and np.allclose(Z.std(axis=0), 1, atol=1e-12)


def test_features_single_cell_and_moment_slots():
    M, n = 64, 10
    counts = np.zeros((M, M), dtype=np.int64)
    counts[9, 50] = n << 32              # all mass in one cell: block (9 // 2, 50 // 2)
    mom = np.arange(8, dtype=np.float64)
    f = LO.features(counts, n, mom)
    assert f.shape == (LO.FEAT_DIM,)
    blocks = f[:1024].reshape(32, 32)
    assert blocks[4, 25] == 8.0 and np.count_nonzero(blocks) == 1
    assert np.array_equal(f[1024:1030], [4, 5, 6, 7, np.log10(n) / 4, 1])
    assert not f[1030:].any()


def test_theta_to_H_closed_forms():
    H = LO.theta_to_H((np.log(0.3), 0.0, np.log(0.2)))
    assert np.allclose(H, np.diag([0.09, 0.04]), rtol=1e-14, atol=0)
    a, beta, c = -1.0, 0.75, -1.5
    H = LO.theta_to_H((a, beta, c))
    assert abs(np.linalg.det(H) - np.exp(2 * a + 2 * c)) < 1e-14
    assert abs(H[0, 1] / np.sqrt(H[0, 0] * H[1, 1]) - beta / np.sqrt(1 + beta ** 2)) < 1e-14


def test_bf16_round_values():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even significand wins (1);
    # 1 + 3 * 2^-8 ties between 1 + 2^-7 and 1 + 2^-6 (even): 1 + 2^-6;
    # values already on the BF16 grid are unchanged
    x = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -7, -3.0, 2.0 ** -130, 0.0])
    assert np.array_equal(LO.bf16_round(x), [1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -3.0, 2.0 ** -130, 0.0])


def test_bf16_gradient_is_the_fp64_one_on_bf16_grid_values():
    """With inputs and parameters already on the BF16 grid and activations
    that stay on it, the rounded network equals the plain one."""
    p = np.array([1, 0, 0, 1, 0, 0, 2, 1, -1, 3, .5, .5, 1, 1, -1], dtype=np.float64)
    X, T = np.array([[1.0, -2.0]]), np.array([[0.5]])
    a = LO.mlp_loss_grad(p, X, T, 2, 2, 1)
    b = LO.mlp_loss_grad(p, X, T, 2, 2, 1, bf16=True)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_batched_candidate_construction_matches_oracle():
    """The learned selection builds every dataset's candidates at once
    (thetas_to_H over arrays, neighbourhood of many thetas); each matrix must
    equal the oracle's R R^T for its theta, and each neighbourhood the
    single-theta one."""
    from paper_1508_02766_gb300 import learned as Lm
    rng = np.random.default_rng(12)
    T = np.stack([rng.uniform(-3, 0, 40), rng.uniform(-1.5, 1.5, 40), rng.uniform(-3, 0, 40)], 1)
    H = Lm.thetas_to_H(T)
    for t, h in zip(T, H):
        ref = LO.theta_to_H(t)
        assert np.allclose(h, ref, rtol=1e-14, atol=0.0)
        assert h[0, 1] == h[1, 0]
    N = Lm.neighbourhood(T[:5])
    assert N.shape == (5, 27, 3)
    for i in range(5):
        assert np.array_equal(N[i], Lm.neighbourhood(T[i]))
    # the centre of each neighbourhood is the theta itself
    assert np.array_equal(N[:, 13], T[:5])
    HH = Lm.thetas_to_H(N)
    assert HH.shape == (5, 27, 2, 2)
    assert np.array_equal(HH[2, 7], Lm.theta_to_H(N[2, 7]))
