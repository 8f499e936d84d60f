"""Seeded synthetic inputs for binned FFT KDE with an unconstrained bandwidth.

The paper demonstrates its method on a 2-D dataset that is not distributed
with it (Sec. 3, Figure 1).  These generators stand in for it: Gaussian
mixtures with correlated components, a full (non-diagonal) bandwidth matrix H
and a grid whose range covers the data plus a margin of 4 sqrt(lambda_max(H)).

This module only draws inputs.  It holds none of the estimator's arithmetic
(no binning, no kernel weights, no transforms); both the CUDA path and the CPU
oracle receive what it returns.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    """One problem instance: samples X (n x d), bandwidth H (d x d), grid lo/hi/M."""

    name: str
    X: np.ndarray
    H: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    M: tuple
    precision: str          # "f32" or "f64": arithmetic type of the evaluation
    tau: float = 3.7        # effective-support constant of Eq. 15
    notes: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return self.X.shape[1]

    @property
    def n(self) -> int:
        return self.X.shape[0]


def mixture_samples(rng, n, means, covs, weights=None):
    """Draw n samples (float64) from a Gaussian mixture."""
    means = np.asarray(means, dtype=np.float64)
    k, d = means.shape
    if weights is None:
        weights = np.full(k, 1.0 / k)
    comp = rng.choice(k, size=n, p=weights)
    z = rng.standard_normal((n, d))
    X = np.empty((n, d))
    for c in range(k):
        idx = np.nonzero(comp == c)[0]
        R = np.linalg.cholesky(np.asarray(covs[c], dtype=np.float64))
        X[idx] = means[c] + z[idx] @ R.T
    return X


def grid_range(X, H, margin=4.0):
    """Grid ends: data min/max widened by margin * sqrt(largest eigenvalue of H)."""
    lam = float(np.linalg.eigvalsh(np.asarray(H, dtype=np.float64)).max())
    pad = margin * np.sqrt(lam)
    Xd = X.astype(np.float64)
    return Xd.min(axis=0) - pad, Xd.max(axis=0) + pad


def _corr_cov(rho):
    return np.array([[1.0, rho], [rho, 1.0]])


MIX2_MEANS = [(0.0, 0.0), (2.0, 1.0), (-1.0, 2.0)]
MIX2_COVS = [_corr_cov(0.8), _corr_cov(-0.5), _corr_cov(0.0)]


def haar_orthogonal(rng, d):
    """Haar-distributed orthogonal matrix (QR of a Gaussian matrix, sign-fixed)."""
    A = rng.standard_normal((d, d))
    Q, R = np.linalg.qr(A)
    return Q * np.sign(np.diag(R))


def random_spd(rng, d, cond_lo=1.0, cond_hi=50.0, scale=1.0):
    """SPD matrix Q diag(1, kappa^-1/2, kappa^-1) Q^T (d=3) with kappa ~ U[lo, hi]."""
    kappa = rng.uniform(cond_lo, cond_hi)
    ev = kappa ** (-np.linspace(0.0, 1.0, d))
    Q = haar_orthogonal(rng, d)
    return scale * (Q * ev) @ Q.T


def rotated_bandwidth(eig_major, eig_minor, angle_rad=np.pi / 4):
    """2x2 H with the given eigenvalues, major axis at angle_rad."""
    c, s = np.cos(angle_rad), np.sin(angle_rad)
    R = np.array([[c, -s], [s, c]])
    return R @ np.diag([eig_major, eig_minor]) @ R.T


def normal_reference_bandwidth(X):
    """Textbook normal-reference H = (4/(d+2))^(2/(d+4)) n^(-2/(d+4)) S."""
    n, d = X.shape
    S = np.cov(X.astype(np.float64), rowvar=False)
    return (4.0 / (d + 2)) ** (2.0 / (d + 4)) * n ** (-2.0 / (d + 4)) * S


def kde2d_128_f64(seed=1, n=10_000):
    """d=2, n=1e4, 3-component mixture, H=[[.09,.07],[.07,.09]], 128x128, FP64."""
    rng = np.random.default_rng(seed)
    X = mixture_samples(rng, n, MIX2_MEANS, MIX2_COVS)
    H = np.array([[0.09, 0.07], [0.07, 0.09]])
    lo, hi = grid_range(X, H)
    return Workload("kde2d_128_f64", X, H, lo, hi, (128, 128), "f64")


def kde2d_1024_f32(seed=2, n=1_000_000):
    """d=2, n=1e6, the same mixture scaled x3, H correlation 0.95 (eig .2/.005), 1024^2, FP32."""
    rng = np.random.default_rng(seed)
    X = 3.0 * mixture_samples(rng, n, MIX2_MEANS, MIX2_COVS)
    H = rotated_bandwidth(0.2, 0.005)
    lo, hi = grid_range(X, H)
    return Workload("kde2d_1024_f32", X.astype(np.float32), H, lo, hi, (1024, 1024), "f32")


def kde3d_256_f32(seed=3, n=10_000_000):
    """d=3, n=1e7, 4-component mixture with random SPD covariances (cond 1-50), 256^3, FP32."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-3.0, 3.0, size=(4, 3))
    covs = [random_spd(rng, 3) for _ in range(4)]
    X = mixture_samples(rng, n, means, covs)
    H = normal_reference_bandwidth(X)
    lo, hi = grid_range(X, H)
    return Workload("kde3d_256_f32", X.astype(np.float32), H, lo, hi, (256, 256, 256), "f32")


WORKLOADS = {
    "kde2d_128_f64": kde2d_128_f64,
    "kde2d_1024_f32": kde2d_1024_f32,
    "kde3d_256_f32": kde3d_256_f32,
}


def small_case(seed, d, M, n, precision="f64", H=None, corr=0.7, scale=0.05):
    """A small random problem for parity tests: any d in 1..3, ragged M."""
    rng = np.random.default_rng(seed)
    if H is None:
        if d == 1:
            H = np.array([[scale]])
        else:
            A = np.full((d, d), corr) + (1.0 - corr) * np.eye(d)
            D = np.diag(rng.uniform(0.6, 1.4, size=d))
            H = scale * (D @ A @ D)
    means = rng.uniform(-1.0, 1.0, size=(2, d))
    covs = [np.eye(d) * 0.3, np.eye(d) * 0.1 + 0.05]
    X = mixture_samples(rng, n, means, covs)
    lo, hi = grid_range(X, H)
    dt = np.float64 if precision == "f64" else np.float32
    return Workload(f"small_d{d}", X.astype(dt), np.asarray(H, dtype=np.float64),
                    lo, hi, tuple(int(m) for m in M), precision)


def log_cholesky_candidates(rng, count, d=2, diag_lo=-4.0, diag_hi=0.0, off=1.0):
    """Candidate bandwidths H = R R^T, R lower triangular with diagonal
    exp(U[diag_lo, diag_hi]) and off-diagonal U[-off, off]."""
    out = np.empty((count, d, d))
    for i in range(count):
        R = np.zeros((d, d))
        R[np.diag_indices(d)] = np.exp(rng.uniform(diag_lo, diag_hi, size=d))
        for a in range(d):
            for b in range(a):
                R[a, b] = rng.uniform(-off, off)
        out[i] = R @ R.T
    return out


@dataclass
class LscvWorkload:
    """Bandwidth selection: one binned grid, many candidate bandwidths."""

    name: str
    X: np.ndarray
    H: np.ndarray          # (count, d, d)
    lo: np.ndarray
    hi: np.ndarray
    M: tuple
    precision: str
    tau: float = 3.7

    @property
    def d(self):
        return self.X.shape[1]

    @property
    def n(self):
        return self.X.shape[0]


def lscv2d_512_f32(seed=4, n=2_000_000, count=1024):
    """d=2, n=2e6 from the 3-component mixture, 512^2 grid, 1024 candidate H
    sampled in log-Cholesky space; the grid covers the data plus
    4 sqrt(largest eigenvalue over the candidates)."""
    rng = np.random.default_rng(seed)
    X = mixture_samples(rng, n, MIX2_MEANS, MIX2_COVS)
    H = log_cholesky_candidates(rng, count)
    lam = max(float(np.linalg.eigvalsh(h).max()) for h in H)
    pad = 4.0 * np.sqrt(lam)
    lo = X.min(axis=0) - pad
    hi = X.max(axis=0) + pad
    return LscvWorkload("lscv2d_512_f32", X.astype(np.float32), H, lo, hi, (512, 512), "f32")


def lscv_small(seed, d, M, n, count, precision="f64", diag_lo=-4.0, diag_hi=-1.5):
    """A small bandwidth-selection problem for parity tests."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(2, d))
    covs = [np.eye(d) * 0.2, np.eye(d) * 0.05]
    X = mixture_samples(rng, n, means, covs)
    H = log_cholesky_candidates(rng, count, d, diag_lo, diag_hi, off=0.1)
    lam = max(float(np.linalg.eigvalsh(h).max()) for h in H)
    pad = 4.0 * np.sqrt(lam)
    dt = np.float64 if precision == "f64" else np.float32
    return LscvWorkload(f"lscv_small_d{d}", X.astype(dt), H, X.min(axis=0) - pad,
                        X.max(axis=0) + pad, tuple(int(m) for m in M), precision)


def ragged64_f32(seed=5, count=64):
    """A ragged batch: 64 independent 2-D datasets, n log-uniform in
    [1e3, 1e6], grids drawn from {64, 128, 256, 512, 1024}^2, each with its
    own correlated bandwidth (normal-reference scale, random orientation)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(10 ** rng.uniform(3.0, 6.0)))
        m = int(rng.choice([64, 128, 256, 512, 1024]))
        X = mixture_samples(rng, n, MIX2_MEANS, MIX2_COVS)
        scale = n ** (-1.0 / 3.0)
        H = rotated_bandwidth(scale * rng.uniform(0.5, 2.0), scale * rng.uniform(0.02, 0.3),
                              rng.uniform(0, np.pi))
        lo, hi = grid_range(X, H)
        out.append(Workload("ragged", X.astype(np.float32), H, lo, hi, (m, m), "f32"))
    return out


def mixture_dataset_chunk(seed, chunk, count, n=10_000):
    """Chunk `chunk` of a stream of learned-proposal datasets, as one
    count x n x 2 float32 array: the recipe of mixture_datasets (2-5
    components, weights Dirichlet(2), means U[-3, 3]^2, covariances
    Q diag(s1, s2) Q^T with s ~ exp(U[log 0.05, log 1.5]) and Q a random
    rotation), with the component sizes drawn multinomially and each
    component's samples stored together.  Chunks are seeded by (seed,
    chunk), so any subset can be drawn in any order or process."""
    rng = np.random.default_rng([seed, chunk])
    out = np.empty((count, n, 2), dtype=np.float32)
    z = rng.standard_normal((count, n, 2), dtype=np.float32)
    for b in range(count):
        k = int(rng.integers(2, 6))
        w = rng.dirichlet(np.full(k, 2.0))
        means = rng.uniform(-3.0, 3.0, size=(k, 2)).astype(np.float32)
        ang = rng.uniform(0.0, np.pi, size=k)
        sd = np.sqrt(np.exp(rng.uniform(np.log(0.05), np.log(1.5), size=(k, 2))))
        sizes = rng.multinomial(n, w)
        a = 0
        for j in range(k):
            c, s = np.cos(ang[j]), np.sin(ang[j])
            # Q diag(sd): its product with its transpose is the covariance
            A = np.array([[c * sd[j, 0], -s * sd[j, 1]], [s * sd[j, 0], c * sd[j, 1]]],
                         dtype=np.float32)
            e = a + int(sizes[j])
            np.matmul(z[b, a:e], A.T, out=out[b, a:e])
            out[b, a:e] += means[j]
            a = e
    return out


def mixture_datasets(seed, count, n=10_000):
    """Datasets for the learned bandwidth proposal: 2-D Gaussian mixtures with
    2-5 components, weights Dirichlet(2), means U[-3, 3]^2 and covariances
    Q diag(s1, s2) Q^T with s ~ exp(U[log 0.05, log 1.5]) and Q a random
    rotation; n samples each (float32)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        k = int(rng.integers(2, 6))
        w = rng.dirichlet(np.full(k, 2.0))
        means = rng.uniform(-3.0, 3.0, size=(k, 2))
        covs = []
        for _ in range(k):
            ang = rng.uniform(0, np.pi)
            c, s = np.cos(ang), np.sin(ang)
            Q = np.array([[c, -s], [s, c]])
            ev = np.exp(rng.uniform(np.log(0.05), np.log(1.5), size=2))
            covs.append((Q * ev) @ Q.T)
        out.append(mixture_samples(rng, n, means, covs, w).astype(np.float32))
    return out
