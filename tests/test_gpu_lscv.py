"""Bandwidth selection by LSCV on the GPU (count spectrum once, batched
kernel spectra fused with the dot product) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import kde_oracle as O
from paper_1508_02766_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import os

    from paper_1508_02766_gb300 import build, kde
    if not os.path.exists(build.LIB):
        build.build()
    return kde


def plan_for(K, w, **opts):
    """A plan whose padding fits 2H for every candidate (largest eigenvalue)."""
    lam = [np.linalg.eigvalsh(h).max() for h in w.H]
    big = 2.0 * w.H[int(np.argmax(lam))]
    info = K.kde_plan_info_compute(w.M, w.lo, w.hi, big, precision=w.precision, tau=w.tau)
    return K.Plan(w.M, w.lo, w.hi, big, precision=w.precision, tau=w.tau, P_min=info.P, **opts)


def run_lscv(K, w, **opts):
    plan = plan_for(K, w, **opts)
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    Wsp = K.kde_power_spectrum(plan, counts)
    S = torch.empty(2 * len(w.H), dtype=torch.float64, device="cuda")
    lscv = K.kde_lscv(plan, w.n, w.H, Wsp, pair_sums=S)
    torch.cuda.synchronize()
    return lscv.cpu().numpy(), S.cpu().numpy(), counts.cpu().numpy(), plan


def oracle_lscv(w, counts, idx):
    c = O.counts_to_c(counts)
    out, S = [], []
    for i in idx:
        H = w.H[i]
        s = []
        for A in (H, 2 * H):
            L = O.support_L(A, w.lo, w.hi, w.M, w.tau)
            s.append(O.binned_pair_sum(c, A, w.lo, w.hi, w.M, L))
        K0 = float(O.scaled_gaussian(np.zeros((1, w.d)), H)[0])
        S.append(s)
        out.append(O.lscv_binned(counts, w.n, H, w.lo, w.hi, w.M, w.tau))
    return np.array(out), np.array(S)


@pytest.mark.parametrize("prec,cols", [("f64", "lines"), ("f64", "simd"), ("f32", "lines"),
                                       ("f32", "simd")])
def test_lscv_2d_every_candidate(K, prec, cols):
    """40 candidates (two batches), every pair sum and score against the oracle."""
    w = W.lscv_small(7, 2, (36, 44), n=3000, count=40, precision=prec)
    lscv, S, counts, plan = run_lscv(K, w, cols=cols)
    ref, Sref = oracle_lscv(w, counts, range(len(w.H)))
    tol = 1e-12 if prec == "f64" else 2e-5
    assert np.max(np.abs(S.reshape(-1, 2) - Sref) / np.abs(Sref)) < tol
    scale = np.max(np.abs(Sref[:, 1])) / w.n ** 2
    assert np.max(np.abs(lscv - ref)) < tol * 10 * scale
    if prec == "f64":
        assert int(np.argmin(lscv)) == int(np.argmin(ref))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_lscv_1d(K, prec):
    w = W.lscv_small(8, 1, (300,), n=2000, count=35, precision=prec)
    lscv, S, counts, plan = run_lscv(K, w)
    ref, Sref = oracle_lscv(w, counts, range(len(w.H)))
    tol = 1e-12 if prec == "f64" else 2e-5
    assert np.max(np.abs(S.reshape(-1, 2) - Sref) / np.abs(Sref)) < tol


def test_lscv_rejects_candidates_outside_the_plan(K):
    w = W.lscv_small(9, 2, (30, 30), n=500, count=3, precision="f64")
    plan = K.Plan(w.M, w.lo, w.hi, w.H[0], precision="f64")
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    Wsp = K.kde_power_spectrum(plan, counts)
    with pytest.raises(K.KDEError) as e:
        K.kde_lscv(plan, w.n, np.stack([w.H[0] * 400.0]), Wsp)
    assert e.value.status == 1
    with pytest.raises(K.KDEError) as e:
        K.kde_lscv(plan, w.n, np.stack([np.array([[1.0, 2.0], [2.0, 1.0]]) * 1e-4]), Wsp)
    assert e.value.status == 2


def test_lscv_full_size_sampled_candidates(K):
    """512^2, n = 2e6, 1024 candidates: five candidates against the oracle's
    spectral pair sums (Eq. 10 with Parseval, plain DFT)."""
    w = W.lscv2d_512_f32()
    lscv, S, counts, plan = run_lscv(K, w)
    assert np.all(np.isfinite(lscv))
    c = O.counts_to_c(counts)
    P = plan.info.P
    rng = np.random.default_rng(3)
    for i in [int(np.argmin(lscv))] + list(rng.choice(len(w.H), 4, replace=False)):
        for h, A in enumerate((w.H[i], 2 * w.H[i])):
            L = O.support_L(A, w.lo, w.hi, w.M, w.tau)
            ref = O.binned_pair_sum_dft(c, A, w.lo, w.hi, w.M, L, P)
            assert abs(S[2 * i + h] - ref) < 2e-5 * abs(ref), (i, h)
