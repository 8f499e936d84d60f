"""Nearly singular bandwidths (correlation within 5e-4 of +-1) against the
FP64 oracle.  The kernel's exponent near the long axis of such an H is a
small difference of large products of lags; in FP32 the expanded quadratic
form loses it to cancellation (about 5e-5 relative on the 2-D density case
below), the completed squares of the Cholesky factor do not."""
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


def rel_err(gpu, ref):
    return float(np.max(np.abs(gpu - ref)) / np.max(np.abs(ref)))


def density(K, w):
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    plan = K.Plan(w.M, w.lo, w.hi, w.H, precision=w.precision, tau=w.tau)
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    ws = plan.workspace()
    Ks = K.kde_kernel_grid(plan, w.n, workspace=ws)
    dens = K.kde_fft_eval(plan, counts, Ks, workspace=ws)
    torch.cuda.synchronize()
    return dens.cpu().numpy()


def singular_3d(scale):
    Q, _ = np.linalg.qr(np.random.default_rng(1).normal(size=(3, 3)))
    return scale * Q @ np.diag([1.0, 0.1, 2e-4]) @ Q.T


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("case", ["2d", "3d"])
def test_density(K, case, prec):
    if case == "2d":
        H = W.rotated_bandwidth(0.02, 0.02 * 2e-4, np.pi / 4 + 0.1)
        w = W.small_case(11, 2, (96, 80), n=3000, precision=prec, H=H)
    else:
        w = W.small_case(13, 3, (40, 36, 44), n=3000, precision=prec, H=singular_3d(0.05))
    f, _, _, _ = O.binned_estimate(w.X, w.H, w.lo, w.hi, w.M, tau=w.tau)
    assert rel_err(density(K, w), f) <= (1e-5 if prec == "f32" else 1e-12)


def test_lscv_pair_sums_both_paths(K):
    """Eight candidates with eigenvalue ratios 1e-4 .. 1e-3 at assorted
    angles: the autocorrelation and the spectrum-dot pair sums, each against
    the oracle's direct binned sum within its FP32 tolerance."""
    rng = np.random.default_rng(21)
    base = W.lscv_small(21, 2, (96, 96), n=3000, count=1, precision="f32")
    H = np.stack([W.rotated_bandwidth(0.03, 0.03 * r, a)
                  for r, a in zip(np.geomspace(1e-4, 1e-3, 8), rng.uniform(0, np.pi, 8))])
    lam = max(float(np.linalg.eigvalsh(h).max()) for h in H)
    pad = 4.0 * np.sqrt(lam)
    X = base.X.astype(np.float64)
    w = W.LscvWorkload("lscv_singular", base.X, H, X.min(axis=0) - pad, X.max(axis=0) + pad,
                       (96, 96), "f32")
    lam2 = [np.linalg.eigvalsh(h).max() for h in H]
    big = 2.0 * H[int(np.argmax(lam2))]
    info = K.kde_plan_info_compute(w.M, w.lo, w.hi, big, precision="f32", tau=w.tau)
    plan = K.Plan(w.M, w.lo, w.hi, big, precision="f32", tau=w.tau, P_min=info.P)
    Xd = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    counts = K.kde_bin(Xd, w.lo, w.hi, w.M)
    R = K.kde_autocorrelation(plan, counts)
    S_ac = torch.empty(2 * len(H), dtype=torch.float64, device="cuda")
    K.kde_lscv_autocorr(plan, w.n, H, R, pair_sums=S_ac)
    Wsp = K.kde_power_spectrum(plan, counts)
    S_sp = torch.empty(2 * len(H), dtype=torch.float64, device="cuda")
    K.kde_lscv(plan, w.n, H, Wsp, pair_sums=S_sp)
    torch.cuda.synchronize()
    c = O.counts_to_c(counts.cpu().numpy())
    ref = []
    for h in H:
        for A in (h, 2 * h):
            L = O.support_L(A, w.lo, w.hi, w.M, w.tau)
            ref.append(O.binned_pair_sum(c, A, w.lo, w.hi, w.M, L))
    ref = np.array(ref)
    assert np.max(np.abs(S_ac.cpu().numpy() - ref) / ref) < 2e-6
    assert np.max(np.abs(S_sp.cpu().numpy() - ref) / ref) < 2e-5
