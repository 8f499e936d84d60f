"""Densities for many bandwidths from one count spectrum (kde_fft_eval_multi,
Eq. 10 with C = F(c) reused): every node of several candidates against the
FP64 oracle's Eq. 7 within the FP32 path's 1e-5 (max error over max value),
every candidate against the per-bandwidth path (kernel grid + evaluation),
more candidates than one launch chunk, and the full-size 512^2 workload with
1024 candidates at sampled nodes."""
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


def plan_for_all(K, w):
    """A plan whose padding fits every candidate (the widest support)."""
    big = max(w.H, key=lambda h: np.linalg.eigvalsh(h).max())
    info = K.kde_plan_info_compute(w.M, w.lo, w.hi, big, precision="f32", tau=w.tau)
    return K.Plan(w.M, w.lo, w.hi, big, precision="f32", tau=w.tau, P_min=info.P)


@pytest.mark.parametrize("count", [5, 70])
def test_small_grid_every_candidate(K, count):
    w = W.lscv_small(91 + count, 2, (96, 80), 5000, count, precision="f32", diag_lo=-3.5, diag_hi=-1.5)
    plan = plan_for_all(K, w)
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    dens = K.kde_fft_eval_multi(plan, w.n, w.H, counts).cpu().numpy()
    c_ref, _ = O.bin_linear(w.X, w.lo, w.hi, w.M)
    assert np.array_equal(counts.cpu().numpy(), c_ref)
    for h in range(count):
        # the per-bandwidth path on the same padding
        ph = K.Plan(w.M, w.lo, w.hi, w.H[h], precision="f32", tau=w.tau, P_min=plan.info.P)
        assert ph.info.P == plan.info.P
        ws = ph.workspace()
        Ks = K.kde_kernel_grid(ph, w.n, workspace=ws)
        one = K.kde_fft_eval(ph, counts, Ks, workspace=ws).cpu().numpy()
        assert rel_err(dens[h], one) <= 1e-5, h
    for h in sorted({0, count // 2, count - 1}):
        f, _, _, _ = O.binned_estimate(w.X, w.H[h], w.lo, w.hi, w.M, tau=w.tau)
        assert rel_err(dens[h], f) <= 1e-5, h


def test_full_size_candidates_sampled(K):
    w = W.lscv2d_512_f32()
    plan = plan_for_all(K, w)
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    dens = K.kde_fft_eval_multi(plan, w.n, w.H, counts)
    torch.cuda.synchronize()
    c = O.counts_to_c(counts.cpu().numpy())
    rng = np.random.default_rng(7)
    lam = np.array([np.linalg.eigvalsh(h).max() for h in w.H])
    picks = sorted({int(np.argmin(lam)), int(np.argmax(lam)), 0, 513, 1023})
    for h in picks:
        L = O.support_L(w.H[h], w.lo, w.hi, w.M, w.tau)
        k = O.kernel_weights(w.H[h], w.lo, w.hi, w.M, L, w.n)
        d = dens[h].cpu().numpy()
        nodes = np.stack([rng.integers(0, m, 1500) for m in w.M], axis=1)
        peak = np.array(np.unravel_index(np.argmax(d), d.shape))
        nodes = np.concatenate([nodes, peak[None, :]])
        ref = O.binned_direct_at(c, k, L, nodes)
        assert rel_err(d[tuple(nodes.T)], ref) <= 1e-5, h


def test_rejects_unsupported_and_bad_bandwidths(K):
    w = W.lscv_small(3, 2, (40, 36), 1000, 3, precision="f64")
    plan = K.Plan(w.M, w.lo, w.hi, w.H[0], precision="f64")
    counts = torch.zeros(w.M, dtype=torch.int64, device="cuda")
    with pytest.raises(K.KDEError) as e:
        K.kde_fft_eval_multi(plan, 10, w.H, counts, workspace=torch.empty(256, dtype=torch.uint8,
                                                                          device="cuda"))
    assert e.value.status == 7
    plan = K.Plan(w.M, w.lo, w.hi, w.H[0], precision="f32")
    with pytest.raises(K.KDEError) as e:
        K.kde_fft_eval_multi(plan, 10, [np.array([[1.0, 2.0], [2.0, 1.0]])], counts)
    assert e.value.status == 2
    wide = np.eye(2) * 1e3       # support beyond the plan's padding
    with pytest.raises(K.KDEError) as e:
        K.kde_fft_eval_multi(plan, 10, [wide], counts)
    assert e.value.status == 1
