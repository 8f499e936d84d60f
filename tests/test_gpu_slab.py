"""Slab passes of 3-D evaluations (thread-block clusters, Eq. 10).

The slab kernels run the same transforms with the same arithmetic as the
separate row and column passes; only where the intermediate half spectra
live differs (distributed shared memory instead of global memory).  The
compiler may contract multiply-adds differently in the two kernels, so the
densities agree to rounding (1e-6 of the peak, a few FP32 ulps), and each
matches the oracle within the FP32 tolerance.  Every evaluation is followed
by kde_plan_check: a bounded exchange wait that gave up fails the test.  The
shapes cover ragged slabs: odd M1 (an unpaired last row), Q not a multiple
of 8 (a partial last column block), slabs with fewer rows or columns than
the cluster has blocks, and axes 1 and 2 with different splits (the generic
kernel).
"""
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
    from paper_1508_02766_gb300 import build, kde
    import os
    if not os.path.exists(build.LIB):
        build.build()
    return kde


def close(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))) <= 1e-6


def evaluate(K, w, counts, slab):
    plan = K.Plan(w.M, w.lo, w.hi, w.H, precision="f32", tau=w.tau, slab=slab)
    ws = plan.workspace()
    Ks = K.kde_kernel_grid(plan, w.n, workspace=ws)
    before = K.launch_count()
    dens = K.kde_fft_eval(plan, counts, Ks, workspace=ws)
    launches = K.launch_count() - before
    K.plan_check(plan)
    return dens.cpu().numpy(), plan, launches


SHAPES = [
    (20, 17, 24),   # odd M1
    (2, 2, 2),      # every block but one idle
    (6, 31, 45),    # odd M1, Q not a multiple of 8
    (3, 64, 100),
    (12, 9, 3),     # Q smaller than the cluster
    (5, 40, 130),
]


@pytest.mark.parametrize("M", SHAPES)
def test_slab_equals_separate_passes_and_oracle(K, M):
    w = W.small_case(11, 3, M, n=3000, precision="f32")
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    got, plan, launches = evaluate(K, w, counts, "on")
    ref, plan_off, launches_off = evaluate(K, w, counts, "off")
    assert plan.info.engine == "two_phase"
    assert plan.info.slab_passes and not plan_off.info.slab_passes
    assert launches == 3 and launches_off == 5
    assert close(got, ref)
    exp = O.binned_estimate(w.X, w.H, w.lo, w.hi, w.M, tau=w.tau)[0]
    assert float(np.max(np.abs(got - exp)) / np.max(np.abs(exp))) <= 1e-5


def test_slab_generic_kernel_for_unequal_splits(K):
    # axes 1 and 2 padded to different lengths: not one of the compiled pairs
    w = W.small_case(5, 3, (7, 50, 70), n=4000, precision="f32",
                     H=np.diag([0.02, 0.01, 0.08]))
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    got, plan, _ = evaluate(K, w, counts, "on")
    assert plan.info.slab_passes
    assert plan.info.split[1] != plan.info.split[2]
    ref, _, _ = evaluate(K, w, counts, "off")
    assert close(got, ref)
    exp = O.binned_estimate(w.X, w.H, w.lo, w.hi, w.M, tau=w.tau)[0]
    assert float(np.max(np.abs(got - exp)) / np.max(np.abs(exp))) <= 1e-5


def test_slab_full_size_equals_separate_passes(K):
    w = W.WORKLOADS["kde3d_256_f32"]()
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    got, plan, _ = evaluate(K, w, counts, "on")
    assert plan.info.slab_passes
    ref, _, _ = evaluate(K, w, counts, "off")
    assert close(got, ref)


def test_slab_noalloc_and_repeat(K):
    w = W.small_case(3, 3, (10, 33, 47), n=2000, precision="f32")
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    a, _, _ = evaluate(K, w, counts, "on")
    b, _, _ = evaluate(K, w, counts, "on")
    assert np.array_equal(a, b)
    plan = K.Plan(w.M, w.lo, w.hi, w.H, precision="f32", tau=w.tau, slab="on")
    assert plan.info.slab_passes
    Ks = K.kde_kernel_grid(plan, w.n, workspace=plan.workspace())
    out = torch.empty(w.M, dtype=torch.float32, device="cuda")
    K.kde_fft_eval_noalloc(plan, counts, Ks, out)
    K.plan_check(plan)
    assert np.array_equal(a, out.cpu().numpy())
