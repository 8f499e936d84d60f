"""The path at the largest padded length (P_k = KDE_MAX_P = 4096) and on
either side of the length where FP32 plans leave the two-phase engine for
the Stockham one, against the oracle on every node.

Eq. 7 does not depend on P once P_k >= M_k + L_k (Eq. 10 then has no
wrap-around), so small grids planned with a requested minimum length
(P_min) reach these lengths while the oracle stays cheap.  Counts are
compared bit for bit, densities within 1e-12 (FP64) or 1e-5 (FP32) of the
oracle's maximum.
"""
import numpy as np
import pytest

from oracle import kde_oracle as O
from paper_1508_02766_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_P = 4096
TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1508_02766_gb300 import build, kde
    import os
    if not os.path.exists(build.LIB):
        build.build()
    return kde


def run_case(K, w, P_min):
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    plan = K.Plan(w.M, w.lo, w.hi, w.H, precision=w.precision, tau=w.tau, P_min=P_min)
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    ws = plan.workspace()
    Ks = K.kde_kernel_grid(plan, w.n, workspace=ws)
    dens = K.kde_fft_eval(plan, counts, Ks, workspace=ws)
    torch.cuda.synchronize()
    f, c_ref, L, _ = O.binned_estimate(w.X, w.H, w.lo, w.hi, w.M, tau=w.tau)
    assert plan.info.L == tuple(L)
    assert np.array_equal(counts.cpu().numpy(), c_ref)
    got = dens.cpu().numpy()
    err = float(np.max(np.abs(got - f)) / np.max(np.abs(f)))
    assert err <= TOL[w.precision], (w.M, plan.info.P, err)
    return plan.info


LIMIT_CASES = [
    (1, (1500,), "f64", (MAX_P,)),
    (1, (1500,), "f32", (MAX_P,)),
    (2, (900, 40), "f32", (MAX_P, 0)),
    (2, (40, 900), "f64", (0, MAX_P)),
    (2, (300, 120), "f32", (0, MAX_P)),
    (3, (6, 7, 300), "f32", (0, 0, MAX_P)),
]


@pytest.mark.parametrize("d,M,prec,P_min", LIMIT_CASES)
def test_largest_padded_length(K, d, M, prec, P_min):
    w = W.small_case(700 + d, d, M, n=3000, precision=prec, scale=2e-3)
    info = run_case(K, w, P_min)
    assert max(info.P) == MAX_P


def test_either_side_of_the_two_phase_engine_s_longest_line(K):
    from paper_1508_02766_gb300 import kde
    w = W.small_case(711, 2, (200, 40), n=3000, precision="f32", scale=2e-3)
    # the longest axis-0 requirement the two-phase engine plans
    last = max(p for p in range(256, MAX_P + 1, 1)
               if kde.kde_plan_info_compute(w.M, w.lo, w.hi, w.H, precision="f32", tau=w.tau,
                                            P_min=(p, 0)).engine == "two_phase")
    assert last < MAX_P
    a = run_case(K, w, (last, 0))
    b = run_case(K, w, (last + 1, 0))
    assert a.engine == "two_phase" and b.engine == "stockham"
    assert a.P[0] >= last and b.P[0] >= last + 1
