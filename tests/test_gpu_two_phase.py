"""The two-phase FFT engine (FP32): every factor size of its generic kernels
as both factors of a line (P = s^2, split s x s) and every split that has
kernels of its own (two and three factors), on the row axis and on the column axis of small 2-D
grids, each node against the FP64 oracle within the FP32 path's 1e-5 (max
error over max value); a few unbalanced splits; 3-D grids; and the
full-size workloads against the Stockham engine."""
import os
import re

import numpy as np
import pytest

from oracle import kde_oracle as O
from paper_1508_02766_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 18, 20]


def compiled(macro):
    """The splits listed in the library's source (KDE_FX_PAIRS, KDE_FX_TRIPLES)."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "paper_1508_02766_gb300", "csrc", "fx_pairs.h")).read()
    body = text[text.index("#define " + macro):]
    body = body[:body.index("\n\n")]
    return [tuple(int(v) for v in m.split(",")) for m in re.findall(r"X\(([\d,\s]+)\)", body)]


PAIRS = compiled("KDE_FX_PAIRS") + compiled("KDE_FX_TRIPLES")


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


def case_with_P(K, seed, axis, P, other=12):
    """A 2-D FP32 problem whose padded length along `axis` is exactly P
    (forced through P_min) with the data as long as the support allows."""
    m = max(2, P - 2)
    for _ in range(100):
        M = [other, other]
        M[axis] = m
        w = W.small_case(seed, 2, tuple(M), n=2000, precision="f32")
        Pmin = [0, 0]
        Pmin[axis] = P
        info = K.kde_plan_info_compute(w.M, w.lo, w.hi, w.H, precision="f32", P_min=Pmin)
        if info.P[axis] == P or m == 2:
            break
        m = max(2, min(m - 1, P - info.L[axis]))   # M + L must fit in P
    return w, Pmin, info


def run(K, w, **opts):
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    plan = K.Plan(w.M, w.lo, w.hi, w.H, precision="f32", tau=w.tau, **opts)
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    ws = plan.workspace()
    Ks = K.kde_kernel_grid(plan, w.n, workspace=ws)
    dens = K.kde_fft_eval(plan, counts, Ks, workspace=ws)
    torch.cuda.synchronize()
    return dens.cpu().numpy(), counts, plan


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("s", SIZES)
def test_every_factor_size(K, s, axis):
    w, Pmin, info = case_with_P(K, 500 + s, axis, s * s)
    assert info.P[axis] == s * s and info.split[axis] == (s, s)
    dens, counts, plan = run(K, w, P_min=Pmin, engine="two_phase")
    assert plan.info.engine == "two_phase"
    f, c_ref, L, _ = O.binned_estimate(w.X, w.H, w.lo, w.hi, w.M, tau=w.tau)
    assert np.array_equal(counts.cpu().numpy(), c_ref)
    assert rel_err(dens, f) <= 1e-5


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("split", PAIRS)
def test_every_compiled_split(K, split, axis):
    P = int(np.prod(split))
    w, Pmin, info = case_with_P(K, 800 + P, axis, P)
    assert info.P[axis] == P and info.split[axis] == split
    dens, counts, _ = run(K, w, P_min=Pmin, engine="two_phase")
    f, c_ref, _, _ = O.binned_estimate(w.X, w.H, w.lo, w.hi, w.M, tau=w.tau)
    assert np.array_equal(counts.cpu().numpy(), c_ref)
    assert rel_err(dens, f) <= 1e-5


@pytest.mark.parametrize("split", [(2, 3), (3, 7), (5, 7), (8, 9), (9, 14), (12, 15)])
def test_unbalanced_splits(K, split):
    P = split[0] * split[1]
    for axis in (0, 1):
        w, Pmin, info = case_with_P(K, 600 + P, axis, P, other=20)
        assert info.split[axis] == split
        dens, counts, _ = run(K, w, P_min=Pmin, engine="two_phase")
        f, _, _, _ = O.binned_estimate(w.X, w.H, w.lo, w.hi, w.M, tau=w.tau)
        assert rel_err(dens, f) <= 1e-5


@pytest.mark.parametrize("M", [(20, 17, 24), (31, 9, 40), (9, 13, 2)])
def test_3d_small_every_node(K, M):
    w = W.small_case(700 + M[0], 3, M, n=3000, precision="f32")
    dens, counts, plan = run(K, w, engine="two_phase")
    f, c_ref, L, _ = O.binned_estimate(w.X, w.H, w.lo, w.hi, w.M, tau=w.tau)
    assert np.array_equal(counts.cpu().numpy(), c_ref)
    assert rel_err(dens, f) <= 1e-5


@pytest.mark.parametrize("name", ["kde2d_1024_f32", "kde3d_256_f32"])
def test_full_size_against_the_stockham_engine(K, name):
    w = W.WORKLOADS[name]()
    d2, counts, p2 = run(K, w, engine="two_phase")
    d1, _, p1 = run(K, w, engine="stockham")
    assert p2.info.engine == "two_phase" and p1.info.engine == "stockham"
    assert rel_err(d2, d1) <= 1e-5


@pytest.mark.parametrize("rows", [12, 3300])
def test_three_factor_rows_few_and_many(K, rows):
    """Long rows of a three-factor split (448 = 7 x 8 x 8), few (12) and many
    (3300, two per line in 1650 lines), against Eq. 7 at sampled nodes
    (every node of the small grid), within the FP32 1e-5."""
    w = W.small_case(77, 2, (rows, 430), n=20000 if rows > 100 else 3000, precision="f32")
    info = K.kde_plan_info_compute(w.M, w.lo, w.hi, w.H, precision="f32")
    assert info.P[1] > 400   # a three-factor line
    dens, counts, plan = run(K, w)
    L = tuple(plan.info.L)
    c = O.counts_to_c(counts.cpu().numpy())
    k = O.kernel_weights(w.H, w.lo, w.hi, w.M, L, w.n)
    rng = np.random.default_rng(3)
    if rows * 430 <= 6000:
        nodes = np.argwhere(np.ones(w.M, dtype=bool))
    else:
        nodes = np.stack([rng.integers(0, m, size=2500) for m in w.M], axis=1)
        peak = np.array(np.unravel_index(int(np.argmax(dens)), w.M))
        nodes = np.concatenate([nodes, peak[None, :]], axis=0)
    ref = O.binned_direct_at(c, k, L, nodes)
    got = dens[tuple(nodes.T)]
    assert rel_err(got, ref) <= 1e-5
