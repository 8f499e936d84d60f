"""Ragged batches (kde_batch_*): every problem of the batch against the
oracle, against the single-problem path, for every launch shape."""
import numpy as np
import pytest

from oracle import kde_oracle as O
from paper_1508_02766_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import os

    from paper_1508_02766_gb300 import build, kde
    if not os.path.exists(build.LIB):
        build.build()
    return kde


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def small_batch(prec, count=9, seed=70):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        M = (int(rng.integers(8, 90)), int(rng.integers(8, 120)))
        out.append(W.small_case(seed + i, 2, M, n=int(rng.integers(50, 3000)), precision=prec,
                                corr=float(rng.uniform(-0.8, 0.9)), scale=float(rng.uniform(0.01, 0.1))))
    return out


def run_batch(K, problems, prec, shape=None, mode="persistent", bp=None):
    if bp is None:
        bp = K.BatchPlan([(w.M, w.lo, w.hi, w.H, w.n) for w in problems], precision=prec)
    bp.set_mode(mode)
    if shape:
        bp.set_shape(*shape)
    X = torch.from_numpy(np.ascontiguousarray(np.concatenate([w.X for w in problems]))).cuda()
    dens = bp.eval(X)
    torch.cuda.synchronize()
    out, off = [], 0
    d = dens.cpu().numpy()
    for w in problems:
        m = int(np.prod(w.M))
        out.append(d[off:off + m].reshape(w.M))
        off += m
    return out, bp, X


@pytest.mark.parametrize("mode", ["persistent", "persistent-stages", "staged"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_small_ragged_batch_every_node(K, prec, mode):
    problems = small_batch(prec)
    bp = K.BatchPlan([(w.M, w.lo, w.hi, w.H, w.n) for w in problems], precision=prec)
    if mode == "persistent-stages":
        bp.set_queue_order("stages")
    dens, bp, _ = run_batch(K, problems, prec, mode=mode.split("-")[0], bp=bp)
    bp.check()
    for w, g in zip(problems, dens):
        f, _, _, _ = O.binned_estimate(w.X, w.H, w.lo, w.hi, w.M, tau=w.tau)
        assert rel_err(g, f) <= TOL[prec]


@pytest.mark.parametrize("mode,shape", [("staged", (32, 32)), ("staged", (64, 128)),
                                        ("staged", (128, 64)), ("staged", (128, 128)),
                                        ("persistent", (32, 32)), ("persistent", (128, 128))])
def test_every_launch_shape(K, shape, mode):
    problems = small_batch("f64", count=5, seed=90)
    dens, _, _ = run_batch(K, problems, "f64", shape, mode)
    for w, g in zip(problems, dens):
        f, _, _, _ = O.binned_estimate(w.X, w.H, w.lo, w.hi, w.M, tau=w.tau)
        assert rel_err(g, f) <= 1e-12


def test_ragged64_against_single_problem_path_and_tuner(K):
    problems = W.ragged64_f32()
    dens, bp, X = run_batch(K, problems, "f32")
    density = torch.empty(bp.density_elems, dtype=torch.float32, device="cuda")
    # room for the longer paddings the tuner may choose
    ws = torch.empty(2 * bp.workspace_bytes, dtype=torch.uint8, device="cuda")
    ms = bp.tune(X, density, ws, reps=2)
    assert ms > 0 and bp.shape()[0] in (32, 64, 128)
    pad, order, P, queue = bp.config(len(problems))
    assert queue in ("stages", "problems")
    assert pad in ("smallest", "fewest_stages") and order in ("largest_first", "smallest_first")
    assert all(Pk >= m for (p2, w) in zip(P, problems) for Pk, m in zip(p2, w.M))
    assert bp.workspace_bytes <= ws.numel()
    tuned = bp.eval(X, density, ws).cpu().numpy()
    bp.check()
    off = 0
    rng = np.random.default_rng(2)
    check = set(rng.choice(len(problems), 10, replace=False).tolist())
    for i, (w, g) in enumerate(zip(problems, dens)):
        m = int(np.prod(w.M))
        assert np.allclose(tuned[off:off + m].reshape(w.M), g, rtol=0, atol=1e-5 * np.abs(g).max())
        off += m
        if i not in check:
            continue
        Xd = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
        single, _, _ = K.kde_eval(Xd, w.H, w.lo, w.hi, w.M, precision="f32")
        assert rel_err(g, single.cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_samples_on_grid_edges_and_outside(K, prec):
    """Samples exactly on the grid's edges and corners (a node of the last
    row or column: its far corners have weight 0) and outside the grid
    (dropped; in FP32 an edge sample may round outside, as in the oracle),
    in a batch of three grids, against the oracle."""
    import dataclasses
    problems = []
    for i, M in enumerate([(17, 23), (40, 9), (64, 64)]):
        w = W.small_case(400 + i, 2, M, n=500, precision=prec)
        lo, hi = np.asarray(w.lo, dtype=np.float64), np.asarray(w.hi, dtype=np.float64)
        t = np.linspace(0.0, 1.0, 7)
        edge = np.concatenate([
            np.stack([np.full(7, hi[0]), lo[1] + t * (hi[1] - lo[1])], 1),
            np.stack([lo[0] + t * (hi[0] - lo[0]), np.full(7, hi[1])], 1),
            np.array([[lo[0], lo[1]], [hi[0], hi[1]], [lo[0], hi[1]], [hi[0], lo[1]]]),
            np.array([[hi[0] + 1.0, 0.5 * (lo[1] + hi[1])], [lo[0] - 1.0, lo[1] - 1.0]]),
        ])
        X = np.concatenate([w.X.astype(np.float64), edge]).astype(w.X.dtype)
        problems.append(dataclasses.replace(w, X=X))
    dens, _, _ = run_batch(K, problems, prec)
    for w, g in zip(problems, dens):
        f, _, _, n_out = O.binned_estimate(w.X, w.H, w.lo, w.hi, w.M, tau=w.tau)
        assert n_out >= 2
        assert rel_err(g, f) <= TOL[prec]


def test_persistent_wait_runs_out_and_recovers(K):
    """A stage whose completions are withheld (count rows): the middle-axis
    items wait for them, give up after their poll limit, and the status says
    so; nothing faults or hangs, and the next launch (normal waits) gives the
    right densities."""
    import time
    problems = small_batch("f32", count=4, seed=120)
    good, bp, X = run_batch(K, problems, "f32")
    bp.check()
    bp.set_wait(2000, withhold_stage=4)
    t0 = time.perf_counter()
    bp.eval(X)
    with pytest.raises(K.KDEError) as e:
        bp.check()
    assert e.value.status == 6
    assert time.perf_counter() - t0 < 30.0
    bp.set_wait(1 << 22, withhold_stage=-1)
    again = bp.eval(X).cpu().numpy()
    bp.check()
    off = 0
    for g in good:
        m = g.size
        assert np.array_equal(again[off:off + m].reshape(g.shape), g)
        off += m
