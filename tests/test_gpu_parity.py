"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

Counts must be bit-identical.  Densities are compared as max |gpu - oracle|
divided by max |oracle| over the compared nodes: at most 1e-12 on the FP64
path and 1e-5 on the FP32 path.  Small grids are compared on every node;
the full-size workloads on sampled nodes (plus a window around the peak),
with the oracle evaluating Eq. 7 node by node.
"""
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
    from paper_1508_02766_gb300 import build, kde
    import os
    if not os.path.exists(build.LIB):
        build.build()
    return kde


def rel_err(gpu, ref):
    return float(np.max(np.abs(gpu - ref)) / np.max(np.abs(ref)))


def run_gpu(K, w, method="tiled", **opts):
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    plan = K.Plan(w.M, w.lo, w.hi, w.H, precision=w.precision, tau=w.tau, **opts)
    nout = torch.zeros(1, dtype=torch.int64, device="cuda")
    counts = K.kde_bin(X, w.lo, w.hi, w.M, n_outside=nout, method=method)
    ws = plan.workspace()
    Ks = K.kde_kernel_grid(plan, w.n, workspace=ws)
    dens = K.kde_fft_eval(plan, counts, Ks, workspace=ws)
    torch.cuda.synchronize()
    return dens.cpu().numpy(), counts.cpu().numpy(), int(nout.item()), plan


def oracle_full(w, range_mode="corrected", layout="corrected"):
    return O.binned_estimate(w.X, w.H, w.lo, w.hi, w.M, tau=w.tau, range_mode=range_mode,
                             layout=layout)


SMALL = [
    (1, (700,), "f64"), (1, (700,), "f32"), (1, (2,), "f64"),
    (2, (37, 53), "f64"), (2, (37, 53), "f32"), (2, (130, 67), "f32"), (2, (2, 3), "f64"),
    (3, (9, 13, 11), "f64"), (3, (20, 17, 24), "f32"), (3, (2, 2, 2), "f32"),
]


@pytest.mark.parametrize("method,cols,engine", [("tiled", "lines", "auto"), ("direct", "simd", "auto"),
                                                ("direct", "lines", "stockham")])
@pytest.mark.parametrize("d,M,prec", SMALL)
def test_small_grids_every_node(K, d, M, prec, method, cols, engine):
    w = W.small_case(100 + d * 7 + len(M) + M[0], d, M, n=3000, precision=prec)
    dens, counts, nout, plan = run_gpu(K, w, method=method, cols=cols, engine=engine)
    f, c_ref, L, nout_ref = oracle_full(w)
    assert plan.info.L == L
    assert nout == nout_ref
    assert np.array_equal(counts, c_ref)
    assert rel_err(dens, f) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_support_is_whole_grid(K, prec):
    """L = M - 1 on every axis (a wide H): every lag of Eq. 5 is kept."""
    w = W.small_case(7, 2, (24, 19), n=500, precision=prec)
    w.tau = 40.0                          # tau sqrt(lambda) / delta > M - 1 on both axes
    dens, counts, _, plan = run_gpu(K, w)
    assert plan.info.L == (23, 18)
    f, c_ref, L, _ = oracle_full(w)
    assert np.array_equal(counts, c_ref)
    assert rel_err(dens, f) <= TOL[prec]


def test_kde2d_128_f64_every_node(K):
    w = W.kde2d_128_f64()
    dens, counts, nout, plan = run_gpu(K, w)
    f, c_ref, L, nout_ref = oracle_full(w)
    assert nout == nout_ref == 0
    assert np.array_equal(counts, c_ref)
    assert int(counts.sum()) == w.n << 32
    assert rel_err(dens, f) <= 1e-12


def sampled_nodes(rng, M, dens, m=3000, window=5):
    nodes = np.stack([rng.integers(0, Mk, m) for Mk in M], axis=1)
    peak = np.array(np.unravel_index(np.argmax(dens), dens.shape))
    offs = np.stack(np.meshgrid(*[np.arange(-window, window + 1)] * len(M), indexing="ij"),
                    -1).reshape(-1, len(M))
    win = np.clip(peak + offs, 0, np.array(M) - 1)
    return np.concatenate([nodes, win])


@pytest.mark.parametrize("name", ["kde2d_1024_f32", "kde3d_256_f32"])
def test_full_size_sampled_nodes(K, name):
    w = W.WORKLOADS[name]()
    dens, counts, nout, plan = run_gpu(K, w)
    assert int(counts.sum()) == (w.n - nout) << 32
    L = O.support_L(w.H, w.lo, w.hi, w.M, w.tau)
    assert plan.info.L == L
    k = O.kernel_weights(w.H, w.lo, w.hi, w.M, L, w.n)
    rng = np.random.default_rng(1)
    nodes = sampled_nodes(rng, w.M, dens, m=3000 if w.d == 2 else 1500, window=5 if w.d == 2 else 2)
    # Counts: the oracle's binning on the same samples.
    c_ref, nout_ref = O.bin_linear(w.X, w.lo, w.hi, w.M)
    assert nout == nout_ref
    assert np.array_equal(counts, c_ref)
    ref = O.binned_direct_at(O.counts_to_c(c_ref), k, L, nodes)
    got = dens[tuple(nodes.T)]
    assert rel_err(got, ref) <= 1e-5


def test_per_axis_range_truncates_correlated_kernel(K):
    """Sec. 4.2 / Eq. 15: with correlation .95 the per-axis range drops kernel
    mass the corrected range keeps; the GPU reproduces both estimates."""
    w = W.kde2d_1024_f32(n=200_000)
    w.M = (256, 256)
    d_c, _, _, pc = run_gpu(K, w)
    d_a, _, _, pa = run_gpu(K, w, range_mode="per_axis")
    assert all(a < c for a, c in zip(pa.info.L, pc.info.L))
    f_c, _, _, _ = oracle_full(w)
    f_a, _, _, _ = oracle_full(w, range_mode="per_axis")
    assert rel_err(d_c, f_c) <= 1e-5
    assert rel_err(d_a, f_a) <= 1e-5
    # The two estimates differ by more than the FP32 tolerance, as the
    # oracle's do, and by the same amount.
    assert rel_err(d_a, d_c) > 2e-5
    assert abs(rel_err(d_a, d_c) - rel_err(f_a, f_c)) < 2e-6


def test_wand_layout_matches_oracle_and_fails_for_full_H(K):
    """Wand's layout (Eq. 8) on the GPU equals the oracle's k_{|l|} sum, and
    differs from the corrected estimate by O(1) for correlated H (Figure 1(b))."""
    w = W.small_case(3, 2, (64, 48), n=2000, precision="f64", corr=0.9)
    d_w, _, _, _ = run_gpu(K, w, layout="wand")
    d_c, _, _, _ = run_gpu(K, w)
    f_w, _, _, _ = oracle_full(w, layout="wand")
    assert rel_err(d_w, f_w) <= 1e-12
    assert rel_err(d_w, d_c) > 1e-2


def test_wand_layout_exact_for_diagonal_H(K):
    w = W.small_case(4, 3, (12, 10, 9), n=800, precision="f64", H=np.diag([0.02, 0.05, 0.03]))
    d_w, _, _, _ = run_gpu(K, w, layout="wand")
    d_c, _, _, _ = run_gpu(K, w)
    assert rel_err(d_w, d_c) <= 1e-13


@pytest.mark.parametrize("method", ["tiled", "direct"])
def test_edge_samples_and_outside(K, method):
    """Samples exactly at lo/hi, on nodes, outside and NaN (binning spec)."""
    rng = np.random.default_rng(5)
    for dt, prec in [(np.float64, "f64"), (np.float32, "f32")]:
        X = rng.uniform(-0.1, 1.1, size=(4000, 2)).astype(dt)
        X[:10] = 1.0
        X[10:20] = 0.0
        X[20:30, 1] = np.nan
        X[30:60] = (rng.integers(0, 20, size=(30, 2)) / 19.0).astype(dt)
        w = W.Workload("edges", X, np.array([[0.01, 0.004], [0.004, 0.008]]), np.zeros(2),
                       np.ones(2), (20, 23), prec)
        dens, counts, nout, _ = run_gpu(K, w, method=method)
        f, c_ref, _, nout_ref = oracle_full(w)
        assert nout == nout_ref and nout > 20
        assert np.array_equal(counts, c_ref)
        assert rel_err(dens, f) <= TOL[prec]


def test_empty_input_and_errors(K):
    X = torch.empty((0, 2), dtype=torch.float32, device="cuda")
    for method in ("tiled", "direct"):
        nout = torch.full((1,), 7, dtype=torch.int64, device="cuda")
        counts = torch.full((5, 6), 3, dtype=torch.int64, device="cuda")
        K.kde_bin(X, (0, 0), (1, 1), (5, 6), counts=counts, n_outside=nout, method=method)
        torch.cuda.synchronize()
        assert counts.abs().sum().item() == 0 and nout.item() == 0
    Xs = torch.zeros((10, 2), dtype=torch.float32, device="cuda")
    tiny = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(K.KDEError) as e:
        K.kde_bin(Xs, (0, 0), (1, 1), (5, 6), workspace=tiny[:16], method="tiled")
    assert e.value.status == 4
    plan = K.Plan((5, 6), (0, 0), (1, 1), np.eye(2) * 0.01)
    with pytest.raises(K.KDEError) as e:
        K.kde_kernel_grid(plan, 0)
    assert e.value.status == 1
    small_ws = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(K.KDEError) as e:
        K.kde_kernel_grid(plan, 10, workspace=small_ws)
    assert e.value.status == 4


def test_deterministic_and_launch_count(K):
    w = W.kde2d_1024_f32(n=300_000)
    before = K.launch_count()
    a, ca, _, _ = run_gpu(K, w)
    mid = K.launch_count()
    b, cb, _, _ = run_gpu(K, w)
    assert np.array_equal(ca, cb)
    assert np.array_equal(a, b)
    assert mid - before >= 5       # twiddles, bin, kernel grid (2), eval (3)


def test_tiled_binning_heavy_tiles(K):
    """Most samples in one tile (split into several work items whose partial
    tiles are merged), in 2-D and 3-D."""
    rng = np.random.default_rng(41)
    for d, M in [(2, (128, 256)), (3, (48, 48, 96))]:
        n = 300_000
        X = np.concatenate([rng.normal(0.3, 0.01, size=(n, d)), rng.uniform(0, 1, size=(n // 10, d))])
        lo, hi = np.zeros(d), np.ones(d)
        Xd = torch.from_numpy(np.ascontiguousarray(X.astype(np.float32))).cuda()
        counts = K.kde_bin(Xd, lo, hi, M, method="tiled").cpu().numpy()
        c_ref, _ = O.bin_linear(X.astype(np.float32), lo, hi, M)
        assert np.array_equal(counts, c_ref)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_tiled_binning_carries(K, d):
    """Every sample at one point (each adds about 2^31 to the same cells, so
    the low 32-bit word of a cell overflows on every other sample) or exactly
    on one node (weight 2^32 to one cell): the shared accumulators carry into
    the high word exactly."""
    M = {1: (300,), 2: (40, 50), 3: (12, 10, 14)}[d]
    lo, hi = np.zeros(d), np.array(M, dtype=np.float64) - 1.0
    n = 300_000
    X = np.concatenate([np.full((n, d), 5.7), np.full((n // 3, d), 3.0), np.full((n // 5, d), 7.25)])
    for dt in (np.float32, np.float64):
        Xd = torch.from_numpy(np.ascontiguousarray(X.astype(dt))).cuda()
        counts = K.kde_bin(Xd, lo, hi, M, method="tiled").cpu().numpy()
        c_ref, _ = O.bin_linear(X.astype(dt), lo, hi, M)
        assert np.array_equal(counts, c_ref)
        assert int(counts.sum()) == X.shape[0] << 32


@pytest.mark.parametrize("name", ["kde2d_1024_f32", "kde3d_256_f32"])
def test_tiled_and_direct_binning_identical(K, name):
    """The two binning methods give bit-identical counts at full size, and the
    tiled one writes every cell (the output starts as garbage)."""
    w = W.WORKLOADS[name]()
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    a = torch.full(w.M, -5, dtype=torch.int64, device="cuda")
    b = torch.full(w.M, -7, dtype=torch.int64, device="cuda")
    K.kde_bin(X, w.lo, w.hi, w.M, counts=a, method="tiled")
    K.kde_bin(X, w.lo, w.hi, w.M, counts=b, method="direct")
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert int(a.sum().item()) == w.n << 32


@pytest.mark.parametrize("d,M", [(1, (9000,)), (2, (70, 150)), (3, (40, 35, 70))])
def test_tiled_binning_tile_faces(K, d, M):
    """Samples whose base node is the last node of a tile along one or more
    axes feed the neighbouring tile; place many samples there and on nodes."""
    rng = np.random.default_rng(31 + d)
    tile = {1: (8192,), 2: (64, 128), 3: (16, 16, 32)}[d]
    n = 20000
    faces = [np.arange(t - 1, m - 1, t) for t, m in zip(tile, M)]
    idx = np.stack([rng.choice(f, n) if len(f) else rng.integers(0, m - 1, n)
                    for f, m in zip(faces, M)], axis=1).astype(np.float64)
    frac = rng.uniform(0, 1, size=(n, d))
    frac[: n // 4] = 0.0
    frac[n // 4: n // 2] = rng.integers(0, 2, size=(n // 4, d)) * 0.999999
    lo, hi = np.zeros(d), np.array(M, dtype=np.float64) - 1.0   # s = 1: t = x
    X = np.clip(idx + frac, 0, hi)
    rand = rng.uniform(0, hi, size=(n, d))
    X = np.ascontiguousarray(np.concatenate([X, rand]))
    Xd = torch.from_numpy(X).cuda()
    nout = torch.zeros(1, dtype=torch.int64, device="cuda")
    counts = K.kde_bin(Xd, lo, hi, M, n_outside=nout, method="tiled").cpu().numpy()
    c_ref, nout_ref = O.bin_linear(X, lo, hi, M)
    assert int(nout.item()) == nout_ref == 0
    assert np.array_equal(counts, c_ref)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_many_line_lengths(K, prec):
    """Grids whose padded lengths cover every radix of the engine (direct and
    nested), in 1-D and 2-D, against the oracle on every node."""
    seen = set()
    for i, M in enumerate(list(range(2, 420, 17)) + [511, 767, 1000]):
        w = W.small_case(500 + i, 1, (M,), n=400, precision=prec)
        dens, counts, _, plan = run_gpu(K, w)
        seen.update(plan.info.radices[0])
        f, c_ref, _, _ = oracle_full(w)
        assert np.array_equal(counts, c_ref)
        assert rel_err(dens, f) <= TOL[prec], (M, plan.info.P)
    for i, M in enumerate([(9, 70), (33, 21), (50, 100), (75, 40)]):
        w = W.small_case(600 + i, 2, M, n=800, precision=prec)
        dens, counts, _, plan = run_gpu(K, w, cols=("simd" if i % 2 else "lines"))
        for r in plan.info.radices:
            seen.update(r)
        f, c_ref, _, _ = oracle_full(w)
        assert rel_err(dens, f) <= TOL[prec], (M, plan.info.P)
    assert seen >= {2, 3, 4, 5, 7, 8}, sorted(seen)


def test_direct_binning_after_producer_kernel_and_unaligned_counts(K):
    """The binning kernel starts as a programmatic dependent of the kernel
    that zeroes the counts and loads its first samples before it waits:
    samples written by a kernel just before the call, and counts that start
    8 bytes past a 16-byte boundary (the zeroing kernel's scalar path),
    still give the oracle's counts exactly."""
    w = W.small_case(77, 2, (300, 257), n=200_000, precision="f32")
    base = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    for _ in range(3):
        X = (base * 1.0).contiguous()          # produced by a kernel on the stream
        store = torch.full((300 * 257 + 1,), -3, dtype=torch.int64, device="cuda")
        counts = store[1:].view(300, 257)       # 8-byte offset
        K.kde_bin(X, w.lo, w.hi, w.M, counts=counts, method="direct")
        torch.cuda.synchronize()
        c_ref, _ = O.bin_linear(w.X, w.lo, w.hi, w.M)
        assert np.array_equal(counts.cpu().numpy(), c_ref)
        assert int(store[0].item()) == -3


def test_binning_size_limits_are_refused_before_any_launch(K):
    """The bounds under which the int64 counts in units of 2^-32 cannot
    overflow (every cell below n 2^32 < 2^63 needs n < 2^31) and the grid
    limits are checked on the host: each call below returns
    KDE_ERR_INVALID_ARG (1) or KDE_ERR_UNSUPPORTED (7) and writes nothing
    (the counts keep their marker value); the same call inside the bounds
    then bins."""
    import ctypes
    L = K.lib()
    X = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    counts = torch.full((8,), 5, dtype=torch.int64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(fn, n, d, M, x=X):
        return fn(ctypes.c_void_p(x.data_ptr()), K.F32, n, d, K._darr([0.0] * d), K._darr([1.0] * d),
                  K._iarr(M), ctypes.c_void_p(counts.data_ptr()), ctypes.c_void_p(0),
                  ctypes.c_void_p(0), 0, s)

    for fn in (L.kde_bin, L.kde_bin_accumulate):
        assert call(fn, 1 << 31, 2, (4, 2)) == 1          # n >= 2^31
        assert call(fn, -1, 2, (4, 2)) == 1
        assert call(fn, 4, 2, ((1 << 24) + 1, 2)) == 1    # M_k > 2^24
        assert call(fn, 4, 3, (1 << 14, 1 << 14, 1 << 12)) == 1   # prod(M) >= 2^40
        assert call(fn, 4, 2, (1, 8)) == 1                # M_k < 2
        assert call(fn, 4, 4, (2, 2, 2, 2)) == 7          # d = 4
    torch.cuda.synchronize()
    assert torch.all(counts == 5)
    # the same call with sizes inside the bounds runs: four samples at lo,
    # all on node 0
    assert call(L.kde_bin, 4, 2, (4, 2)) == 0
    torch.cuda.synchronize()
    assert int(counts[0].item()) == 4 << 32 and int(counts[1:].abs().sum().item()) == 0
