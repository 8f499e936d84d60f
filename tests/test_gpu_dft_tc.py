"""The tensor-core first pass (opts dft_tc): the counts rows' DFT as a split
TF32 matrix product.  Densities against the FP64 oracle within the FP32
path's 1e-5 (max error over max value), on small ragged grids in full and on
the full-size workloads at sampled nodes; the count spectrum against the
FFT path's; and the plan's checks."""
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


def rel_err(gpu, ref):
    return float(np.max(np.abs(gpu - ref)) / np.max(np.abs(ref)))


def run(K, w, **opts):
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    plan = K.Plan(w.M, w.lo, w.hi, w.H, precision="f32", tau=w.tau, **opts)
    counts = K.kde_bin(X, w.lo, w.hi, w.M, method="direct")
    ws = plan.workspace()
    Ks = K.kde_kernel_grid(plan, w.n, workspace=ws)
    dens = K.kde_fft_eval(plan, counts, Ks, workspace=ws)
    torch.cuda.synchronize()
    K.plan_check(plan)   # no tensor-core wait gave up (else the output is invalid)
    return dens.cpu().numpy(), counts, plan


# rows not a multiple of the 128-row tile, last axis not a multiple of 32
@pytest.mark.parametrize("d,M", [(2, (37, 53)), (2, (130, 67)), (2, (200, 33)), (3, (20, 17, 24)),
                                 (3, (9, 13, 40))])
def test_small_grids_every_node(K, d, M):
    w = W.small_case(300 + d + M[0], d, M, n=3000, precision="f32")
    dens, _, _ = run(K, w, dft="tc")
    f, _, _, _ = O.binned_estimate(w.X, w.H, w.lo, w.hi, w.M, tau=w.tau)
    assert rel_err(dens, f) <= 1e-5
    dens_fft, _, _ = run(K, w)
    assert rel_err(dens, dens_fft) <= 1e-5


@pytest.mark.parametrize("name", ["kde2d_1024_f32", "kde3d_256_f32"])
def test_full_size_sampled_nodes(K, name):
    w = W.WORKLOADS[name]()
    dens, counts, plan = run(K, w, dft="tc")
    L = O.support_L(w.H, w.lo, w.hi, w.M, w.tau)
    k = O.kernel_weights(w.H, w.lo, w.hi, w.M, L, w.n)
    rng = np.random.default_rng(4)
    m = 2000 if w.d == 2 else 800
    nodes = np.stack([rng.integers(0, Mk, m) for Mk in w.M], axis=1)
    peak = np.unravel_index(np.argmax(dens), dens.shape)
    nodes = np.concatenate([nodes, np.array(peak)[None, :]])
    ref = O.binned_direct_at(O.counts_to_c(counts.cpu().numpy()), k, L, nodes)
    got = dens[tuple(nodes.T)]
    assert rel_err(got, ref) <= 1e-5


def test_power_spectrum_matches_fft_path(K):
    w = W.small_case(77, 2, (150, 97), n=5000, precision="f32")
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    counts = K.kde_bin(X, w.lo, w.hi, w.M, method="direct")
    out = []
    for dft in ("fft", "tc"):
        plan = K.Plan(w.M, w.lo, w.hi, w.H, precision="f32", dft=dft)
        out.append(K.kde_power_spectrum(plan, counts, workspace=plan.workspace()).cpu().numpy())
        K.plan_check(plan)
    assert rel_err(out[1], out[0]) <= 2e-5


def test_plan_rejects_tc_where_unsupported(K):
    with pytest.raises(K.KDEError) as e:
        K.Plan((64, 64), (0, 0), (1, 1), np.eye(2) * 1e-3, precision="f64", dft="tc")
    assert e.value.status == 7
    with pytest.raises(K.KDEError) as e:
        K.Plan((64,), (0,), (1,), np.eye(1) * 1e-3, precision="f32", dft="tc")
    assert e.value.status == 7
