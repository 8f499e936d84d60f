"""Binning added to existing counts (kde_bin_accumulate) and evaluation that
leaves the counts zeroed (kde_fft_eval_consume), through the C ABI.

The binned counts of Eq. 7 are a sum over samples (Sec. 2), so samples
binned in parts and added must give the oracle's counts of all of them bit
for bit, with the samples outside the grid counted once each.  The
consuming evaluation must give kde_fft_eval's density bit for bit and leave
every count at zero, and a stream of steps on one counts array (accumulate,
consume, accumulate, ...) must reproduce the step-by-step kde_bin +
kde_fft_eval results.
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


CASES = [(1, (700,), "f32"), (2, (37, 53), "f32"), (2, (130, 67), "f64"),
         (3, (20, 17, 24), "f32"), (3, (9, 13, 11), "f64")]


def with_outside(w, seed):
    """The case's samples with a few moved outside the grid (counted, not binned)."""
    rng = np.random.default_rng(seed)
    X = np.array(w.X, copy=True)
    idx = rng.choice(X.shape[0], size=17, replace=False)
    X[idx, 0] = w.hi[0] + 1.0
    return X


@pytest.mark.parametrize("method", ["direct", "tiled"])
@pytest.mark.parametrize("d,M,prec", CASES)
def test_bin_in_parts_equals_oracle(K, method, d, M, prec):
    w = W.small_case(31 + d, d, M, n=3000, precision=prec)
    Xh = with_outside(w, 5)
    X = torch.from_numpy(np.ascontiguousarray(Xh)).cuda()
    nout = torch.full((1,), 999, dtype=torch.int64, device="cuda")
    counts = K.kde_bin(X[:1100], w.lo, w.hi, w.M, n_outside=nout, method=method)
    K.kde_bin(X[1100:2300], w.lo, w.hi, w.M, counts=counts, n_outside=nout, method=method,
              accumulate=True)
    K.kde_bin(X[2300:2300], w.lo, w.hi, w.M, counts=counts, n_outside=nout, method=method,
              accumulate=True)   # no samples: nothing changes
    K.kde_bin(X[2300:], w.lo, w.hi, w.M, counts=counts, n_outside=nout, method=method,
              accumulate=True)
    torch.cuda.synchronize()
    ref, ref_out = O.bin_linear(Xh, w.lo, w.hi, w.M)
    assert np.array_equal(counts.cpu().numpy(), ref)
    assert int(nout.item()) == ref_out == 17


@pytest.mark.parametrize("d,M,prec", CASES)
def test_consume_gives_the_same_density_and_zero_counts(K, d, M, prec):
    w = W.small_case(41 + d, d, M, n=2500, precision=prec)
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    plan = K.Plan(w.M, w.lo, w.hi, w.H, precision=w.precision, tau=w.tau)
    ws = plan.workspace()
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    Ks = K.kde_kernel_grid(plan, w.n, workspace=ws)
    ref = K.kde_fft_eval(plan, counts, Ks, workspace=ws).cpu().numpy()
    got = K.kde_fft_eval(plan, counts, Ks, workspace=ws, consume=True)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), ref)
    assert int(torch.count_nonzero(counts).item()) == 0


@pytest.mark.parametrize("d,M,prec", [(2, (96, 80), "f32"), (3, (20, 17, 24), "f32"),
                                      (2, (37, 53), "f64")])
def test_stream_of_steps_on_one_counts_array(K, d, M, prec):
    """Three datasets through PreparedPath(counts_kept_zero=True) on one counts
    array: each density equals that dataset's own kde_bin + kde_fft_eval."""
    sets = [W.small_case(51 + i, d, M, n=1500 + 400 * i, precision=prec) for i in range(3)]
    w0 = sets[0]
    plan = K.Plan(w0.M, w0.lo, w0.hi, w0.H, precision=w0.precision, tau=w0.tau)
    ws = plan.workspace()
    counts = torch.zeros(plan.M, dtype=torch.int64, device="cuda")
    Ks = torch.empty(plan.info.kspec_elems, dtype=plan.real_dtype(), device="cuda")
    dens = torch.empty(plan.M, dtype=plan.real_dtype(), device="cuda")
    for w in sets:
        X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
        path = K.PreparedPath(plan, X, counts, Ks, dens, ws, n=w.n, counts_kept_zero=True)
        path()
        torch.cuda.synchronize()
        got = dens.cpu().numpy()
        assert int(torch.count_nonzero(counts).item()) == 0
        c_ref = K.kde_bin(X, plan.lo, plan.hi, plan.M)
        K_ref = K.kde_kernel_grid(plan, w.n, workspace=ws)
        ref = K.kde_fft_eval(plan, c_ref, K_ref, workspace=ws).cpu().numpy()
        assert np.array_equal(got, ref)
