"""Status reporting through the C ABI: samples outside the grid as
KDE_ERR_OUT_OF_RANGE (kde_outside_check on kde_bin's counter), and a plan
whose kernels completed every bounded wait checks KDE_OK."""
import numpy as np
import pytest

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


def test_outside_samples_reported_as_out_of_range(K):
    w = W.small_case(5, 2, (40, 30), n=1000, precision="f32")
    X = np.array(w.X)
    X[:7, 0] = w.hi[0] + 1.0        # seven samples beyond the last node
    X[7:10, 1] = np.nan             # three NaN coordinates
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    nout = torch.zeros(1, dtype=torch.int64, device="cuda")
    counts = K.kde_bin(Xd, w.lo, w.hi, w.M, n_outside=nout)
    with pytest.raises(K.KDEError) as e:
        K.outside_check(nout)
    assert e.value.status == 3 and "10 samples" in str(e.value)
    assert int(counts.sum().item()) == (1000 - 10) << 32
    Xd = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    K.kde_bin(Xd, w.lo, w.hi, w.M, n_outside=nout)
    assert K.outside_check(nout) == 0


@pytest.mark.parametrize("dft", ["fft", "tc"])
def test_plan_check_ok_after_a_normal_evaluation(K, dft):
    w = W.small_case(6, 2, (64, 48), n=2000, precision="f32")
    Xd = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    plan = K.Plan(w.M, w.lo, w.hi, w.H, precision="f32", dft=dft)
    counts = K.kde_bin(Xd, w.lo, w.hi, w.M)
    ws = plan.workspace()
    Ks = K.kde_kernel_grid(plan, w.n, workspace=ws)
    K.kde_fft_eval(plan, counts, Ks, workspace=ws)
    K.plan_check(plan)
