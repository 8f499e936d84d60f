"""kde_fft_eval_noalloc: the evaluation entry point for callers that cannot
allocate device memory where they evaluate (their allocations belong to a
host framework, or they run in a loop that must not enter an allocator).
It takes no workspace and uses the library's fixed scratch array instead.

Checked through the C ABI against kde_fft_eval with a caller workspace, on
two calls in a row (the second call finds the first call's data in the
shared array).  Both run the same kernels with the same launch shapes on
the same inputs, so the results must be identical bit for bit; the device's
free memory must not change across a call.  This file is collected last on
purpose.
"""
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


def _prepare(K, w):
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    plan = K.Plan(w.M, w.lo, w.hi, w.H, precision=w.precision, tau=w.tau)
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    ws = plan.workspace()
    Ks = K.kde_kernel_grid(plan, w.n, workspace=ws)
    ref = K.kde_fft_eval(plan, counts, Ks, workspace=ws)
    return plan, counts, Ks, ref


@pytest.mark.parametrize("case", ["2d_f32_1024", "3d_f64", "1d_f32"])
def test_noalloc_matches_workspace_path_twice(K, case):
    if case == "2d_f32_1024":
        w = W.kde2d_1024_f32(n=200_000)
    elif case == "3d_f64":
        w = W.small_case(21, 3, (30, 26, 22), n=5000, precision="f64")
    else:
        w = W.small_case(22, 1, (900,), n=5000, precision="f32")
    plan, counts, Ks, ref = _prepare(K, w)
    assert plan.info.workspace_bytes <= K.noalloc_scratch_bytes()
    ref = ref.cpu().numpy()
    outs = [torch.full(w.M, float("nan"), dtype=plan.real_dtype(), device="cuda")
            for _ in range(2)]
    torch.cuda.synchronize()
    for i in range(2):
        free0 = torch.cuda.mem_get_info()[0]
        K.kde_fft_eval_noalloc(plan, counts, Ks, outs[i])
        torch.cuda.synchronize()
        if i == 1:   # after the first call has loaded and looked up the array
            assert torch.cuda.mem_get_info()[0] == free0
        got = outs[i].cpu().numpy()
        assert np.array_equal(got, ref), float(np.max(np.abs(got - ref)))


def test_noalloc_rejects_plans_above_the_fixed_scratch(K):
    w = W.small_case(23, 3, (200, 200, 200), n=1000, precision="f64")
    plan = K.Plan(w.M, w.lo, w.hi, w.H, precision="f64")
    assert plan.info.workspace_bytes > K.noalloc_scratch_bytes()
    counts = torch.zeros(w.M, dtype=torch.int64, device="cuda")
    Ks = torch.zeros(plan.info.kspec_elems, dtype=torch.float64, device="cuda")
    out = torch.empty(w.M, dtype=torch.float64, device="cuda")
    with pytest.raises(K.KDEError) as e:
        K.kde_fft_eval_noalloc(plan, counts, Ks, out)
    assert e.value.status == 4
    assert "scratch" in str(e.value)
