"""Samples read and densities written in place in page-locked host memory
(the in-place end-to-end path): the same kernels on the same values give
bit-identical counts and densities as with device buffers, for both
binning methods, FP32 and FP64, d = 1, 2, 3."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1508_02766_gb300 import kde as K  # noqa: E402
from paper_1508_02766_gb300 import workloads as W  # noqa: E402


@pytest.mark.parametrize("d,M,prec", [(1, (900,), "f64"), (2, (130, 67), "f32"),
                                      (2, (64, 80), "f64"), (3, (20, 17, 24), "f32")])
@pytest.mark.parametrize("method", ["direct", "tiled"])
def test_pinned_host_buffers_match_device_buffers(d, M, prec, method):
    w = W.small_case(300 + d, d, M, n=5000, precision=prec)
    Xh = torch.from_numpy(np.ascontiguousarray(w.X)).pin_memory()
    Xd = Xh.cuda()
    plan = K.Plan(w.M, w.lo, w.hi, w.H, precision=w.precision, tau=w.tau)
    ws = plan.workspace()
    Ks = K.kde_kernel_grid(plan, w.n, workspace=ws)
    c_dev = K.kde_bin(Xd, w.lo, w.hi, w.M, method=method)
    c_host = K.kde_bin(Xh, w.lo, w.hi, w.M, method=method)
    dens_dev = K.kde_fft_eval(plan, c_dev, Ks, workspace=ws)
    dens_host = torch.empty(w.M, dtype=plan.real_dtype()).pin_memory()
    K.kde_fft_eval(plan, c_host, Ks, density=dens_host, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(c_host, c_dev)
    assert np.array_equal(dens_host.numpy(), dens_dev.cpu().numpy())


def test_pageable_host_buffers_are_refused():
    X = torch.zeros(10, 2, dtype=torch.float32)
    with pytest.raises(ValueError):
        K.kde_bin(X, (0, 0), (1, 1), (8, 8))
