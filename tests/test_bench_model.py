"""Byte model of the bench's roofline figures (host only): the step total
counts every kernel that ran once per launch and nothing that did not run."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _info(name):
    from paper_1508_02766_gb300 import kde
    from paper_1508_02766_gb300 import workloads as W
    w = W.WORKLOADS[name]()
    return w, kde.kde_plan_info_compute(w.M, w.lo, w.hi, w.H, precision=w.precision, tau=w.tau)


def _by_hand_2d(info, n):
    """The per-pass bytes of a 2-D FP32 evaluation written out (one read of
    what a pass consumes, one write of what it produces)."""
    M0, M1 = info.M
    P0 = info.P[0]
    Q = info.Q
    L0 = info.L[0]
    return ((n * 2 * 4 + 8 * M0 * M1)                       # binning
            + (2 * L0 + 1) * Q * 8                           # kernel rows
            + (2 * L0 + 1) * Q * 8 + P0 * Q * 4              # kernel spectrum
            + 8 * M0 * M1 + M0 * Q * 8                       # counts rows
            + 2 * M0 * Q * 8 + P0 * Q * 4                    # middle axis
            + M0 * Q * 8 + M0 * M1 * 4)                      # output rows


def test_step_bytes_2d_counts_each_pass_once():
    w, info = _info("kde2d_1024_f32")
    alg = bench.algorithmic_bytes(info, w.n, 4)
    steps = 20
    names = ["kde_bin_kernel", "kde_rows_r2c_kgen_kernel", "kde_cols_kgen_real_kernel",
             "kde_rows_r2c_counts_kernel", "kde_cols_mid_kernel", "kde_rows_c2r_kernel"]
    prof = {k: (1.0, steps) for k in names}
    total, missing = bench.step_bytes(alg, prof, steps)
    assert missing == []
    assert total == pytest.approx(_by_hand_2d(info, w.n), rel=1e-12)
    # the two-phase kernels of the same passes give the same total
    prof2 = {k.replace("kde_", "kde_fx_", 1) if k != "kde_bin_kernel" else k: v
             for k, v in prof.items()}
    assert bench.step_bytes(alg, prof2, steps)[0] == pytest.approx(total, rel=1e-12)
    # with the tensor-core first pass, it replaces the counts rows: same total
    prof3 = dict(prof)
    prof3["kde_rows_r2c_tc_kernel"] = prof3.pop("kde_rows_r2c_counts_kernel")
    assert bench.step_bytes(alg, prof3, steps)[0] == pytest.approx(total, rel=1e-12)
    # about 52 MB per 1024^2 step
    assert 50e6 < total < 55e6


def test_step_bytes_reports_unmodelled_kernels():
    w, info = _info("kde2d_128_f64")
    alg = bench.algorithmic_bytes(info, w.n, 8)
    total, missing = bench.step_bytes(alg, {"kde_bin_kernel": (1.0, 2), "mystery": (1.0, 2)}, 2)
    assert missing == ["mystery"]
    assert total == pytest.approx(w.n * 2 * 8 + 8 * int(np.prod(w.M)))


@pytest.mark.parametrize("name", ["kde2d_1024_f32", "kde3d_256_f32"])
def test_tiled_binning_counts_the_same_bytes_as_direct(name):
    """The tiled binning's three kernels together count the samples read once
    and the counts written once, like the direct kernel; zeroing counts
    nothing."""
    w, info = _info(name)
    alg = bench.algorithmic_bytes(info, w.n, 4)
    steps = 5
    direct, _ = bench.step_bytes(alg, {"kde_bin_kernel": (1.0, steps),
                                       "kde_zero_counts_kernel": (1.0, steps)}, steps)
    tiled, missing = bench.step_bytes(
        alg, {k: (1.0, steps) for k in ("kde_bin_count_kernel", "kde_bin_scatter_kernel",
                                        "kde_bin_accum_kernel")}, steps)
    assert missing == []
    assert tiled == direct == w.n * info.d * 4 + 8 * int(np.prod(w.M))
