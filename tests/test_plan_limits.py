"""Padded lengths at the limits of the plan (host only, no GPU).

Eq. 10 evaluates the binned estimate without wrap-around whenever every
axis has P_k >= M_k + L_k, with L_k from Eq. 15.  The plan must give every
requirement up to the largest supported length (KDE_MAX_P = 4096) such a
P_k, never above that length, and must refuse a requirement above it with
KDE_ERR_UNSUPPORTED instead of planning a shorter, aliased transform.
"""
import numpy as np
import pytest

from oracle import kde_oracle as O
from paper_1508_02766_gb300 import kde

MAX_P = 4096
TINY = 1e-12   # H so small that L_k = 1 on every axis of these grids


def _plan(M, precision, **opts):
    d = len(M)
    return kde.kde_plan_info_compute(M, [0.0] * d, [1.0] * d, np.eye(d) * TINY,
                                     precision=precision, **opts)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_every_requirement_up_to_the_limit_is_planned(precision):
    engines = set()
    for need in range(3, MAX_P + 1):
        M = (need - 1, 50)
        info = _plan(M, precision)
        assert info.L == O.support_L(np.eye(2) * TINY, [0, 0], [1, 1], M) == (1, 1)
        assert need <= info.P[0] <= MAX_P, (need, info.P)
        assert info.P[1] >= 51
        engines.add(info.engine)
    # FP32 2-D plans use the two-phase engine where it has a split, else Stockham
    assert engines == ({"two_phase", "stockham"} if precision == "f32" else {"stockham"})


def test_one_dimensional_lengths_up_to_the_limit():
    for need in list(range(3, 200)) + list(range(3900, MAX_P + 1)):
        info = _plan((need - 1,), "f64")
        assert need <= info.P[0] <= MAX_P, (need, info.P)


@pytest.mark.parametrize("d,precision", [(1, "f64"), (2, "f32"), (2, "f64"), (3, "f32")])
def test_requirements_above_the_limit_are_refused(d, precision):
    for need in range(MAX_P + 1, MAX_P + 40):
        M = (need - 1,) + (8,) * (d - 1)
        with pytest.raises(kde.KDEError, match="UNSUPPORTED"):
            _plan(M, precision)
    # the same through a requested minimum padded length
    with pytest.raises(kde.KDEError, match="UNSUPPORTED"):
        _plan((20,) * d, precision, P_min=[MAX_P + 1] + [0] * (d - 1))
    # and exactly at the limit it is accepted
    info = _plan((20,) * d, precision, P_min=[MAX_P] + [0] * (d - 1))
    assert info.P[0] == MAX_P


def test_last_axis_at_the_limit_sets_the_half_spectrum():
    info = _plan((20, 30), "f32", P_min=[0, MAX_P])
    assert info.P[1] == MAX_P and info.Q == MAX_P // 2 + 1
