"""CPU-side checks of the CUDA library: it loads, exports every symbol its
header declares, and its host planning (Eq. 4, Eq. 15, padded sizes, H
checks) agrees with the oracle.  No compute call needs a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import kde_oracle as O
from paper_1508_02766_gb300 import build as B
from paper_1508_02766_gb300 import kde
from paper_1508_02766_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    if not os.path.exists(B.LIB):
        B.build()
    return B.LIB


def header_functions():
    text = open(os.path.join(ROOT, "include", "kde_gb300.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(kde_\w+)\s*\(", text, re.M)))


def test_header_symbols_exported():
    names = header_functions()
    assert "kde_bin" in names and "kde_fft_eval" in names and "kde_kernel_grid" in names
    L = ctypes.CDLL(B.LIB)
    for n in names:
        assert hasattr(L, n), n
    assert set(kde.EXPORTS) <= set(names)


def _is_7smooth(x):
    for p in (2, 3, 5, 7):
        while x % p == 0:
            x //= p
    return x == 1


def _compiled(macro):
    text = open(os.path.join(ROOT, "paper_1508_02766_gb300", "csrc", "fx_pairs.h")).read()
    body = text[text.index("#define " + macro):]
    body = body[:body.index("\n\n")]
    return [tuple(int(v) for v in m.split(",")) for m in re.findall(r"X\(([\d,\s]+)\)", body)]


def _two_phase_plan(need):
    """The two-phase planner's rule: up to 400, the smallest P >= need with a
    split into 7-smooth factors <= 20 (most balanced), unless a compiled
    pair is at most 10% longer; above that, the smallest compiled
    three-factor length."""
    comp = sorted((a * b, (a, b)) for a, b in _compiled("KDE_FX_PAIRS") if a * b >= need)
    for P in range(need, 401):
        splits = [(a, P // a) for a in range(2, int(P ** 0.5) + 1)
                  if P % a == 0 and P // a <= 20 and _is_7smooth(a) and _is_7smooth(P // a)]
        if not splits:
            continue
        if comp and comp[0][0] <= 1.1 * P:
            break
        return P, splits[-1]
    if comp:
        return comp[0]
    tri = sorted((a * b * c, (a, b, c)) for a, b, c in _compiled("KDE_FX_TRIPLES") if a * b * c >= need)
    return tri[0] if tri else (None, None)


def test_compiled_splits_cover_the_lengths():
    pairs = _compiled("KDE_FX_PAIRS")
    tri = _compiled("KDE_FX_TRIPLES")
    assert all(a * b <= 400 and _is_7smooth(a * b) for a, b in pairs)
    lens = sorted(a * b * c for a, b, c in tri)
    assert lens[0] > 400 and lens[0] <= 1.12 * 400
    assert all(b <= 1.125 * a for a, b in zip(lens, lens[1:]))   # spaced by at most 12.5%


@pytest.mark.parametrize("name", ["kde2d_128_f64", "kde2d_1024_f32"])
@pytest.mark.parametrize("range_mode", ["corrected", "per_axis"])
@pytest.mark.parametrize("engine", ["auto", "stockham"])
def test_plan_matches_oracle_support(name, range_mode, engine):
    w = W.WORKLOADS[name](n=2000)
    info = kde.kde_plan_info_compute(w.M, w.lo, w.hi, w.H, precision=w.precision,
                                     range_mode=range_mode, engine=engine)
    assert info.L == O.support_L(w.H, w.lo, w.hi, w.M, range_mode=range_mode)
    assert np.allclose(info.delta, O.binwidths(w.lo, w.hi, w.M), rtol=0, atol=0)
    assert abs(info.lambda_max - np.linalg.eigvalsh(w.H).max()) < 1e-14
    two = engine == "auto" and w.precision == "f32"
    assert info.engine == ("two_phase" if two else "stockham")
    for k in range(w.d):
        need = w.M[k] + info.L[k]
        assert info.P[k] >= need
        assert _is_7smooth(info.P[k])
        if two:
            assert (info.P[k], info.split[k]) == _two_phase_plan(need)
        else:
            assert info.split[k] == (0, 0)
            assert all(not _is_7smooth(p) for p in range(need, info.P[k]))
        assert int(np.prod(info.radices[k])) == info.P[k]
    assert info.Q == info.P[-1] // 2 + 1


def test_plan_two_phase_engine_limits():
    # forced two-phase needs FP32 and d >= 2, and lines of at most 40 x 40
    with pytest.raises(kde.KDEError) as e:
        kde.kde_plan_info_compute((64, 64), (0, 0), (1, 1), np.eye(2) * 1e-3, precision="f64",
                                  engine="two_phase")
    assert e.value.status == 7
    with pytest.raises(kde.KDEError) as e:
        kde.kde_plan_info_compute((2000, 64), (0, 0), (1, 1), np.eye(2) * 1e-3, engine="two_phase")
    assert e.value.status == 7
    # auto falls back to the Stockham engine there
    info = kde.kde_plan_info_compute((2000, 64), (0, 0), (1, 1), np.eye(2) * 1e-3)
    assert info.engine == "stockham" and info.split == ((0, 0), (0, 0))
    info = kde.kde_plan_info_compute((256, 256, 256), (0,) * 3, (1,) * 3, np.eye(3) * 1e-3)
    assert info.engine == "two_phase"
    for k in range(3):
        assert info.split[k][0] * info.split[k][1] == info.P[k]


def test_plan_3d_eigenvalue_and_support():
    rng = np.random.default_rng(0)
    for _ in range(20):
        H = W.random_spd(rng, 3, 1.0, 50.0, scale=0.05)
        lo, hi, M = [0, 0, 0], [3.0, 2.0, 4.0], [64, 48, 80]
        info = kde.kde_plan_info_compute(M, lo, hi, H)
        assert abs(info.lambda_max - np.linalg.eigvalsh(H).max()) < 1e-13 * np.abs(H).max()
        assert abs(info.det_H - np.linalg.det(H)) < 1e-12 * abs(np.linalg.det(H))
        assert info.L == O.support_L(H, lo, hi, M)


def test_plan_workload_sizes():
    """The padded sizes of the benchmark workloads (>= M + L)."""
    w = W.kde2d_128_f64()
    assert kde.kde_plan_info_compute(w.M, w.lo, w.hi, w.H, precision="f64").P == (144, 144)
    w = W.kde2d_1024_f32(n=100_000)
    info = kde.kde_plan_info_compute(w.M, w.lo, w.hi, w.H)
    assert info.P == (1080, 1080) and info.split == ((9, 10, 12), (9, 10, 12))
    info = kde.kde_plan_info_compute(w.M, w.lo, w.hi, w.H, engine="stockham")
    assert info.P == (1080, 1080) and info.engine == "stockham"


def test_plan_rejects_bad_input():
    ok = dict(M=(8, 8), lo=(0, 0), hi=(1, 1))
    with pytest.raises(kde.KDEError) as e:
        kde.kde_plan_info_compute(H=[[1.0, 0.5], [0.4, 1.0]], **ok)
    assert e.value.status == 1
    with pytest.raises(kde.KDEError) as e:
        kde.kde_plan_info_compute(H=[[1.0, 2.0], [2.0, 1.0]], **ok)
    assert e.value.status == 2
    with pytest.raises(kde.KDEError) as e:
        kde.kde_plan_info_compute(M=(1, 8), lo=(0, 0), hi=(1, 1), H=np.eye(2))
    assert e.value.status == 1
    with pytest.raises(kde.KDEError) as e:
        kde.kde_plan_info_compute(M=(8, 8), lo=(0, 1), hi=(1, 1), H=np.eye(2))
    assert e.value.status == 1
    with pytest.raises(kde.KDEError) as e:
        kde.kde_plan_info_compute(M=(8, 8, 8, 8), lo=(0,) * 4, hi=(1,) * 4, H=np.eye(4))
    assert e.value.status == 7
    with pytest.raises(kde.KDEError) as e:
        kde.kde_plan_info_compute(M=(5000,), lo=(0,), hi=(1,), H=np.eye(1) * 1e-4)
    assert e.value.status == 7
    with pytest.raises(kde.KDEError) as e:
        kde.kde_plan_info_compute(H=[[np.nan, 0], [0, 1.0]], **ok)
    assert e.value.status == 1


def test_plan_respects_P_min_and_modes():
    info = kde.kde_plan_info_compute((100, 60), (0, 0), (1, 1), [[0.01, 0.0], [0.0, 0.02]],
                                     P_min=(256, 0), precision="f64")
    assert info.P[0] == 256 and info.precision == "f64"
    assert info.workspace_bytes > 0 and info.kspec_bytes == info.kspec_elems * 8


def test_bin_workspace_sizes():
    for d, M, n in [(1, (5000,), 10), (2, (1024, 1024), 10**6), (3, (256, 256, 256), 10**7)]:
        b = kde.kde_bin_workspace_bytes(n, d, M)
        # a 16-byte record per tile a sample touches (at most 2^d), plus tables
        assert b >= (16 << d) * n
        assert b < (16 << d) * n + (8 << 20)


def test_batch_preparation_and_search_reject_bad_handles():
    """Host checks of the batched calls run before any device work: a NULL
    plan or candidate set, or too many datasets, is refused."""
    L = kde.lib()
    b = ctypes.c_size_t(7)
    assert L.kde_prepare2_batch_workspace_bytes(None, 4, 100, ctypes.byref(b)) == 1
    assert L.kde_lscv_autocorr_cands_batch_workspace_bytes(None, 4, ctypes.byref(b)) == 1
    off = (ctypes.c_int64 * 2)(0, 10)
    null = ctypes.c_void_p(0)
    assert L.kde_prepare2_batch(None, 1, null, off, null, null, null, null, null, 0, null) == 1
    n = (ctypes.c_int64 * 1)(10)
    assert L.kde_lscv_autocorr_cands_batch(None, 1, n, null, null, null, null, 0, null) == 1
    d6 = (ctypes.c_double * 6)()
    assert L.kde_lscv_theta_select(None, 1, n, null, d6, 1, d6, d6, null, null, null, null, 0,
                                   null) == 1
    assert L.kde_lscv_theta_select_workspace_bytes(None, 1, 1, ctypes.byref(b)) == 1


def _slab_fits(M1, Q, sr, sc):
    """The slab passes' block shape (8 blocks per slab, RP row pairs and W
    half-spectrum columns each) and its limit: 113 KB of shared memory."""
    RP = -(-((M1 + 1) // 2) // 8)
    W_ = -(-Q // 8)
    SKr = sr[1] | 1
    SKc = W_ * sc[1]
    while SKc % 16 != W_ % 16:
        SKc += 1
    ex = max(RP * sr[0] * SKr, sc[0] * SKc)
    smem = 16 + max(ex + M1 * W_, ex + 2 * RP * Q) * 8
    return smem <= 113 * 1024


@pytest.mark.parametrize("M,opts,expect", [
    ((256, 256, 256), {}, True),
    ((20, 17, 24), {}, True),
    ((2, 2, 2), {}, True),
    ((256, 256, 256), {"slab": "off"}, False),
    ((40, 50, 60), {"slab": None}, False),   # the default: separate passes
    ((256, 256, 256), {"dft": "tc"}, False),
    ((256, 256, 256), {"engine": "stockham"}, False),
    ((40, 50, 60), {"precision": "f64"}, False),
    ((64, 320, 300), {"tau": 1.0}, True),   # P = 320 or so: more tasks than threads
    ((4, 400, 390), {"tau": 0.5}, False),  # exchange and cluster buffer above 113 KB
    ((4, 500, 40), {}, False),           # axis 1 longer than 400: three factors
])
def test_slab_pass_eligibility(M, opts, expect):
    H = np.diag([0.002, 0.002, 0.002]) if M[1] >= 256 else np.diag([0.01, 0.02, 0.015])
    o = {"precision": "f32", "slab": "on", **opts}
    if o["slab"] is None:
        del o["slab"]
    info = kde.kde_plan_info_compute(M, (0, 0, 0), (1, 1, 1), H, **o)
    assert info.slab_passes == expect
    if info.engine == "two_phase" and len(info.split[1]) == 2 and len(info.split[2]) == 2 \
            and not set(opts) - {"tau"}:
        assert _slab_fits(M[1], info.Q, info.split[2], info.split[1]) == expect
    two_d = kde.kde_plan_info_compute((64, 64), (0, 0), (1, 1), np.diag([0.01, 0.01]))
    assert not two_d.slab_passes
    with pytest.raises(kde.KDEError):
        bad = kde.Opts()
        bad.slab_passes = 7
        kde._check(kde.lib().kde_plan_info_compute(
            3, kde._iarr(M), kde._darr((0, 0, 0)), kde._darr((1, 1, 1)), kde._darr(H),
            ctypes.byref(bad), ctypes.byref(kde.PlanInfo())))
