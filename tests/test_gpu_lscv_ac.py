"""LSCV from the counts' autocorrelation (kde_autocorrelation +
kde_lscv_autocorr) against the FP64 oracle: the autocorrelation itself by
brute force, every pair sum and score on small grids, sampled candidates at
full size, and agreement with the spectrum-dot path."""
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
    import os

    from paper_1508_02766_gb300 import build, kde
    if not os.path.exists(build.LIB):
        build.build()
    return kde


def plan_for(K, w, **opts):
    lam = [np.linalg.eigvalsh(h).max() for h in w.H]
    big = 2.0 * w.H[int(np.argmax(lam))]
    info = K.kde_plan_info_compute(w.M, w.lo, w.hi, big, precision=w.precision, tau=w.tau)
    return K.Plan(w.M, w.lo, w.hi, big, precision=w.precision, tau=w.tau, P_min=info.P, **opts)


def run(K, w, **opts):
    plan = plan_for(K, w, **opts)
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    R = K.kde_autocorrelation(plan, counts)
    S = torch.empty(2 * len(w.H), dtype=torch.float64, device="cuda")
    lscv = K.kde_lscv_autocorr(plan, w.n, w.H, R, pair_sums=S)
    torch.cuda.synchronize()
    return lscv.cpu().numpy(), S.cpu().numpy(), counts.cpu().numpy(), R.cpu().numpy(), plan


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_autocorrelation_by_brute_force(K, prec):
    """R(l) = sum_j c_j c_{j-l} on a 12 x 10 grid at every lag |l_k| <= P_k - M_k
    (the largest support any candidate of the plan may have; larger lags
    wrap around the cyclic grid and are never read)."""
    w = W.lscv_small(4, 2, (12, 10), n=400, count=2, precision=prec)
    _, _, counts, R, plan = run(K, w)
    c = O.counts_to_c(counts)
    P0, P1 = plan.info.P
    M0, M1 = w.M
    A0, A1 = min(P0 - M0, M0 - 1), min(P1 - M1, M1 - 1)
    got, ref = [], []
    for a in range(-A0, A0 + 1):
        for b in range(-A1, A1 + 1):
            s = 0.0
            for j0 in range(max(0, a), min(M0, M0 + a)):
                for j1 in range(max(0, b), min(M1, M1 + b)):
                    s += c[j0, j1] * c[j0 - a, j1 - b]
            ref.append(s)
            got.append(R[a % P0, b % P1])
    got, ref = np.array(got), np.array(ref)
    tol = 1e-12 if prec == "f64" else 2e-6
    assert np.max(np.abs(got - ref)) <= tol * np.abs(ref).max()


@pytest.mark.parametrize("prec,layout", [("f64", "corrected"), ("f32", "corrected"),
                                         ("f64", "wand")])
def test_every_candidate(K, prec, layout):
    """40 candidates (two chunks): every pair sum and score against the oracle."""
    w = W.lscv_small(7, 2, (36, 44), n=3000, count=40, precision=prec)
    lscv, S, counts, _, _ = run(K, w, layout=layout)
    c = O.counts_to_c(counts)
    Sref, ref = [], []
    for H in w.H:
        s = []
        for A in (H, 2 * H):
            L = O.support_L(A, w.lo, w.hi, w.M, w.tau)
            if layout == "wand":
                k = O.kernel_weights(A, w.lo, w.hi, w.M, L, n=1, layout="wand")
                s.append(float(np.sum(c * O.binned_direct(c, k, L))))
            else:
                s.append(O.binned_pair_sum(c, A, w.lo, w.hi, w.M, L))
        Sref.append(s)
        if layout == "corrected":
            ref.append(O.lscv_binned(counts, w.n, H, w.lo, w.hi, w.M, w.tau))
    Sref = np.array(Sref)
    tol = 1e-12 if prec == "f64" else 2e-6
    assert np.max(np.abs(S.reshape(-1, 2) - Sref) / np.abs(Sref)) < tol
    if layout == "corrected":
        ref = np.array(ref)
        scale = np.max(np.abs(Sref[:, 1])) / w.n ** 2
        assert np.max(np.abs(lscv - ref)) < tol * 10 * scale
        assert int(np.argmin(lscv)) == int(np.argmin(ref))


def test_full_size_sampled_candidates_and_spectrum_path(K):
    """512^2, n = 2e6, 1024 candidates: every score against the spectrum-dot
    path, and against the oracle's spectral pair sums the selected
    candidate, four random ones and the two where the paths differ most."""
    w = W.lscv2d_512_f32()
    lscv, S, counts, _, plan = run(K, w)
    assert np.all(np.isfinite(lscv))
    cd = torch.from_numpy(counts).cuda()
    Wsp = K.kde_power_spectrum(plan, cd)
    S2 = torch.empty(2 * len(w.H), dtype=torch.float64, device="cuda")
    K.kde_lscv(plan, w.n, w.H, Wsp, pair_sums=S2)
    S2 = S2.cpu().numpy()
    diff = np.abs(S - S2) / np.abs(S2)
    assert np.max(diff) < 2e-5
    c = O.counts_to_c(counts)
    P = plan.info.P
    rng = np.random.default_rng(3)
    worst = [int(j) // 2 for j in np.argsort(-diff)[:2]]
    for i in [int(np.argmin(lscv))] + list(rng.choice(len(w.H), 4, replace=False)) + worst:
        for h, A in enumerate((w.H[i], 2 * w.H[i])):
            L = O.support_L(A, w.lo, w.hi, w.M, w.tau)
            ref = O.binned_pair_sum_dft(c, A, w.lo, w.hi, w.M, L, P)
            # the FP32 LSCV bound of the spectrum path's tests
            assert abs(S[2 * i + h] - ref) < 2e-5 * abs(ref), (i, h)
            assert abs(S2[2 * i + h] - ref) < 2e-5 * abs(ref), (i, h)


def test_rejects_unsupported(K):
    w = W.lscv_small(9, 2, (30, 30), n=500, count=3, precision="f64")
    plan = K.Plan(w.M, w.lo, w.hi, w.H[0], precision="f64")
    X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
    counts = K.kde_bin(X, w.lo, w.hi, w.M)
    R = K.kde_autocorrelation(plan, counts)
    with pytest.raises(K.KDEError) as e:
        K.kde_lscv_autocorr(plan, w.n, np.stack([w.H[0] * 400.0]), R)
    assert e.value.status == 1
    p1 = K.Plan((300,), (0.0,), (1.0,), np.eye(1) * 1e-3, precision="f64")
    with pytest.raises(K.KDEError) as e:
        K.kde_lscv_autocorr_workspace_bytes(p1)
    assert e.value.status == 7


def test_batch_over_datasets_matches_single_calls(K):
    """kde_lscv_autocorr_batch: three datasets (different n, own candidate
    lists, 600 candidates each so the batch spans two launches) scored in one
    call equal the per-dataset calls bit for bit, and the first set's pair
    sums match the oracle."""
    sets = [W.lscv_small(40 + i, 2, (36, 44), n=n, count=600, precision="f32")
            for i, n in enumerate((900, 2500, 4000))]
    w0 = sets[0]
    lam = [np.linalg.eigvalsh(h).max() for w in sets for h in w.H]
    big = 2.0 * [h for w in sets for h in w.H][int(np.argmax(lam))]
    # one grid for every set (the grid of set 0, widened to hold them all)
    lo = np.min([w.lo for w in sets], axis=0)
    hi = np.max([w.hi for w in sets], axis=0)
    info = K.kde_plan_info_compute(w0.M, lo, hi, big, precision="f32", tau=w0.tau)
    plan = K.Plan(w0.M, lo, hi, big, precision="f32", tau=w0.tau, P_min=info.P)
    P0, P1 = plan.info.P
    R = torch.empty(len(sets), P0, P1, dtype=torch.float32, device="cuda")
    counts = []
    for i, w in enumerate(sets):
        X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
        c = K.kde_bin(X, lo, hi, w.M)
        K.kde_autocorrelation(plan, c, R=R[i])
        counts.append(c.cpu().numpy())
    H = np.stack([w.H for w in sets])
    ns = [w.n for w in sets]
    S = torch.empty(len(sets), 600, 2, dtype=torch.float64, device="cuda")
    got = K.kde_lscv_autocorr_batch(plan, ns, H, R, pair_sums=S).cpu().numpy()
    for i, w in enumerate(sets):
        one = K.kde_lscv_autocorr(plan, w.n, w.H, R[i]).cpu().numpy()
        assert np.array_equal(got[i], one)
    c = O.counts_to_c(counts[0])
    S = S.cpu().numpy()
    for j in (0, 17, 599):
        for h, A in enumerate((w0.H[j], 2 * w0.H[j])):
            L = O.support_L(A, lo, hi, w0.M, w0.tau)
            ref = O.binned_pair_sum(c, A, lo, hi, w0.M, L)
            assert abs(S[0, j, h] - ref) < 2e-6 * abs(ref)


def test_prepared_candidate_set_matches_per_call_scoring(K):
    """kde_lscv_cands_*: 1500 candidates (two chunks) prepared once and
    scored against two datasets' autocorrelations equal kde_lscv_autocorr
    on the same inputs bit for bit, pair sums included."""
    a = W.lscv_small(50, 2, (40, 40), n=1500, count=1500, precision="f32")
    b = W.lscv_small(51, 2, (40, 40), n=3500, count=1, precision="f32")
    lam = [np.linalg.eigvalsh(h).max() for h in a.H]
    big = 2.0 * a.H[int(np.argmax(lam))]
    lo = np.minimum(a.lo, b.lo)
    hi = np.maximum(a.hi, b.hi)
    info = K.kde_plan_info_compute(a.M, lo, hi, big, precision="f32", tau=a.tau)
    plan = K.Plan(a.M, lo, hi, big, precision="f32", tau=a.tau, P_min=info.P)
    cs = K.LscvCands(plan, a.H)
    for w in (a, b):
        X = torch.from_numpy(np.ascontiguousarray(w.X)).cuda()
        R = K.kde_autocorrelation(plan, K.kde_bin(X, lo, hi, w.M))
        S1 = torch.empty(1500, 2, dtype=torch.float64, device="cuda")
        S2 = torch.empty(1500, 2, dtype=torch.float64, device="cuda")
        got = cs.score(w.n, R, pair_sums=S1).cpu().numpy()
        ref = K.kde_lscv_autocorr(plan, w.n, a.H, R, pair_sums=S2).cpu().numpy()
        assert np.array_equal(got, ref)
        assert torch.equal(S1, S2)
