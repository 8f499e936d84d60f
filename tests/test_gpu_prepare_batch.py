"""GPU checks of the batched preparation (kde_prepare2_batch) and the batched
plain search (kde_lscv_autocorr_cands_batch): each dataset of a batch gets
what the per-dataset calls give it (counts, moments and features bit for
bit, autocorrelations to FP32 rounding, candidate scores bit for bit on the
same autocorrelation), and the batched labels equal the one-by-one labels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import kde_oracle as O  # noqa: E402
from paper_1508_02766_gb300 import kde  # noqa: E402
from paper_1508_02766_gb300 import learned as Lm  # noqa: E402
from paper_1508_02766_gb300 import workloads as W  # noqa: E402

DEV = "cuda"


@pytest.fixture(scope="module")
def scorer():
    return Lm.LscvScorer(20_000)


def _ragged_sets(seed, count):
    """Mixture datasets of ragged sizes (a few samples up to 20 000), some
    with samples beyond the standardised grid."""
    rng = np.random.default_rng(seed)
    out = []
    for i, X in enumerate(W.mixture_datasets(seed, count, n=20_000)):
        n = int(rng.choice([2, 3, 37, 1000, 4099, 20_000])) if i else 20_000
        X = X[:n].copy()
        if i % 3 == 2 and n > 10:
            X[0] = [40.0, -40.0]     # far outside: dropped by binning, counted in n
        out.append(X)
    return out


def test_prepare_batch_matches_per_dataset(scorer):
    sets = _ragged_sets(71, 9)
    Xc, off = scorer.concat(sets)
    F, Rs, ns = scorer.prepare_batch(Xc, off)
    torch.cuda.synchronize()
    counts_b = scorer.bprep.counts[:len(sets)].clone()
    mom_b = scorer.bprep.moments[:len(sets)].clone()
    info = scorer.plan.info
    for i, X in enumerate(sets):
        assert ns[i] == X.shape[0]
        f1 = torch.empty(kde.FEAT_DIM, dtype=torch.float32, device=DEV)
        R1 = torch.empty(info.P[0], info.P[1], dtype=torch.float32, device=DEV)
        scorer.prepare(torch.from_numpy(X).to(DEV), feat=f1, R=R1)
        torch.cuda.synchronize()
        assert torch.equal(scorer.counts, counts_b[i]), i
        assert torch.equal(scorer.mom, mom_b[i]), i
        assert torch.equal(f1, F[i]), i
        r1, rb = R1.cpu().numpy(), Rs[i].cpu().numpy()
        assert np.max(np.abs(r1 - rb)) <= 1e-6 * np.max(np.abs(r1)), i


def test_prepare_batch_counts_match_oracle_binning(scorer):
    sets = _ragged_sets(72, 4)
    Xc, off = scorer.concat(sets)
    scorer.prepare_batch(Xc, off)
    torch.cuda.synchronize()
    lo, hi = np.array([Lm.GRID_LO] * 2), np.array([Lm.GRID_HI] * 2)
    M = (Lm.GRID_M, Lm.GRID_M)
    for i, X in enumerate(sets):
        # the GPU's own standardised samples, binned by the oracle
        f = torch.empty(kde.FEAT_DIM, dtype=torch.float32, device=DEV)
        scorer.prepare(torch.from_numpy(X).to(DEV), feat=f)
        Z = scorer.prep.Z[:X.shape[0]].cpu().numpy()
        c_or, _ = O.bin_linear(Z, lo, hi, M)
        assert np.array_equal(scorer.bprep.counts[i].cpu().numpy(), c_or), i


def test_batched_search_equals_per_dataset(scorer):
    sets = _ragged_sets(73, 6)
    Xc, off = scorer.concat(sets)
    F, Rs, ns = scorer.prepare_batch(Xc, off)
    s_b = scorer.cand_set.score_batch(ns, Rs)
    pairs_b = torch.empty(len(sets), 2 * scorer.cand_set.nH, dtype=torch.float64, device=DEV)
    scorer.cand_set.score_batch(ns, Rs, pair_sums=pairs_b)
    for i in range(len(sets)):
        p1 = torch.empty(2 * scorer.cand_set.nH, dtype=torch.float64, device=DEV)
        s1 = scorer.cand_set.score(int(ns[i]), Rs[i], pair_sums=p1, workspace=scorer.lws)
        assert torch.equal(s1, s_b[i]), i
        assert torch.equal(p1, pairs_b[i]), i
    th, v = scorer.search_batch(Rs, ns)
    for i in range(len(sets)):
        t1, v1 = scorer.search(R=Rs[i], n=int(ns[i]))
        assert np.array_equal(t1, th[i]) and v1 == v[i], i


def test_batched_labels_equal_one_by_one(scorer):
    sets = W.mixture_datasets(74, 5)
    lab = Lm.label_datasets(scorer, sets, batch=2)
    for i, X in enumerate(sets):
        f = scorer.prepare(torch.from_numpy(X).to(DEV))
        t, v = scorer.search()
        assert np.array_equal(lab.feats[i], f.cpu().numpy()), i
        assert np.array_equal(lab.theta[i], t), i
        assert abs(lab.best[i] - v) <= 1e-9 * abs(v), i


def test_prepare_batch_rejects_bad_offsets(scorer):
    X = torch.zeros(10, 2, dtype=torch.float32, device=DEV)
    for off in ([0, 5, 6, 10], [1, 5, 10], [0, 8, 7]):
        with pytest.raises(kde.KDEError):
            scorer.prepare_batch(X, off)


def _box():
    lo = np.array([Lm.A_GRID[0], Lm.BETA_GRID[0], Lm.C_GRID[0]]) - 0.5 * Lm.STEP
    hi = np.array([Lm.A_GRID[-1], Lm.BETA_GRID[-1], Lm.C_GRID[-1]]) + 0.5 * Lm.STEP
    return lo, hi


def test_device_candidates_match_host_candidates(scorer):
    """kde_lscv_theta_select builds each candidate's H on the device; its
    scores match kde_lscv_autocorr_batch on the same bandwidths built on the
    host (FP32 lag sums from FP64 parameters that can differ in the last
    bit), and it picks the same candidate wherever the two best differ by
    more than that."""
    sets = _ragged_sets(75, 7)
    Xc, off = scorer.concat(sets)
    F, Rs, ns = scorer.prepare_batch(Xc, off)
    rng = np.random.default_rng(5)
    lo, hi = _box()
    TH = rng.uniform(lo - 0.3, hi + 0.3, size=(len(sets), 3)).astype(np.float32)   # some clipped
    offs = 0.5 * Lm.NEIGHBOUR_OFFSETS * Lm.STEP
    refs = Lm.normal_reference_thetas(ns)
    lscv = torch.empty(len(sets), len(offs) + 1, dtype=torch.float64, device=DEV)
    out = kde.kde_lscv_theta_select(scorer.plan, ns, torch.from_numpy(TH).to(DEV), lo, hi, offs,
                                    refs, Rs, lscv=lscv)
    base = np.clip(TH.astype(np.float64), lo, hi)
    th_all = np.concatenate([base[:, None, :] + offs, refs[:, None, :]], axis=1)
    ref = kde.kde_lscv_autocorr_batch(scorer.plan, [int(v) for v in ns], Lm.thetas_to_H(th_all),
                                      Rs, workspace=scorer.lws).cpu().numpy()
    got, o = lscv.cpu().numpy(), out.cpu().numpy()
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-6
    for i in range(len(sets)):
        order = np.argsort(ref[i, :-1])
        j = int(o[i, 0])
        assert o[i, 1] == got[i, j] and o[i, 2] == got[i, -1]
        assert np.array_equal(o[i, 3:6], th_all[i, j])
        if ref[i, order[1]] - ref[i, order[0]] > 1e-6 * abs(ref[i, order[0]]):
            assert j == order[0], i


def test_device_candidates_that_do_not_fit_score_inf(scorer):
    sets = _ragged_sets(76, 2)
    Xc, off = scorer.concat(sets)
    F, Rs, ns = scorer.prepare_batch(Xc, off)
    lo, hi = _box()
    TH = torch.zeros(2, 3, dtype=torch.float32, device=DEV)
    offs = np.array([[6.0, 0.0, 6.0], [0.0, 0.0, 0.0]])      # e^6: far wider than the padding
    refs = np.array([[6.0, 0.0, 6.0], [-1.5, 0.0, -1.5]])
    lscv = torch.empty(2, 3, dtype=torch.float64, device=DEV)
    o = kde.kde_lscv_theta_select(scorer.plan, ns, TH, lo, hi, offs, refs, Rs, lscv=lscv)
    v, o = lscv.cpu().numpy(), o.cpu().numpy()
    assert np.isinf(v[:, 0]).all() and np.isfinite(v[:, 1]).all()
    assert np.isinf(v[0, 2]) and np.isfinite(v[1, 2])
    assert (o[:, 0] == 1).all()
    # every offset unfit: no candidate index
    o2 = kde.kde_lscv_theta_select(scorer.plan, ns, TH, lo, hi, offs[:1], refs, Rs).cpu().numpy()
    assert (o2[:, 0] == 1).all() and np.isinf(o2[:, 1]).all()


def test_select_batch_device_and_host_candidates_agree(scorer):
    sets = W.mixture_datasets(77, 12)
    mlp = kde.MLP(in_dim=kde.FEAT_DIM, hidden=256, out_dim=3, max_batch=256, seed=3)
    lab = Lm.label_datasets(scorer, W.mixture_datasets(78, 256))
    Lm.train(mlp, lab.feats, lab.theta, epochs=4, batch=64)
    a = Lm.select_batch(scorer, mlp, sets, device_candidates=True)
    b = Lm.select_batch(scorer, mlp, sets, device_candidates=False)
    for (ta, va, ka, fa), (tb, vb, kb, fb) in zip(a, b):
        assert fa == fb and ka == kb
        assert abs(va - vb) <= 1e-6 * abs(vb)
        assert np.allclose(ta, tb, atol=1e-12) or abs(va - vb) <= 1e-6 * abs(vb)


def test_submitted_batches_collect_like_select_batch(scorer):
    """Two batches enqueued before either is read back give what
    select_batch gives each (the autocorrelations of the first stay valid
    after the second is prepared)."""
    mlp = kde.MLP(in_dim=kde.FEAT_DIM, hidden=256, out_dim=3, max_batch=256, seed=4)
    lab = Lm.label_datasets(scorer, W.mixture_datasets(79, 128))
    Lm.train(mlp, lab.feats, lab.theta, epochs=3, batch=64)
    a_sets, b_sets = W.mixture_datasets(80, 9), W.mixture_datasets(81, 7)
    ref_a = Lm.select_batch(scorer, mlp, a_sets, as_arrays=True)
    ref_b = Lm.select_batch(scorer, mlp, b_sets, as_arrays=True)
    ja = Lm.select_submit(scorer, mlp, *scorer.concat(a_sets))
    jb = Lm.select_submit(scorer, mlp, *scorer.concat(b_sets))
    got_a = Lm.select_collect(scorer, ja, as_arrays=True)
    got_b = Lm.select_collect(scorer, jb, as_arrays=True)
    for got, ref in ((got_a, ref_a), (got_b, ref_b)):
        for g, r in zip(got, ref):
            assert np.array_equal(g, r)
    # fallback of a batch collected after another was prepared: every
    # proposal made worse than the reference by an untrained network
    bad = kde.MLP(in_dim=kde.FEAT_DIM, hidden=256, out_dim=3, max_batch=256, seed=5)
    jc = Lm.select_submit(scorer, bad, *scorer.concat(a_sets))
    Lm.select_submit(scorer, bad, *scorer.concat(b_sets))
    th, v, c, fb = Lm.select_collect(scorer, jc, as_arrays=True)
    ref_c = Lm.select_batch(scorer, bad, a_sets, as_arrays=True)
    for g, r in zip((th, v, c, fb), ref_c):
        assert np.array_equal(g, r)
