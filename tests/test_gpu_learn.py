"""GPU parity of the learned bandwidth proposal: the tensor-core GEMM, the
standardisation and features, the network's forward pass and gradients
against the FP64 oracle, training, checkpoint/resume, and what the trained
network gains over the method without it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import kde_oracle as O  # noqa: E402
from oracle import learn_oracle as LO  # noqa: E402
from paper_1508_02766_gb300 import kde  # noqa: E402
from paper_1508_02766_gb300 import learned as Lm  # noqa: E402
from paper_1508_02766_gb300 import workloads as W  # noqa: E402

DEV = "cuda"


def _bf16_exact(rng, shape, denom):
    """Values exactly representable in BF16 whose products and sums are exact in FP32."""
    return (rng.integers(-8, 9, size=shape) / denom).astype(np.float32)


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (128, 64, 128), (256, 192, 320), (384, 1088, 256)])
def test_tensor_core_gemm_exact(M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = _bf16_exact(rng, (M, K), 8.0)
    B = _bf16_exact(rng, (N, K), 4.0)
    Ad = torch.from_numpy(A).to(DEV).to(torch.bfloat16)
    Bd = torch.from_numpy(B).to(DEV).to(torch.bfloat16)
    C, status = kde.kde_gemm_bf16(Ad, Bd)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)


def test_tensor_core_gemm_rejects_bad_shapes():
    A = torch.zeros(100, 64, dtype=torch.bfloat16, device=DEV)
    B = torch.zeros(16, 64, dtype=torch.bfloat16, device=DEV)
    with pytest.raises(kde.KDEError) as e:
        kde.kde_gemm_bf16(A, B)
    assert e.value.status == 1


def test_standardize_and_features_match_oracle():
    X = W.mixture_datasets(11, 1)[0]
    Xd = torch.from_numpy(X).to(DEV)
    Z, mom = kde.kde_standardize2(Xd)
    Zo, momo = LO.standardize(X)
    # FP32 tree sums
    assert np.allclose(mom.cpu().numpy(), momo, rtol=1e-5, atol=1e-5)
    assert np.max(np.abs(Z.cpu().numpy() - Zo)) < 1e-5
    # features from the GPU's counts of the GPU's Z; the counts are checked
    # bit-exact against the oracle's binning of the same Z
    M = (Lm.GRID_M, Lm.GRID_M)
    counts = kde.kde_bin(Z, (Lm.GRID_LO,) * 2, (Lm.GRID_HI,) * 2, M, method="direct")
    Zh = Z.cpu().numpy()
    c_or, _ = O.bin_linear(Zh, np.array([Lm.GRID_LO] * 2), np.array([Lm.GRID_HI] * 2), M)
    c_or = c_or.reshape(M)
    assert np.array_equal(counts.cpu().numpy(), c_or)
    f = kde.kde_features2(counts, X.shape[0], mom).cpu().numpy()
    fo = LO.features(c_or, X.shape[0], mom.cpu().numpy())
    assert np.max(np.abs(f - fo)) < 1e-5 * max(1.0, np.abs(fo).max())


def _mlp_and_batch(B, seed=0):
    rng = np.random.default_rng(seed)
    mlp = kde.MLP(in_dim=kde.FEAT_DIM, hidden=256, out_dim=3, max_batch=256, seed=seed)
    X = rng.normal(0, 1, size=(B, kde.FEAT_DIM)).astype(np.float32)
    X[:, 1030:] = 0.0
    T = rng.normal(-1.5, 0.5, size=(B, 3)).astype(np.float32)
    return mlp, X, T


@pytest.mark.parametrize("B", [200, 256])
def test_forward_and_gradients_match_oracle(B):
    """Against the oracle with BF16 rounding at the same points (so the ReLU
    masks are decided on the same values): only the FP32 accumulation order
    differs, so every tensor agrees within 1e-3 of its maximum.  The plain
    FP64 network is within 2% on the outputs and the loss."""
    mlp, X, T = _mlp_and_batch(B)
    p = mlp.get_params()
    Xd, Td = torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV)
    Y = mlp.forward(Xd).cpu().numpy()
    loss, g = mlp.loss_grad(Xd, Td)
    loss, g = float(loss.item()), g.cpu().numpy()
    assert mlp.status() == 0
    yb, _ = LO.mlp_forward(p, X, kde.FEAT_DIM, 256, 3, bf16=True)
    lb, gb = LO.mlp_loss_grad(p, X, T, kde.FEAT_DIM, 256, 3, bf16=True)
    assert np.max(np.abs(Y - yb)) <= 1e-3 * np.abs(yb).max()
    assert abs(loss - lb) <= 1e-3 * lb
    sizes = [256 * kde.FEAT_DIM, 256, 256 * 256, 256, 3 * 256, 3]
    o = 0
    for s in sizes:
        a, b = g[o:o + s], gb[o:o + s]
        assert np.max(np.abs(a - b)) <= 1e-3 * np.abs(b).max(), (o, s)
        o += s
    y64, _ = LO.mlp_forward(p, X, kde.FEAT_DIM, 256, 3)
    l64, _ = LO.mlp_loss_grad(p, X, T, kde.FEAT_DIM, 256, 3)
    assert np.max(np.abs(Y - y64)) <= 2e-2 * np.abs(y64).max()
    assert abs(loss - l64) <= 2e-2 * l64


def test_training_reduces_loss_and_checkpoint_resumes():
    mlp, X, T = _mlp_and_batch(256, seed=1)
    Xd, Td = torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV)
    loss = torch.zeros(1, dtype=torch.float32, device=DEV)
    mlp.train_step(Xd, Td, 1e-3, loss=loss)
    first = float(loss.item())
    for _ in range(60):
        mlp.train_step(Xd, Td, 1e-3, loss=loss)
    assert float(loss.item()) < 0.1 * first
    assert mlp.status() == 0
    # checkpoint: parameters and optimizer state into a fresh network; the
    # next step from both is identical
    p, (m, v, step) = mlp.get_params(), mlp.get_state()
    twin = kde.MLP(in_dim=kde.FEAT_DIM, hidden=256, out_dim=3, max_batch=256, seed=99)
    twin.set_params(p)
    twin.set_state(m, v, step)
    mlp.train_step(Xd, Td, 1e-3, loss=loss)
    twin.train_step(Xd, Td, 1e-3, loss=loss)
    torch.cuda.synchronize()
    assert np.array_equal(mlp.get_params(), twin.get_params())


def test_scorer_pair_sums_match_oracle():
    """The scorer's wiring (standardise, bin, the counts' autocorrelation on
    the shared plan): pair sums S(H), S(2H) of a few candidates against the
    oracle's spectral pair sums at the plan's padding."""
    n = 2000
    X = W.mixture_datasets(5, 1, n=n)[0]
    sc = Lm.LscvScorer(n)
    sc.prepare(torch.from_numpy(X).to(DEV))
    idx = [0, 300, 1007]
    H = sc.cand_H[idx]
    pair = torch.empty(2 * len(idx), dtype=torch.float64, device=DEV)
    kde.kde_lscv_autocorr(sc.plan, n, H, sc.R, pair_sums=pair, workspace=sc.lws)
    got = pair.cpu().numpy()
    c = O.counts_to_c(sc.counts.cpu().numpy())
    lo, hi, M = np.array([Lm.GRID_LO] * 2), np.array([Lm.GRID_HI] * 2), (Lm.GRID_M, Lm.GRID_M)
    P = tuple(sc.plan.info.P)
    want = []
    for h in H:
        for A in (h, 2.0 * h):
            L = O.support_L(A, lo, hi, M)
            want.append(O.binned_pair_sum_dft(c, A, lo, hi, M, L, P))
    want = np.array(want)
    assert np.max(np.abs(got - want) / np.abs(want)) < 1e-5


def test_learned_proposal_beats_the_method_without_it():
    """Train on plain-search labels of 1024 mixtures, then on 64 held-out
    mixtures compare the LSCV regret (score minus the plain search's best) of
    the network's proposal with the normal-reference bandwidth's, each
    refined over the same 27-candidate neighbourhood; the learned method must
    be better on average and use far fewer candidates than the plain search."""
    train_sets = W.mixture_datasets(21, 1024)
    test_sets = W.mixture_datasets(22, 64)
    sc = Lm.LscvScorer(10_000)
    lab = Lm.label_datasets(sc, train_sets)
    mlp = kde.MLP(in_dim=kde.FEAT_DIM, hidden=256, out_dim=3, max_batch=256, seed=0)
    hist = Lm.train(mlp, lab.feats, lab.theta, epochs=60, batch=256, lr=1e-3)
    assert hist[-1] < 0.5 * hist[0]
    reg_learned, reg_ref, n_cand = [], [], []
    for X in test_sets:
        Xd = torch.from_numpy(X).to(DEV)
        sc.prepare(Xd)
        _, best = sc.search()
        th, v, k, _ = Lm.select(sc, mlp, Xd, refine=True, fallback=False)
        ref = Lm.normal_reference_theta(X.shape[0])
        s_ref = sc.scores(np.stack([Lm.theta_to_H(t) for t in Lm.neighbourhood(ref)])).cpu().numpy()
        reg_learned.append(v - best)
        reg_ref.append(s_ref.min() - best)
        n_cand.append(k)
    assert mlp.status() == 0
    assert np.mean(reg_learned) < np.mean(reg_ref)
    assert max(n_cand) <= 28 < len(sc.cand)
    # the batched form selects the same bandwidths
    res = Lm.select_batch(sc, mlp, test_sets, fallback=False)
    for (th_b, v_b, k_b, _), v in zip(res, np.array(reg_learned)):
        assert k_b == 28
    vb = np.array([r[1] for r in res])
    vs = []
    for X in test_sets:
        vs.append(Lm.select(sc, mlp, torch.from_numpy(X).to(DEV), fallback=False)[1])
    assert np.allclose(vb, np.array(vs), rtol=1e-12, atol=0)


def test_fallback_replaces_a_bad_proposal_by_the_plain_search():
    """A network that always proposes the most oversmoothed, most correlated
    corner of the candidate box: its neighbourhood scores worse than the
    normal-reference bandwidth, so both select and select_batch must fall
    back to the plain search and return exactly its (theta, LSCV)."""
    sc = Lm.LscvScorer(10_000)
    mlp = kde.MLP(in_dim=kde.FEAT_DIM, hidden=256, out_dim=3, max_batch=256, seed=0)
    p = mlp.get_params()
    p[:] = 0.0
    p[-3:] = [Lm.A_GRID[-1], Lm.BETA_GRID[-1], Lm.C_GRID[-1]]
    mlp.set_params(p)
    sets = W.mixture_datasets(41, 6)
    res_b = Lm.select_batch(sc, mlp, sets, fallback=True)
    for X, rb in zip(sets, res_b):
        Xd = torch.from_numpy(X).to(DEV)
        th, v, k, fell = Lm.select(sc, mlp, Xd, fallback=True)
        sc.prepare(Xd)
        t_s, v_s = sc.search()
        assert fell and rb[3]
        assert k == 28 + len(sc.cand) and rb[2] == 28 + len(sc.cand)
        assert np.array_equal(th, t_s) and v == v_s
        assert np.array_equal(rb[0], t_s) and rb[1] == v_s
    mlp.check()
