"""Learned bandwidth proposal on top of the binned FFT LSCV search.

Orchestration only: every numerical step (standardisation, binning, features,
the counts' autocorrelation, LSCV of every candidate, the network's forward and backward
passes, Adam) runs in the CUDA library through ``kde``; this module picks
which calls to make, holds the candidate grid and keeps the buffers.

Coordinates: each dataset is standardised per axis (Z = (X - mean) / sd) and
binned on one fixed grid of the standardised plane, so every dataset shares
one plan, one padding and one candidate set.  A bandwidth is proposed in
those coordinates as log-Cholesky parameters theta = (a, beta, c),
H_z = R R^T with R = [[e^a, 0], [beta e^c, e^c]]; in the data's coordinates
it is H = D H_z D with D = diag(sd).  The plain method is the batched LSCV
search over the whole candidate grid; the learned method scores the network's
proposal and a small neighbourhood of it with the same FFT-evaluated LSCV and
falls back to the plain search when the best of those is worse than the
normal-reference bandwidth's score.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

from . import kde

GRID_M = 256
GRID_LO, GRID_HI = -6.0, 6.0
A_GRID = np.linspace(-2.8, -0.6, 12)      # log of the first Cholesky diagonal
BETA_GRID = np.linspace(-1.2, 1.2, 7)     # off-diagonal over the second diagonal
C_GRID = np.linspace(-2.8, -0.6, 12)      # log of the second Cholesky diagonal
STEP = np.array([A_GRID[1] - A_GRID[0], BETA_GRID[1] - BETA_GRID[0], C_GRID[1] - C_GRID[0]])


def thetas_to_H(T):
    """H = R R^T for every theta = (a, beta, c) along the last axis of T
    (shape ... x 3 -> ... x 2 x 2), R = [[e^a, 0], [beta e^c, e^c]]."""
    T = np.asarray(T, dtype=np.float64)
    ea, ec = np.exp(T[..., 0]), np.exp(T[..., 2])
    b = T[..., 1] * ec
    H = np.empty(T.shape[:-1] + (2, 2))
    H[..., 0, 0] = ea * ea
    H[..., 0, 1] = ea * b
    H[..., 1, 0] = ea * b
    H[..., 1, 1] = b * b + ec * ec
    return H


def theta_to_H(theta):
    return thetas_to_H(np.asarray(theta, dtype=np.float64)[None, :])[0]


def candidate_thetas():
    """The plain search's candidates: every (a, beta, c) of the grids."""
    return np.array(list(itertools.product(A_GRID, BETA_GRID, C_GRID)), dtype=np.float64)


def normal_reference_theta(n):
    """Textbook normal-reference rule in standardised coordinates:
    H = (4/(d+2))^(2/(d+4)) n^(-2/(d+4)) S with S the identity (d = 2)."""
    h2 = (4.0 / 4.0) ** (2.0 / 6.0) * n ** (-2.0 / 6.0)
    return np.array([0.5 * math.log(h2), 0.0, 0.5 * math.log(h2)])


def normal_reference_thetas(ns):
    """normal_reference_theta for every sample count in ns (B x 3)."""
    h = 0.5 * np.log((4.0 / 4.0) ** (2.0 / 6.0) * np.asarray(ns, dtype=np.float64) ** (-2.0 / 6.0))
    return np.stack([h, np.zeros_like(h), h], axis=1)


NEIGHBOUR_OFFSETS = np.array(list(itertools.product((-1, 0, 1), repeat=3)), dtype=np.float64)


def neighbourhood(theta, scale=0.5):
    """3 x 3 x 3 candidates around theta, spaced scale grid steps apart
    (theta: 3, or B x 3 for B neighbourhoods at once)."""
    theta = np.asarray(theta, dtype=np.float64)
    return theta[..., None, :] + scale * NEIGHBOUR_OFFSETS * STEP


class LscvScorer:
    """One shared plan for the standardised grid and the buffers of one
    dataset at a time: standardise, bin, features, the counts'
    autocorrelation, then the LSCV of any list of candidates."""

    def __init__(self, n_max, device="cuda", tau=3.7):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        cand = candidate_thetas()
        # padding sized by the widest 2 H over the candidate box (and its edges)
        big = max((2.0 * theta_to_H(t) for t in itertools.product(
            (A_GRID[-1] + STEP[0],), (BETA_GRID[0] - STEP[1], BETA_GRID[-1] + STEP[1]),
            (C_GRID[-1] + STEP[2],))), key=lambda h: np.linalg.eigvalsh(h).max())
        M = (GRID_M, GRID_M)
        lo, hi = (GRID_LO, GRID_LO), (GRID_HI, GRID_HI)
        pinfo = kde.kde_plan_info_compute(M, lo, hi, big, precision="f32", tau=tau)
        self.plan = kde.Plan(M, lo, hi, big, precision="f32", tau=tau, P_min=pinfo.P)
        self.M, self.lo, self.hi, self.tau = M, lo, hi, tau
        info = self.plan.info
        self.feat = torch.empty(kde.FEAT_DIM, dtype=torch.float32, device=self.device)
        self.R = torch.empty(info.P[0], info.P[1], dtype=torch.float32, device=self.device)
        self.lws = torch.empty(kde.kde_lscv_autocorr_workspace_bytes(self.plan), dtype=torch.uint8,
                               device=self.device)
        # standardise, bin, features, autocorrelation with arguments marshalled once
        self.prep = kde.FeaturePrep(self.plan, n_max, self.lws)
        self.counts, self.Z, self.mom = self.prep.counts, self.prep.Z, self.prep.moments
        self.n = 0
        self.cand = cand
        self.cand_H = thetas_to_H(cand)
        # the plain search scores the same candidates on every dataset
        self.cand_set = kde.LscvCands(self.plan, self.cand_H)
        self.bprep = None   # batched preparation, sized on first use
        self.bws = None     # workspace of the batched plain search
        self.tws = None     # workspace of the device-built candidates
        self.th_buf = None    # the network's proposals of a submitted batch

    def prepare(self, X, feat=None, R=None):
        """X: n x 2 float32 CUDA tensor of one dataset.  Features go to feat
        and the autocorrelation to R (the scorer's own buffers by default)."""
        feat = self.feat if feat is None else feat
        R = self.R if R is None else R
        self.prep.run(X, feat, R)
        self.n = int(X.shape[0])
        return feat

    def scores(self, H):
        """LSCV of every H (k x 2 x 2, standardised coordinates), on the GPU."""
        torch = self.torch
        out = torch.empty(len(H), dtype=torch.float64, device=self.device)
        kde.kde_lscv_autocorr(self.plan, self.n, np.asarray(H, dtype=np.float64), self.R,
                              lscv=out, workspace=self.lws)
        return out

    def search(self, R=None, n=None):
        """The plain method: argmin of LSCV over the whole candidate grid (of
        the last prepared dataset, or of autocorrelation R with n samples)."""
        s = self.cand_set.score(self.n if n is None else n, self.R if R is None else R,
                                workspace=self.lws)
        i = int(self.torch.argmin(s).item())
        return self.cand[i], float(s[i].item())

    def moments(self):
        return self.mom.cpu().numpy()

    def concat(self, datasets):
        """One (n_total, 2) float32 CUDA tensor and the host row offsets of
        a list of datasets (numpy arrays or CUDA tensors), in one upload."""
        torch = self.torch
        ns = [int(X.shape[0]) for X in datasets]
        off = np.zeros(len(ns) + 1, dtype=np.int64)
        off[1:] = np.cumsum(ns)
        if datasets and torch.is_tensor(datasets[0]):
            Xc = torch.cat([X.to(self.device, torch.float32) for X in datasets]).contiguous()
        else:
            Xc = torch.from_numpy(np.ascontiguousarray(
                np.concatenate(datasets).astype(np.float32, copy=False))).to(self.device)
        return Xc, off

    def prepare_batch(self, X, offsets, F=None, Rs=None):
        """The preparation of many datasets in one call (kde_prepare2_batch):
        X the concatenated samples (CUDA), offsets their host row offsets.
        Returns features (B x FEAT_DIM), autocorrelations (B x P_0 x P_1) and
        the sample counts (numpy)."""
        torch = self.torch
        off = np.asarray(offsets, dtype=np.int64)
        B, total = len(off) - 1, int(off[-1])
        if self.bprep is None or B > self.bprep.nsets_max or total > self.bprep.n_total_max:
            nb = max(B, self.bprep.nsets_max if self.bprep else 0)
            nt = max(total, self.bprep.n_total_max if self.bprep else 0)
            self.bprep = kde.BatchPrep(self.plan, nb, nt, device=self.device)
        info = self.plan.info
        if F is None:
            F = torch.empty(B, kde.FEAT_DIM, dtype=torch.float32, device=self.device)
        if Rs is None:
            Rs = torch.empty(B, info.P[0], info.P[1], dtype=torch.float32, device=self.device)
        self.bprep.run(X, off, F, Rs)
        return F, Rs, np.diff(off)

    def search_batch(self, Rs, ns):
        """The plain method on many datasets: every candidate scored against
        every autocorrelation in one call, argmin per dataset on the device.
        Returns (thetas B x 3, LSCV minima B)."""
        torch = self.torch
        B = len(ns)
        need = self.cand_set.batch_workspace_bytes(B)
        if self.bws is None or self.bws.numel() < need:
            self.bws = torch.empty(max(256, need), dtype=torch.uint8, device=self.device)
        s = self.cand_set.score_batch(ns, Rs, workspace=self.bws)
        v, i = torch.min(s, dim=1)
        i = i.cpu().numpy()
        return self.cand[i], v.cpu().numpy()


@dataclass
class LabelledSet:
    feats: np.ndarray      # D x FEAT_DIM float32
    theta: np.ndarray      # D x 3 (LSCV argmin)
    best: np.ndarray       # D (its LSCV)
    n: np.ndarray          # D


def label_datasets(scorer, datasets, batch=256):
    """Features and plain-search labels for every dataset, batch datasets
    per call: one upload, one batched preparation, one batched search."""
    D = len(datasets)
    feats = np.empty((D, kde.FEAT_DIM), dtype=np.float32)
    theta = np.empty((D, 3))
    best = np.empty(D)
    ns = np.empty(D, dtype=np.int64)
    for b0 in range(0, D, batch):
        part = datasets[b0:b0 + batch]
        Xc, off = scorer.concat(part)
        F, Rs, n = scorer.prepare_batch(Xc, off)
        th, v = scorer.search_batch(Rs, n)
        b1 = b0 + len(part)
        theta[b0:b1], best[b0:b1], ns[b0:b1] = th, v, n
        feats[b0:b1] = F.cpu().numpy()
    return LabelledSet(feats, theta, best, ns)


def train(mlp, feats, theta, epochs=30, batch=256, lr=1e-3, seed=0, device="cuda"):
    """Adam on mean squared error between network output and labels; the
    whole set stays on the device; returns the per-epoch mean loss."""
    import torch
    F = torch.from_numpy(np.ascontiguousarray(feats, dtype=np.float32)).to(device)
    T = torch.from_numpy(np.ascontiguousarray(theta, dtype=np.float32)).to(device)
    rng = np.random.default_rng(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=device)
    hist = []
    D = F.shape[0]
    for _ in range(epochs):
        perm = torch.from_numpy(rng.permutation(D)).to(device)
        acc, nb = 0.0, 0
        for s in range(0, D - batch + 1, batch):
            idx = perm[s:s + batch]
            mlp.train_step(F[idx].contiguous(), T[idx].contiguous(), lr, loss=loss)
            acc += float(loss.item())
            nb += 1
        hist.append(acc / max(1, nb))
    mlp.check()
    return hist


def select(scorer, mlp, X, refine=True, fallback=True, scored=None):
    """The learned method on one dataset: score the network's proposal (and
    its 3 x 3 x 3 neighbourhood), compare with the normal-reference score and
    fall back to the plain search when the proposal is worse.  Returns
    (theta, lscv, candidates scored, fell back); appends the scored H
    matrices to ``scored`` if given."""
    torch = scorer.torch
    f = scorer.prepare(X)
    th = mlp.forward(f.view(1, -1)).cpu().numpy()[0].astype(np.float64)
    mlp.check()
    # keep the neighbourhood inside the box the plan's padding was sized for
    lo = np.array([A_GRID[0], BETA_GRID[0], C_GRID[0]]) - 0.5 * STEP
    hi = np.array([A_GRID[-1], BETA_GRID[-1], C_GRID[-1]]) + 0.5 * STEP
    th = np.clip(th, lo, hi)
    cands = neighbourhood(th) if refine else th[None, :]
    ref = normal_reference_theta(X.shape[0])
    H = np.stack([theta_to_H(t) for t in cands] + [theta_to_H(ref)])
    s = scorer.scores(H).cpu().numpy()
    if scored is not None:
        scored.extend(H)
    i = int(np.argmin(s[:-1]))
    if fallback and s[i] > s[-1]:
        t, v = scorer.search()
        if scored is not None:
            scored.extend(scorer.cand_H)
        return t, v, len(H) + len(scorer.cand), True
    return cands[i], float(s[i]), len(H), False


def select_batch(scorer, mlp, datasets, fallback=True, scored=None, offsets=None,
                 device_candidates=True, as_arrays=False):
    """The learned method on many datasets at once: features and
    autocorrelations of every dataset in one batched preparation call, one
    network forward pass for the batch (at most mlp.max_batch rows per
    pass), then the 27-candidate neighbourhoods and normal-reference scores
    of every dataset enqueued before one host synchronisation; datasets
    whose proposal is worse than the normal-reference score fall back to the
    plain search.  datasets: a list of datasets, or, with offsets (host row
    offsets), their samples already concatenated in one CUDA tensor.  With
    device_candidates the candidates are built and scored on the device
    from the network's output (kde_lscv_theta_select); otherwise they are
    built on the host and scored by kde_lscv_autocorr_batch.
    Returns a list of (theta, lscv, candidates scored, fell back), or with
    as_arrays (device candidates only) the four as arrays over the batch."""
    torch = scorer.torch
    dev = scorer.device
    if offsets is None:
        Xc, off = scorer.concat(datasets)
    else:
        Xc, off = datasets, np.asarray(offsets, dtype=np.int64)
    B = len(off) - 1
    F, Rs, ns = scorer.prepare_batch(Xc, off)
    ns = [int(v) for v in ns]
    TH = torch.empty(B, 3, dtype=torch.float32, device=dev)
    for s0 in range(0, B, mlp.max_batch):
        mlp.forward(F[s0:s0 + mlp.max_batch], Y=TH[s0:s0 + mlp.max_batch])
    lo = np.array([A_GRID[0], BETA_GRID[0], C_GRID[0]]) - 0.5 * STEP
    hi = np.array([A_GRID[-1], BETA_GRID[-1], C_GRID[-1]]) + 0.5 * STEP
    if device_candidates:
        job = _submit(scorer, mlp, F, Rs, ns, TH, lo, hi)
        return select_collect(scorer, job, fallback=fallback, scored=scored, as_arrays=as_arrays)
    mlp.check()
    TH = TH.cpu().numpy().astype(np.float64)
    # every dataset's 27 neighbours and its normal-reference bandwidth, at once
    cands = neighbourhood(np.clip(TH, lo, hi))                        # B x 27 x 3
    refs = normal_reference_thetas(ns)                                # B x 3
    Hs = thetas_to_H(np.concatenate([cands, refs[:, None, :]], axis=1))  # B x 28 x 2 x 2
    out = kde.kde_lscv_autocorr_batch(scorer.plan, ns, Hs, Rs, workspace=scorer.lws)
    if scored is not None:
        scored.extend(Hs.reshape(-1, 2, 2))
    s_all = out.cpu().numpy()
    res = []
    for i in range(B):
        s = s_all[i]
        j = int(np.argmin(s[:-1]))
        if fallback and s[j] > s[-1]:
            t, v = scorer.search(R=Rs[i], n=ns[i])
            if scored is not None:
                scored.extend(scorer.cand_H)
            res.append((t, v, 28 + len(scorer.cand), True))
        else:
            res.append((cands[i][j], float(s[j]), 28, False))
    return res


@dataclass
class SelectionJob:
    """A learned selection enqueued on the device (select_submit): its
    packed results and the network's status are read by select_collect."""
    out: object          # B x 6 FP64 (pinned host, filled in stream order): best index,
                         # its LSCV, reference LSCV, theta
    flag: object         # the network's status word (pinned host int32)
    done: object         # event recorded after both copies
    ns: list
    refs: np.ndarray     # B x 3 reference thetas
    Rs: object           # the autocorrelations (valid until the next preparation)
    offs: np.ndarray     # J x 3 neighbourhood offsets


def _submit(scorer, mlp, F, Rs, ns, TH, lo, hi):
    torch = scorer.torch
    B = len(ns)
    offs = 0.5 * NEIGHBOUR_OFFSETS * STEP
    refs = normal_reference_thetas(ns)
    need = kde.lscv_theta_select_workspace_bytes(scorer.plan, B, len(offs))
    if scorer.tws is None or scorer.tws.numel() < need:
        scorer.tws = torch.empty(max(256, need), dtype=torch.uint8, device=scorer.device)
    out = kde.kde_lscv_theta_select(scorer.plan, ns, TH, lo, hi, offs, refs, Rs,
                                    workspace=scorer.tws)
    # results and the network's status go to pinned host memory in stream
    # order; collecting waits for this batch's event only, not for batches
    # enqueued after it
    out_h = torch.empty(B, 6, dtype=torch.float64, pin_memory=True)
    out_h.copy_(out, non_blocking=True)
    flag_h = torch.empty(1, dtype=torch.int32, pin_memory=True)
    mlp.status_copy(flag_h)
    done = torch.cuda.Event()
    done.record()
    return SelectionJob(out_h, flag_h, done, ns, refs, Rs, offs)


def select_submit(scorer, mlp, Xc, offsets):
    """Enqueues the learned selection of a batch (samples concatenated in the
    CUDA tensor Xc, host row offsets): batched preparation, the network,
    candidates built and scored on the device.  Nothing is synchronised, so
    the next batch can be enqueued before this one is collected; buffers
    are reused in stream order."""
    torch = scorer.torch
    off = np.asarray(offsets, dtype=np.int64)
    B = len(off) - 1
    F, Rs, ns = scorer.prepare_batch(Xc, off)
    ns = [int(v) for v in ns]
    if scorer.th_buf is None or scorer.th_buf.shape[0] < B:
        scorer.th_buf = torch.empty(max(B, 256), 3, dtype=torch.float32, device=scorer.device)
    TH = scorer.th_buf[:B]
    for s0 in range(0, B, mlp.max_batch):
        mlp.forward(F[s0:s0 + mlp.max_batch], Y=TH[s0:s0 + mlp.max_batch])
    lo = np.array([A_GRID[0], BETA_GRID[0], C_GRID[0]]) - 0.5 * STEP
    hi = np.array([A_GRID[-1], BETA_GRID[-1], C_GRID[-1]]) + 0.5 * STEP
    return _submit(scorer, mlp, F, Rs, ns, TH, lo, hi)


def select_collect(scorer, job, fallback=True, scored=None, as_arrays=False, fetch=None):
    """Reads a submitted selection (one copy back) and runs the plain search
    for the datasets whose proposal scores worse than the normal reference.
    fetch(i), when given, returns dataset i's samples for that search (needed
    once a later batch has been prepared, which reuses the autocorrelation
    buffer); otherwise the job's autocorrelations are used."""
    job.done.synchronize()
    o = job.out.numpy()
    if int(job.flag[0]):
        raise kde.KDEError(6, "a tensor-core wait of the network gave up; results are invalid")
    B, J, offs = len(job.ns), len(job.offs), job.offs
    if scored is not None:
        base = o[:, 3:6] - offs[np.minimum(o[:, 0].astype(np.int64), J - 1)]
        scored.extend(thetas_to_H(np.concatenate(
            [base[:, None, :] + offs, job.refs[:, None, :]], axis=1)).reshape(-1, 2, 2))
    # results as arrays; only the datasets that fall back are visited
    theta, best = o[:, 3:6].copy(), o[:, 1].copy()
    ncand = np.full(B, 28, dtype=np.int64)
    fell = (o[:, 0] >= J) | ((o[:, 1] > o[:, 2]) if fallback else False)
    for i in np.nonzero(fell)[0]:
        if fetch is None:
            theta[i], best[i] = scorer.search(R=job.Rs[i], n=job.ns[i])
        else:
            scorer.prepare(fetch(int(i)))
            theta[i], best[i] = scorer.search()
        ncand[i] += len(scorer.cand)
        if scored is not None:
            scored.extend(scorer.cand_H)
    if as_arrays:
        return theta, best, ncand, fell
    return [(theta[i], float(best[i]), int(ncand[i]), bool(fell[i])) for i in range(B)]
