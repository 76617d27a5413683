"""Learned sparse path on the GPU: proposal kernels against the proposal oracle (bit-exact sets,
features), the MLP inference and gradient kernels against the FP64 network oracle, the
restricted recursions against the FP64 oracle when the sets hold every donor, and the sparse
distances against the dense path when they do not.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import proposal as op
from paper_2212_11403_gb300 import synth

pytestmark = pytest.mark.gpu

D_TOL = 1e-5


@pytest.fixture(scope="module")
def ls():
    import torch
    torch.cuda.set_device(0)
    from paper_2212_11403_gb300 import ls as _ls
    return _ls


def d_err(dg, dr):
    """per-entry error of distances: max over entries of |d_gpu - d_ref| / max(|d_ref|, 1)."""
    dg = np.asarray(dg, dtype=np.float64)
    dr = np.asarray(dr, dtype=np.float64)
    return float(np.max(np.abs(dg - dr) / np.maximum(np.abs(dr), 1.0)))


def full_sets(N, Wn):
    import torch
    idx = np.zeros((N, Wn, N - 1), dtype=np.int32)
    for i in range(N):
        idx[i, :, :] = [j for j in range(N) if j != i]
    return torch.from_numpy(idx).cuda()


@pytest.mark.parametrize("WS", [256, 37])
def test_full_sets_reproduce_the_oracle(ls, WS):
    """every donor in every window: the restricted chain is the full one (Eq. fwd1/bck1)."""
    import torch
    w = synth.make_workload("ls_n200_l1000")
    N, L, loci = w["N"], w["L"], w["loci"]
    Wn = (L + WS - 1) // WS
    idx = full_sets(N, Wn)
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        d = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
        rc, pac, nf = ls.ls_sparse_run_all(ctx, idx, N - 1, WS, loci, d, lost_tol=0.0)
        torch.cuda.synchronize()
        d = d.cpu().numpy()
    finally:
        ls.ls_destroy(ctx)
    assert rc == 0 and nf == 0
    ref = oracle.run(w["h"], w["rho"], w["mu"], loci, want=("post", "llf"))
    for k in range(len(loci)):
        dref = oracle.distance_block(ref["post"][:, k, :], np.arange(N))
        assert d_err(d[k], dref) <= D_TOL, (loci[k], d_err(d[k], dref))
    assert abs(pac - ref["llf"].sum()) <= 1e-6 * abs(ref["llf"].sum()) + 2e-7 * L * math.sqrt(N)


def test_raw_proposal_and_features_match_oracle(ls):
    import torch
    w = synth.make_workload("ls_n50000_l20000", N=150, L=1500, seed=21)
    N, L = w["N"], w["L"]
    Wn = op.windows(L)
    K, C = 20, 40
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        idx = torch.empty((N, Wn, K), dtype=torch.int32, device="cuda")
        ls.ls_propose(ctx, C, K, None, idx)
        cand = torch.empty((N, C), dtype=torch.int32, device="cuda")
        feat = torch.empty((N, C, 8), dtype=torch.float32, device="cuda")
        wsel = [0, 2, Wn - 1]
        got = []
        for wi in wsel:
            ls.ls_propose_window(ctx, C, wi, cand, feat)
            got.append((cand.cpu().numpy(), feat.cpu().numpy()))
        idx = idx.cpu().numpy()
    finally:
        ls.ls_destroy(ctx)
    for wi in range(Wn):
        rc, _ = op.stage1(w["h"], wi, K)
        np.testing.assert_array_equal(idx[:, wi, :], rc)
    for (gc, gf), wi in zip(got, wsel):
        rc, rf = op.stage1(w["h"], wi, C)
        np.testing.assert_array_equal(gc, rc)
        assert float(np.max(np.abs(gf - rf))) <= 1e-6


def test_training_labels_match_oracle(ls):
    # posteriors from 1e-16 to 1 (and exact zeros) at random candidates, -1 padding and one id
    # outside [0, N) (NaN by the header's contract)
    import torch
    rng = np.random.default_rng(31)
    w = synth.make_workload("ls_n50000_l20000", N=150, L=300, seed=22)
    N, C = w["N"], 64
    P = np.exp(rng.uniform(np.log(1e-16), 0.0, size=(N, N))).astype(np.float32)
    P[rng.random((N, N)) < 0.05] = 0.0
    P[0, 0] = 1.0
    cand = rng.integers(-1, N, size=(N, C)).astype(np.int32)
    cand[0, 0] = 0
    cand[1, 3] = N
    ctx = ls.ls_create(w["h"])
    try:
        y = torch.full((N, C), -7.0, dtype=torch.float32, device="cuda")
        ls.ls_propose_labels(ctx, torch.from_numpy(P).cuda(), torch.from_numpy(cand).cuda(), C, y)
        y = y.cpu().numpy()
    finally:
        ls.ls_destroy(ctx)
    assert np.isnan(y[1, 3]) and y[0, 0] == 1.0
    cand[1, 3] = -1
    y[1, 3] = 0.0
    ref = op.labels(P.astype(np.float64), cand)
    assert float(np.max(np.abs(y - ref))) <= 3e-6


def test_mlp_inference_and_gradient_match_oracle(ls):
    import torch
    rng = np.random.default_rng(5)
    p = (rng.normal(0, 1, op.N_PARAMS) * 0.15).astype(np.float32)
    X = rng.random((3000, 8)).astype(np.float32)
    X[:, 7] = 0.0
    y = rng.random(3000).astype(np.float32)
    m = ls.ls_mlp_create(p)
    try:
        Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
        s = torch.empty(3000, dtype=torch.float32, device="cuda")
        ls.ls_mlp_forward(m, Xd, s)
        g, loss = ls.ls_mlp_grad(m, Xd, yd)
        np.testing.assert_array_equal(ls.ls_mlp_get(m), p)
        s = s.cpu().numpy().astype(np.float64)
    finally:
        ls.ls_mlp_destroy(m)
    p64, X64 = p.astype(np.float64), X.astype(np.float64)
    ref16 = op.mlp_forward_bf16(p64, X64)
    scale = float(np.max(np.abs(ref16)))
    # FP32 accumulation against exact sums; a pre-activation on a BF16 rounding boundary may round
    # the other way (2^-8 of one hidden unit)
    assert float(np.max(np.abs(s - ref16))) <= 2e-3 * scale, float(np.max(np.abs(s - ref16)))
    ref = op.mlp_forward(p64, X64)
    assert float(np.max(np.abs(s - ref))) <= 3e-2 * scale  # BF16 weights and activations vs exact
    rl, rg = op.mlp_loss_grad(p64, X64, y.astype(np.float64))
    assert abs(loss - rl) <= 1e-5 * rl
    assert float(np.linalg.norm(g - rg) / np.linalg.norm(rg)) <= 1e-5
    assert float(np.max(np.abs(g - rg))) <= 1e-4 * float(np.max(np.abs(rg)))


def test_mlp_scorer_pipeline_many_tiles_per_cta(ls):
    """Several 128-row tiles per persistent CTA (the two-accumulator pipeline in steady state), a
    ragged last tile, and all eight inputs non-zero, against the BF16-rounding network oracle."""
    import torch
    rng = np.random.default_rng(17)
    p = (rng.normal(0, 1, op.N_PARAMS) * 0.15).astype(np.float32)
    n = 152 * 128 * 3 + 77
    X = rng.random((n, 8)).astype(np.float32)
    m = ls.ls_mlp_create(p)
    try:
        s = torch.empty(n, dtype=torch.float32, device="cuda")
        ls.ls_mlp_forward(m, torch.from_numpy(X).cuda(), s)
        s = s.cpu().numpy().astype(np.float64)
    finally:
        ls.ls_mlp_destroy(m)
    ref16 = op.mlp_forward_bf16(p.astype(np.float64), X.astype(np.float64))
    scale = float(np.max(np.abs(ref16)))
    assert float(np.max(np.abs(s - ref16))) <= 2e-3 * scale, float(np.max(np.abs(s - ref16)))


def test_mlp_topk_keeps_the_best_scores(ls):
    import torch
    w = synth.make_workload("ls_n50000_l20000", N=120, L=800, seed=23)
    N, L = w["N"], w["L"]
    Wn = op.windows(L)
    K, C = 16, 64
    ctx = ls.ls_create(w["h"])
    m = ls.ls_mlp_create(None, 3)
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        idx = torch.empty((N, Wn, K), dtype=torch.int32, device="cuda")
        ls.ls_propose(ctx, C, K, m, idx)
        cand = torch.empty((N, C), dtype=torch.int32, device="cuda")
        feat = torch.empty((N, C, 8), dtype=torch.float32, device="cuda")
        wi = 1
        ls.ls_propose_window(ctx, C, wi, cand, feat)
        sc = torch.empty(N * C, dtype=torch.float32, device="cuda")
        ls.ls_mlp_forward(m, feat.reshape(N * C, 8), sc)
        sc = sc.reshape(N, C).cpu().numpy()
        cand = cand.cpu().numpy()
        idx = idx.cpu().numpy()
    finally:
        ls.ls_mlp_destroy(m)
        ls.ls_destroy(ctx)
    for i in range(N):
        order = sorted(range(C), key=lambda q: (-sc[i, q], cand[i, q]))
        best = sorted(int(cand[i, q]) for q in order[:K])
        assert list(idx[i, wi]) == best
        assert np.all(np.diff(idx[i, wi]) > 0) and i not in idx[i, wi]


def sparse_stats(ds, dd, trust):
    """coverage (trusted entries) and |d_sparse - d_dense| statistics over the trusted entries."""
    import torch
    fin = trust
    e = (ds - dd).abs()[fin]
    sample = e[torch.randperm(e.numel(), device=e.device)[:2000000]]
    q = torch.quantile(sample, torch.tensor([0.5, 0.9, 0.99], device=e.device)).tolist()
    return dict(coverage=float(fin.float().mean()), q50=q[0], q90=q[1], q99=q[2], max=float(e.max()),
                frac_le_1e3=float((e <= 1e-3).float().mean()))


def test_sparse_distances_against_dense_and_fallback(ls):
    """K = 128 of N - 1 = 399 donors per window (widened to the neighbouring windows' sets) on the
    N = 50000 generator scaled down (founders N/25 as there): covered entries against the dense
    path, and targets above the lost-mass tolerance fall back to rows equal to the dense path's."""
    import torch
    w = synth.make_workload("ls_n50000_l20000", N=400, L=3000, seed=27, founders=16)
    N, L = w["N"], w["L"]
    loci = synth.decode_loci(L, 4)
    Wn = op.windows(L)
    K, tol = 128, 0.05
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        dd = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
        ls.ls_run_all(ctx, loci, dd)
        idx = torch.empty((N, Wn, K), dtype=torch.int32, device="cuda")
        ls.ls_propose(ctx, K, K, None, idx)
        ds = torch.empty_like(dd)
        lost = torch.empty(N, dtype=torch.float32, device="cuda")
        tm = torch.empty((len(loci), N, (N + 31) // 32), dtype=torch.int32, device="cuda")
        rc, pac, nf = ls.ls_sparse_run_all(ctx, idx, K, 256, loci, ds, lost_tol=-1.0, lost_out=lost, trust_out=tm)
        assert bool(torch.isfinite(ds).all())   # complete: outside donors carry the pool's share
        st0 = sparse_stats(ds, dd, ls.trust_bits(tm, N))
        lost_h = lost.cpu().numpy()
        df = torch.empty_like(dd)
        rc2, _, nf2 = ls.ls_sparse_run_all(ctx, idx, K, 256, loci, df, lost_tol=tol, trust_out=tm)
        torch.cuda.synchronize()
        fb = np.flatnonzero(~(lost_h <= tol))
        assert nf2 == fb.size
        if fb.size:
            sub = df[:, fb][:, :, fb]
            ref = dd[:, fb][:, :, fb]
            assert d_err(sub.cpu().numpy(), ref.cpu().numpy().astype(np.float64)) <= 1e-5
        st1 = sparse_stats(df, dd, ls.trust_bits(tm, N))
    finally:
        ls.ls_destroy(ctx)
    assert rc == 0 and nf == 0
    print("\nsparse K=%d N=%d: %s; with fallback of %d targets: %s" % (K, N, st0, fb.size, st1))
    assert st0["coverage"] > 0.2 and st1["coverage"] >= st0["coverage"]
    assert st0["q50"] <= 1e-2 and st1["q50"] <= st0["q50"] + 1e-6


def test_trained_proposal_against_raw_counts(ls):
    """The network trained on dense posteriors of one instance (N = 1000, founders N/25) against
    the raw match-count sets of the same size on another instance: posterior mass the sets cover
    at the windows' middle loci, and the sparse distances' error."""
    import torch
    from paper_2212_11403_gb300 import proposal
    N, L, F, C, K = 1000, 4096, 40, 256, 64
    wins = list(range(L // 256))
    wt = synth.make_workload("ls_n50000_l20000", N=N, L=L, seed=101, founders=F)
    ctx = ls.ls_create(wt["h"])
    try:
        ls.ls_set_params(ctx, wt["rho"], wt["mu"])
        X, y = proposal.training_set(ctx, N, L, C, wins)
    finally:
        ls.ls_destroy(ctx)
    m, loss = proposal.train(X, y, steps=800, batch=8192, lr=1e-3, seed=5)
    we = synth.make_workload("ls_n50000_l20000", N=N, L=L, seed=202, founders=F)
    ctx = ls.ls_create(we["h"])
    res = {}
    try:
        ls.ls_set_params(ctx, we["rho"], we["mu"])
        P = proposal.dense_posteriors(ctx, N, [proposal.window_mid(L, v) for v in wins])
        loci = np.array([proposal.window_mid(L, v) for v in (3, 8, 13)], dtype=np.int32)
        dd = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
        ls.ls_run_all(ctx, loci, dd)
        for name, net in (("raw", None), ("mlp", m)):
            idx = torch.empty((N, len(wins), K), dtype=torch.int32, device="cuda")
            ls.ls_propose(ctx, C, K, net, idx)
            mass = proposal.set_mass(idx, P, wins)
            ds = torch.empty_like(dd)
            tm = torch.empty((len(loci), N, (N + 31) // 32), dtype=torch.int32, device="cuda")
            ls.ls_sparse_run_all(ctx, idx, K, 256, loci, ds, trust_out=tm)
            res[name] = dict(mass_mean=float(mass.mean()), mass_q01=float(torch.quantile(mass.flatten(), 0.01)),
                             **sparse_stats(ds, dd, ls.trust_bits(tm, N)))
    finally:
        ls.ls_destroy(ctx)
        ls.ls_mlp_destroy(m)
    print("\ntraining loss %.4g; raw %s; mlp %s" % (loss, res["raw"], res["mlp"]))
    assert math.isfinite(loss)
    # the network's sets cover more posterior mass, most of all for the worst-covered targets
    assert res["mlp"]["mass_mean"] >= res["raw"]["mass_mean"]
    assert res["mlp"]["mass_q01"] > res["raw"]["mass_q01"]


@pytest.mark.parametrize("lookahead,pool", [(0, False), (1, False), (2, False), (0, True), (2, True)])
def test_restricted_chain_matches_its_oracle(ls, lookahead, pool):
    """random per-window sets that change between windows: the kernels against the FP64 oracle
    of the restricted chain (oracle/proposal.py sparse_posteriors)."""
    import torch
    rng = np.random.default_rng(41)
    w = synth.make_workload("ls_n50000_l20000", N=40, L=300, seed=43, founders=4)
    N, L = w["N"], w["L"]
    WS, K = 32, 12
    Wn = (L + WS - 1) // WS
    S = -np.ones((N, Wn, K), dtype=np.int32)
    for i in range(N):
        for v in range(Wn):
            k = int(rng.integers(K - 3, K + 1))
            S[i, v, :k] = np.sort(rng.choice([j for j in range(N) if j != i], size=k, replace=False))
    loci = np.array([0, 31, 32, 100, 150, L - 1], dtype=np.int32)
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        d = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
        tm = torch.empty((len(loci), N, (N + 31) // 32), dtype=torch.int32, device="cuda")
        ls.ls_sparse_run_all(ctx, torch.from_numpy(S).cuda(), K, WS, loci, d, lookahead=lookahead, pool=pool,
                             trust_out=tm)
        torch.cuda.synchronize()
        d = d.cpu().numpy().astype(np.float64)
        trust = ls.trust_bits(tm, N).cpu().numpy()
    finally:
        ls.ls_destroy(ctx)
    sets = op.lookahead_sets(S, lookahead) if lookahead else S
    p = op.sparse_posteriors(w["h"], w["rho"], w["mu"], sets, WS, loci, pool=pool)
    eps = 2.0 ** -52
    for k, l in enumerate(loci):
        v = l // WS
        H = np.full((N, N), np.nan)
        inset = np.zeros((N, N), dtype=bool)
        for i in range(N):
            for j in sets[i, v]:
                if j >= 0:
                    inset[i, j] = True
            for j in range(N):
                if j != i and (inset[i, j] or pool):
                    H[i, j] = -0.5 * np.log(max(p[i, k, j], eps))
        ref = H + H.T
        np.fill_diagonal(ref, 0.0)
        # with the pool every entry is defined (outside donors carry the pool's share); without it
        # entries with an outside donor on either side are NaN
        assert np.array_equal(np.isfinite(d[k]), np.isfinite(ref)), l
        fin = np.isfinite(ref)
        err = np.abs(d[k][fin] - ref[fin]) / np.maximum(1.0, np.abs(ref[fin]))
        assert float(err.max()) <= D_TOL, (l, float(err.max()))
        # trust bits (no distance bound given): both halves are chain posteriors
        both = inset & inset.T
        np.fill_diagonal(both, False)
        np.testing.assert_array_equal(trust[k], both)
