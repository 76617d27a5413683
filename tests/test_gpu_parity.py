"""CUDA path vs the FP64 oracle, through the C ABI (pytest -m gpu).

Tolerance.  The recurrences run in FP32 with FP64 log scales.  Distances are judged with
err = max over entries of |d_gpu - d_ref| / max(|d_ref|, 1) <= 1e-5 (dense FP32 target); posteriors,
forward and backward tables with a relative error bound of 2e-4 on entries above 1e-30
(FP32 rounding compounds over the loci between resets of a donor's state, and the stored tables
are not renormalised).  Log scales: each locus adds log of an FP32 normaliser, whose absolute
error is about 2^-24 (the normaliser is near 1 on most loci), so a sum over L loci and n targets
is held to 1e-6 relative plus 2e-7 * L * sqrt(n) absolute.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2212_11403_gb300 import synth

pytestmark = pytest.mark.gpu

D_TOL = 1e-5
TAB_RTOL = 2e-4
LOG_RTOL = 1e-6


def log_close(got, ref, L, n=1):
    """log-likelihood tolerance: relative 1e-6 plus an FP32-normaliser term per locus."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    tol = LOG_RTOL * np.abs(ref) + 2e-7 * L * math.sqrt(n)
    return bool(np.all(np.abs(got - ref) <= tol)), float(np.max(np.abs(got - ref)))


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


def rel_close(got, ref, rtol, floor=1e-30):
    got = np.asarray(got, dtype=np.float64)
    m = np.abs(ref) > floor
    if not m.any():
        return True, 0.0
    e = float(np.max(np.abs(got[m] - ref[m]) / np.abs(ref[m])))
    return e <= rtol, e


def run_all_gpu(ls, w, loci):
    import torch
    N = w["N"]
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        d = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
        st = torch.zeros(N, dtype=torch.int32, device="cuda")
        rc, pac = ls.ls_run_all(ctx, loci, d, status_out=st)
        torch.cuda.synchronize()
        return rc, pac, d.cpu().numpy(), st.cpu().numpy()
    finally:
        ls.ls_destroy(ctx)


# ---------------------------------------------------------------- haplotype cache (integer, exact)
@pytest.mark.parametrize("N,L", [(2, 1), (37, 5), (64, 3), (300, 400), (1000, 7)])
def test_pack_matches_oracle_layout_and_query(ls, N, L):
    rng = np.random.default_rng(N * 31 + L)
    h = (rng.random((L, N)) < 0.5).astype(np.uint8)
    ctx = ls.ls_create(h)
    try:
        words = ls.ls_export_packed(ctx)
        _, ow = oracle.pack_paper_layout(h)
        nw = (N + 31) // 32
        np.testing.assert_array_equal(words[:, :nw], ow[:, :nw])
        assert np.all(words[:, nw:] == 0)
        loci = rng.integers(0, L, size=min(L, 5))
        haps = rng.integers(0, N, size=min(N, 9))
        np.testing.assert_array_equal(ls.ls_query(ctx, loci, haps), h[loci][:, haps])
        info = ls.ls_info(ctx)
        assert info["N"] == N and info["L"] == L and info["row_words"] >= nw + 1
    finally:
        ls.ls_destroy(ctx)


# ---------------------------------------------------------------- the fused pipeline
def test_run_all_n200_l1000_full_parity(ls):
    w = synth.make_workload("ls_n200_l1000")
    loci = w["loci"]
    rc, pac, d, st = run_all_gpu(ls, w, loci)
    assert rc == 0 and not st.any()
    ref = oracle.run(w["h"], w["rho"], w["mu"], loci, want=("post", "llf"))
    for k in range(len(loci)):
        dref = oracle.distance_block(ref["post"][:, k, :], np.arange(w["N"]))
        e = d_err(d[k], dref)
        assert e <= D_TOL, "locus %d: err %.3g" % (loci[k], e)
    assert log_close(pac, ref["llf"].sum(), w["L"], w["N"])[0]


@pytest.mark.parametrize("N", [2, 3, 7, 31, 33, 100, 203, 517, 1290, 2561, 5000])
def test_run_all_ragged_sizes(ls, N):
    L = 60
    w = synth.make_workload("ls_n5000_l20000", N=N, L=L, seed=77 + N)
    loci = np.array([0, 29, L - 1], dtype=np.int32)
    rc, pac, d, st = run_all_gpu(ls, w, loci)
    assert rc == 0
    ref = oracle.run(w["h"], w["rho"], w["mu"], loci, want=("post", "llf"), nthreads=0)
    for k in range(len(loci)):
        dref = oracle.distance_block(ref["post"][:, k, :], np.arange(N))
        assert d_err(d[k], dref) <= D_TOL, (N, k, d_err(d[k], dref))
        assert np.all(np.diag(d[k]) == 0.0)
        np.testing.assert_array_equal(d[k], d[k].T)
    assert log_close(pac, ref["llf"].sum(), L, N)[0], log_close(pac, ref["llf"].sum(), L, N)


def test_single_locus(ls):
    w = synth.make_workload("ls_n200_l1000", N=50, L=1)
    w["rho"] = np.zeros(0)
    rc, pac, d, st = run_all_gpu(ls, w, np.array([0], dtype=np.int32))
    ref = oracle.run(w["h"], w["rho"], w["mu"], [0], want=("post", "llf"))
    dref = oracle.distance_block(ref["post"][:, 0, :], np.arange(50))
    assert d_err(d[0], dref) <= D_TOL
    assert log_close(pac, ref["llf"].sum(), 1, 50)[0]


# ---------------------------------------------------------------- tables
def test_tables_forward_backward_posterior_vs_oracle(ls):
    import torch
    w = synth.make_workload("ls_n200_l1000", N=150, L=300, seed=5)
    N, L = w["N"], w["L"]
    t0, t1 = 10, 50
    T = t1 - t0
    ctx = ls.ls_create(w["h"])
    try:
        hsh = ls.ls_set_params(ctx, w["rho"], w["mu"])
        fw = ls.ls_table_create(ctx, ls.LS_FWD, t0, t1)
        bw = ls.ls_table_create(ctx, ls.LS_BWD, t0, t1)
        fst = [0, 57, 120]
        A = torch.empty((3, T, N), dtype=torch.float32, device="cuda")
        ls.ls_forward(ctx, fw, 120, fst, A)
        bst = [299, 200, 120]
        B = torch.empty((3, T, N), dtype=torch.float32, device="cuda")
        ls.ls_backward(ctx, bw, 120, bst, B)
        P = torch.empty((T, N), dtype=torch.float32, device="cuda")
        ls.ls_posterior(ctx, fw, bw, P)
        lf = torch.empty(T, dtype=torch.float64, device="cuda")
        lgb = torch.empty(T, dtype=torch.float64, device="cuda")
        ls.ls_table_read(fw, logscale=lf)
        ls.ls_table_read(bw, logscale=lgb)
        torch.cuda.synchronize()
        info = ls.ls_table_info(fw)
        assert info["locus"] == 120 and info["hash"] == hsh and info["t_from"] == t0 and info["t_to"] == t1
        targets = np.arange(t0, t1)
        ref = oracle.run(w["h"], w["rho"], w["mu"], [0, 57, 120, 200, 299], targets=targets,
                         want=("alpha", "beta", "post", "logF", "logG"))
        A, B, P = A.cpu().numpy(), B.cpu().numpy(), P.cpu().numpy()
        for k, kk in enumerate([0, 1, 2]):
            ok, e = rel_close(A[k], ref["alpha"][:, kk, :], TAB_RTOL)
            assert ok, ("alpha", fst[k], e)
        for k, kk in enumerate([4, 3, 2]):
            ok, e = rel_close(B[k], ref["beta"][:, kk, :], TAB_RTOL)
            assert ok, ("beta", bst[k], e)
        ok, e = rel_close(P, ref["post"][:, 2, :], TAB_RTOL, floor=1e-12)
        assert ok, ("post", e)
        np.testing.assert_allclose(P.sum(axis=1), 1.0, rtol=1e-5)
        assert log_close(lf.cpu().numpy(), ref["logF"][:, 2], 121)[0]
        assert log_close(lgb.cpu().numpy(), ref["logG"][:, 2], 180)[0]
        # resume the forward table to the last locus: log F there is the log-likelihood
        ls.ls_forward(ctx, fw, L - 1)
        ls.ls_table_read(fw, logscale=lf)
        torch.cuda.synchronize()
        llf = oracle.run(w["h"], w["rho"], w["mu"], [0], targets=targets, want=("llf",))["llf"]
        assert log_close(lf.cpu().numpy(), llf, L)[0]
        ls.ls_table_destroy(fw)
        ls.ls_table_destroy(bw)
    finally:
        ls.ls_destroy(ctx)


def test_resume_and_copy_match_direct_propagation(ls):
    import torch
    w = synth.make_workload("ls_n200_l1000", N=120, L=200, seed=9)
    N = w["N"]
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        a = ls.ls_table_create(ctx, ls.LS_FWD, 0, N)
        b = ls.ls_table_create(ctx, ls.LS_FWD, 0, N)
        c = ls.ls_table_create(ctx, ls.LS_FWD, 0, N)
        ls.ls_forward(ctx, a, 150)
        ls.ls_forward(ctx, b, 40)
        ls.ls_table_copy(c, b)          # CopyTable: deep copy, then both move on independently
        ls.ls_forward(ctx, b, 150)
        ls.ls_forward(ctx, c, 99)
        ls.ls_forward(ctx, c, 150)
        xa, xb, xc = (torch.empty((N, N), dtype=torch.float32, device="cuda") for _ in range(3))
        for t, x in ((a, xa), (b, xb), (c, xc)):
            ls.ls_table_read(t, state=x)
        torch.cuda.synchronize()
        np.testing.assert_allclose(xb.cpu().numpy(), xa.cpu().numpy(), rtol=1e-5, atol=1e-30)
        np.testing.assert_allclose(xc.cpu().numpy(), xa.cpu().numpy(), rtol=1e-5, atol=1e-30)
        # a reset table starts again at locus 0
        ls.ls_table_reset(c)
        assert ls.ls_table_info(c)["locus"] == -1
        ls.ls_forward(ctx, c, 150)
        ls.ls_table_read(c, state=xc)
        torch.cuda.synchronize()
        np.testing.assert_allclose(xc.cpu().numpy(), xa.cpu().numpy(), rtol=1e-6, atol=1e-30)
        # backward resume
        e = ls.ls_table_create(ctx, ls.LS_BWD, 0, N)
        f = ls.ls_table_create(ctx, ls.LS_BWD, 0, N)
        ls.ls_backward(ctx, e, 30)
        ls.ls_backward(ctx, f, 120)
        ls.ls_backward(ctx, f, 30)
        ls.ls_table_read(e, state=xa)
        ls.ls_table_read(f, state=xb)
        torch.cuda.synchronize()
        np.testing.assert_allclose(xb.cpu().numpy(), xa.cpu().numpy(), rtol=1e-5, atol=1e-30)
        for t in (a, b, c, e, f):
            ls.ls_table_destroy(t)
    finally:
        ls.ls_destroy(ctx)


def test_distance_from_tables_matches_run_all(ls):
    import torch
    w = synth.make_workload("ls_n200_l1000", N=130, L=150, seed=13)
    N = w["N"]
    l = 77
    rc, pac, d_all, st = run_all_gpu(ls, w, np.array([l], dtype=np.int32))
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        fw = ls.ls_table_create(ctx, ls.LS_FWD, 0, N)
        bw = ls.ls_table_create(ctx, ls.LS_BWD, 0, N)
        ls.ls_forward(ctx, fw, l)
        ls.ls_backward(ctx, bw, l)
        d = torch.empty((N, N), dtype=torch.float32, device="cuda")
        ls.ls_distance(ctx, fw, bw, d)
        torch.cuda.synchronize()
        assert d_err(d.cpu().numpy(), d_all[0].astype(np.float64)) <= 1e-6
        ls.ls_table_destroy(fw)
        ls.ls_table_destroy(bw)
    finally:
        ls.ls_destroy(ctx)


# ---------------------------------------------------------------- errors and numerical status
def test_error_paths(ls):
    import torch
    w = synth.make_workload("ls_n200_l1000", N=40, L=30, seed=3)
    ctx = ls.ls_create(w["h"])
    try:
        with pytest.raises(ls.LSError) as ei:
            ls.ls_table_create(ctx, ls.LS_FWD, 0, 40)
        assert ei.value.code == ls.LS_ERR_STATE  # parameters not set yet
        bad = w["rho"].copy()
        bad[3] = 1.5
        with pytest.raises(ls.LSError) as ei:
            ls.ls_set_params(ctx, bad, w["mu"])
        assert ei.value.code == ls.LS_ERR_ARG
        with pytest.raises(ls.LSError):
            ls.ls_set_params(ctx, w["rho"], -1e-3)
        Pi = torch.full((40, 40), 1.0 / 39, dtype=torch.float32, device="cuda")
        with pytest.raises(ls.LSError) as ei:
            ls.ls_set_params(ctx, w["rho"], w["mu"], Pi)  # nonzero diagonal
        assert ei.value.code == ls.LS_ERR_ARG
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        fw = ls.ls_table_create(ctx, ls.LS_FWD, 0, 40)
        bw = ls.ls_table_create(ctx, ls.LS_BWD, 0, 40)
        ls.ls_forward(ctx, fw, 20)
        with pytest.raises(ls.LSError) as ei:
            ls.ls_forward(ctx, fw, 10)
        assert ei.value.code == ls.LS_ERR_DIRECTION
        with pytest.raises(ls.LSError) as ei:
            ls.ls_backward(ctx, fw, 10)  # wrong kind
        assert ei.value.code == ls.LS_ERR_ARG
        ls.ls_backward(ctx, bw, 15)
        P = torch.empty((40, 40), dtype=torch.float32, device="cuda")
        with pytest.raises(ls.LSError) as ei:
            ls.ls_posterior(ctx, fw, bw, P)
        assert ei.value.code == ls.LS_ERR_LOCUS_MISMATCH
        with pytest.raises(ls.LSError) as ei:
            ls.ls_backward(ctx, bw, 20)
        assert ei.value.code == ls.LS_ERR_DIRECTION
        with pytest.raises(ls.LSError) as ei:
            ls.ls_forward(ctx, fw, 28, store_loci=[25, 24], alpha_out=torch.empty((2, 40, 40), device="cuda"))
        assert ei.value.code == ls.LS_ERR_ARG
        part = ls.ls_table_create(ctx, ls.LS_BWD, 0, 20)
        ls.ls_backward(ctx, part, 20)
        with pytest.raises(ls.LSError) as ei:
            ls.ls_posterior(ctx, fw, part, P)
        assert ei.value.code == ls.LS_ERR_RANGE
        # a new parameter set invalidates tables propagated under the old one (Sec. 4.1.2)
        ls.ls_set_params(ctx, w["rho"] * 0.5, w["mu"])
        with pytest.raises(ls.LSError) as ei:
            ls.ls_forward(ctx, fw, 25)
        assert ei.value.code == ls.LS_ERR_PARAM_MISMATCH
        with pytest.raises(ls.LSError) as ei:
            ls.ls_run_all(ctx, np.arange(65, dtype=np.int32) % 30, torch.empty((65, 40, 40), device="cuda"))
        for t in (fw, bw, part):
            ls.ls_table_destroy(t)
    finally:
        ls.ls_destroy(ctx)


def test_total_underflow_sets_status(ls):
    # mu = 0 and a private allele: all emissions vanish at that locus (App. A.3 total underflow)
    N, L = 40, 12
    h = np.zeros((L, N), dtype=np.uint8)
    h[5, 7] = 1
    w = dict(h=h, N=N, L=L, rho=np.full(L - 1, 0.05), mu=0.0)
    rc, pac, d, st = run_all_gpu(ls, w, np.array([2], dtype=np.int32))
    assert rc == ls.LS_WARN_UNDERFLOW
    assert st[7] & ls.LS_STATUS_UNDERFLOW
    assert not math.isfinite(pac)


# ---------------------------------------------------------------- full-size workload, sampled
def test_run_all_n5000_l20000_sampled_targets(ls):
    """Dense FP32 workload at its full size, in the launch configuration the benchmark times:
    d among 64 seeded-random targets and their log-likelihoods against the oracle."""
    import torch
    w = synth.make_workload("ls_n5000_l20000")
    N, L, loci = w["N"], w["L"], w["loci"]
    rng = np.random.default_rng(2024)
    targets = np.sort(rng.choice(N, size=64, replace=False)).astype(np.int32)
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        d = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
        rc, pac = ls.ls_run_all(ctx, loci, d)
        fw = ls.ls_table_create(ctx, ls.LS_FWD, 0, N)
        ls.ls_forward(ctx, fw, L - 1)
        lf = torch.empty(N, dtype=torch.float64, device="cuda")
        ls.ls_table_read(fw, logscale=lf)
        torch.cuda.synchronize()
        ls.ls_table_destroy(fw)
        sub = d[:, targets][:, :, targets].cpu().numpy()
        lf = lf.cpu().numpy()
    finally:
        ls.ls_destroy(ctx)
    assert rc == 0
    assert abs(pac - lf.sum()) <= 1e-9 * abs(pac)
    ref = oracle.run(w["h"], w["rho"], w["mu"], loci, targets=targets, want=("post", "llf"))
    assert log_close(lf[targets], ref["llf"], L)[0], log_close(lf[targets], ref["llf"], L)
    for k in range(len(loci)):
        dref = oracle.distance_block(ref["post"][:, k, :], targets)
        e = d_err(sub[k], dref)
        assert e <= D_TOL, "locus %d: err %.3g" % (loci[k], e)


# ------------------------------------------------ large N (state in registers and shared memory)
@pytest.mark.parametrize("N", [20481, 30001, 50000, 57000])
def test_run_all_large_n_sampled(ls, N):
    """N beyond the register-tile kernels (one target per CTA of 512 threads, state partly in shared
    memory): d among 16 sampled targets and their log-likelihoods against the oracle."""
    import torch
    L = 40
    w = synth.make_workload("ls_n50000_l20000", N=N, L=L, seed=900 + N % 97, founders=N // 25)
    loci = np.array([0, 19, L - 1], dtype=np.int32)
    targets = np.sort(np.random.default_rng(N).choice(N, size=16, replace=False))
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        d = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
        rc, pac = ls.ls_run_all(ctx, loci, d)
        ti = torch.from_numpy(targets.astype(np.int64)).cuda()
        sub = d[:, ti][:, :, ti].cpu().numpy()
        del d
        fw = ls.ls_table_create(ctx, ls.LS_FWD, 0, N)
        ls.ls_forward(ctx, fw, L - 1)
        lf = torch.empty(N, dtype=torch.float64, device="cuda")
        ls.ls_table_read(fw, logscale=lf)
        torch.cuda.synchronize()
        ls.ls_table_destroy(fw)
        lf = lf.cpu().numpy()
    finally:
        ls.ls_destroy(ctx)
    assert rc == 0
    assert abs(pac - lf.sum()) <= 1e-9 * abs(pac)
    ref = oracle.run(w["h"], w["rho"], w["mu"], loci, targets=targets, want=("post", "llf"))
    assert log_close(lf[targets], ref["llf"], L)[0]
    for k in range(len(loci)):
        dref = oracle.distance_block(ref["post"][:, k, :], targets)
        assert d_err(sub[k], dref) <= D_TOL, (N, k, d_err(sub[k], dref))


def test_large_n_fallback_rows_match_dense(ls):
    """the sparse path's dense fallback (one-target CTAs over a target list) at N = 30000."""
    import torch
    N, L, K = 30000, 1000, 32
    w = synth.make_workload("ls_n50000_l20000", N=N, L=L, seed=77, founders=N // 25)
    loci = np.array([10, 600, 999], dtype=np.int32)
    Wn = (L + 255) // 256
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        idx = torch.empty((N, Wn, K), dtype=torch.int32, device="cuda")
        ls.ls_propose(ctx, K, K, None, idx)
        ds = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
        lost = torch.empty(N, dtype=torch.float32, device="cuda")
        ls.ls_sparse_run_all(ctx, idx, K, 256, loci, ds, lost_tol=-1.0, lost_out=lost)
        lh = lost.cpu().numpy()
        tol = float(np.sort(lh)[-11])  # the (at most) ten targets with the largest lost mass fall back
        rc, _, nf = ls.ls_sparse_run_all(ctx, idx, K, 256, loci, ds, lost_tol=tol)
        fb = np.flatnonzero(~(lh <= tol))
        assert nf == fb.size > 0
        ti = torch.from_numpy(fb.astype(np.int64)).cuda()
        sub = ds[:, ti][:, :, ti].cpu().numpy()
        del ds
        dd = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
        ls.ls_run_all(ctx, loci, dd)
        ref = dd[:, ti][:, :, ti].cpu().numpy()
        del dd
    finally:
        ls.ls_destroy(ctx)
    assert d_err(sub, ref.astype(np.float64)) <= 1e-5


@pytest.mark.parametrize("N", [20481, 30001])
def test_large_n_resume_matches_direct_propagation(ls, N):
    """large-N kernels (state partly in shared memory) stopped and resumed through a table: the
    forward 0 -> 20 -> 50 and the backward L-1 -> 35 -> 10 end in the states of direct runs."""
    import torch
    L, T0, T1 = 60, 1000, 1064
    w = synth.make_workload("ls_n50000_l20000", N=N, L=L, seed=31, founders=N // 25)
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        xs = [torch.empty((T1 - T0, N), dtype=torch.float32, device="cuda") for _ in range(4)]
        lg = [torch.empty(T1 - T0, dtype=torch.float64, device="cuda") for _ in range(4)]
        for kind, stops, out in ((ls.LS_FWD, ([50], [20, 50]), (0, 1)), (ls.LS_BWD, ([10], [35, 10]), (2, 3))):
            for path, o in zip(stops, out):
                t = ls.ls_table_create(ctx, kind, T0, T1)
                for to in path:
                    (ls.ls_forward if kind == ls.LS_FWD else ls.ls_backward)(ctx, t, to)
                ls.ls_table_read(t, state=xs[o], logscale=lg[o])
                torch.cuda.synchronize()
                ls.ls_table_destroy(t)
    finally:
        ls.ls_destroy(ctx)
    x = [v.cpu().numpy() for v in xs]
    g = [v.cpu().numpy() for v in lg]
    for a, b in ((0, 1), (2, 3)):
        assert np.all(np.isfinite(x[a])) and x[a].max() > 0
        np.testing.assert_allclose(x[b], x[a], rtol=1e-5, atol=1e-30)
        # the resumed run re-sums the loaded state in its own order: FP32 rounding of one normaliser
        # per locus, about 1e-7 in the log each
        np.testing.assert_allclose(g[b], g[a], rtol=0, atol=1e-5)


def test_run_all_on_a_user_stream_and_without_tail_overlap(ls):
    """a main/tail plan (N=5000: four full waves plus a tail) forks its tail onto a side stream and
    joins it back; on a caller-created stream, and with the overlap switched off, the results are
    bit-identical to the default run."""
    import os
    import torch
    w = synth.make_workload("ls_n5000_l20000", N=5000, L=300, seed=5)
    N = w["N"]
    loci = np.array([0, 150, 299], dtype=np.int32)
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        d0 = torch.empty((3, N, N), dtype=torch.float32, device="cuda")
        rc0, pac0 = ls.ls_run_all(ctx, loci, d0)
        s = torch.cuda.Stream()
        d1 = torch.full_like(d0, float("nan"))
        with torch.cuda.stream(s):
            rc1, pac1 = ls.ls_run_all(ctx, loci, d1, stream=s)
        s.synchronize()
        os.environ["LS_TAIL_OVERLAP"] = "0"
        try:
            d2 = torch.empty_like(d0)
            rc2, pac2 = ls.ls_run_all(ctx, loci, d2)
        finally:
            del os.environ["LS_TAIL_OVERLAP"]
        torch.cuda.synchronize()
        assert rc0 == rc1 == rc2 == 0
        assert pac0 == pac1 == pac2
        assert torch.equal(d0, d1) and torch.equal(d0, d2)
    finally:
        ls.ls_destroy(ctx)
