"""Forward checkpoints (FP32 and binary16) and replay, against the FP64 oracle.

Bounds.  An FP32 snapshot is the table state itself: relative error 2e-4 as for stored alpha.  A
binary16 snapshot stores alpha_j / s (s = max_j alpha_j of the target) rounded to nearest, so
its error against the FP64 alpha is at most max(2^-11 alpha_j, 2^-25 s) on top of the FP32
error.  A replay decodes the nearest snapshot and propagates forward: FP32 replays meet the
table tolerance; binary16 replays carry the snapshot's rounding forward, damped by
recombination, and are held to the binary16 bound of the snapshot they started from (relative
2^-11 plus the FP32 term) on entries above 2^-14 s, with the absolute term scaled by the
largest forward growth of a small entry (one step adds at least theta rho pi_j).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2212_11403_gb300 import synth

pytestmark = pytest.mark.gpu

TAB_RTOL = 2e-4
U16 = 2.0 ** -11      # binary16 unit roundoff
SUB16 = 2.0 ** -25    # half the binary16 subnormal spacing


@pytest.fixture(scope="module")
def ls():
    import torch
    torch.cuda.set_device(0)
    from paper_2212_11403_gb300 import ls as _ls
    return _ls


def bisection_loci(a, b):
    """c_0 = a, c_k = b - floor((b - a) / 2^k), K = ceil(log2(b - a + 1))."""
    K = max(1, math.ceil(math.log2(b - a + 1)))
    return [a] + [b - ((b - a) >> k) for k in range(1, K)]


def rel_err(got, ref, floor=1e-30):
    got = np.asarray(got, dtype=np.float64)
    m = np.abs(ref) > floor
    return float(np.max(np.abs(got[m] - ref[m]) / np.abs(ref[m]))) if m.any() else 0.0


def f16_excess(got, ref):
    """max over entries of |got - ref| / (max(U16 |ref|, SUB16 s) + TAB_RTOL |ref|); <= 1 passes."""
    got = np.asarray(got, dtype=np.float64)
    s = ref.max(axis=-1, keepdims=True)
    bound = np.maximum(U16 * np.abs(ref), SUB16 * s) + TAB_RTOL * np.abs(ref) + 1e-300
    return float(np.max(np.abs(got - ref) / bound))


def l1_rel(got, ref):
    got = np.asarray(got, dtype=np.float64)
    return float(np.max(np.abs(got - ref).sum(axis=-1) / ref.sum(axis=-1)))


def make_ctx(ls, w, Pi32=None):
    import torch
    ctx = ls.ls_create(w["h"])
    ls.ls_set_params(ctx, w["rho"], w["mu"], None if Pi32 is None else torch.from_numpy(Pi32).cuda())
    return ctx


@pytest.mark.parametrize("prior", ["uniform", "gamma"])
def test_snapshots_match_oracle_alpha(ls, prior):
    import torch
    w = synth.make_workload("ls_n200_l1000")
    N, L = w["N"], w["L"]
    Pi = synth.gamma_prior_f32(w["pi_seed"], N) if prior == "gamma" else None
    t0, t1 = 0, N
    ctx = make_ctx(ls, w, Pi)
    try:
        cks = {}
        for dt in (ls.LS_CKPT_F32, ls.LS_CKPT_F16):
            fw = ls.ls_table_create(ctx, ls.LS_FWD, t0, t1)
            cks[dt] = ls.ls_checkpoints(ctx, fw, 0, L - 1, dt)
            assert ls.ls_table_info(fw)["locus"] == L - 1
            ls.ls_table_destroy(fw)
        info = ls.ls_ckpt_info(cks[ls.LS_CKPT_F16])
        loci = bisection_loci(0, L - 1)
        assert list(info["loci"]) == loci and info["n"] == 10
        assert info["device_bytes"] == 10 * N * (2 * N + 12)
        ref = oracle.run(w["h"], w["rho"], w["mu"], loci, Pi=Pi, want=("alpha", "logF"))
        A = torch.empty((N, N), dtype=torch.float32, device="cuda")
        lf = torch.empty(N, dtype=torch.float64, device="cuda")
        worst = {}
        for dt, name in ((ls.LS_CKPT_F32, "f32"), (ls.LS_CKPT_F16, "f16")):
            for k, l in enumerate(loci):
                ls.ls_ckpt_read(cks[dt], k, A, lf)
                torch.cuda.synchronize()
                a = A.cpu().numpy()
                ra = ref["alpha"][:, k, :]
                if dt == ls.LS_CKPT_F32:
                    e = rel_err(a, ra)
                    assert e <= TAB_RTOL, (l, e)
                else:
                    e = f16_excess(a, ra)
                    assert e <= 1.0, (l, e)
                worst[name] = max(worst.get(name, 0.0), l1_rel(a, ra))
                np.testing.assert_allclose(lf.cpu().numpy(), ref["logF"][:, k], rtol=1e-6, atol=2e-7 * (l + 1))
        print("\nsnapshot L1 relative error vs FP64 (%s prior): %s" % (prior, worst))
        for ck in cks.values():
            ls.ls_ckpt_destroy(ck)
    finally:
        ls.ls_destroy(ctx)


@pytest.mark.parametrize("prior", ["uniform", "gamma"])
def test_replay_posterior_matches_oracle(ls, prior):
    import torch
    w = synth.make_workload("ls_n200_l1000", N=180, L=700, seed=17)
    N, L = w["N"], w["L"]
    Pi = synth.gamma_prior_f32(19, N) if prior == "gamma" else None
    t0, t1 = 30, 110
    T = t1 - t0
    targets = np.arange(t0, t1)
    probe = [0, 137, 349, 350, 600, 697, 698, 699]
    ctx = make_ctx(ls, w, Pi)
    try:
        src = ls.ls_table_create(ctx, ls.LS_FWD, t0, t1)
        ls.ls_forward(ctx, src, 5)
        ck32 = ls.ls_checkpoints(ctx, src, 5, L - 1, ls.LS_CKPT_F32)
        ls.ls_table_reset(src)
        ck16 = ls.ls_checkpoints(ctx, src, 0, L - 1, ls.LS_CKPT_F16)
        assert list(ls.ls_ckpt_info(ck32)["loci"]) == bisection_loci(5, L - 1)
        fw = ls.ls_table_create(ctx, ls.LS_FWD, t0, t1)
        bw = ls.ls_table_create(ctx, ls.LS_BWD, t0, t1)
        ref = oracle.run(w["h"], w["rho"], w["mu"], probe, targets=targets, Pi=Pi, want=("alpha", "post"))
        A = torch.empty((T, N), dtype=torch.float32, device="cuda")
        P = torch.empty((T, N), dtype=torch.float32, device="cuda")
        errs = {"f32": 0.0, "f16": 0.0}
        for k in range(len(probe) - 1, -1, -1):
            l = probe[k]
            ls.ls_backward(ctx, bw, l)
            for ck, name in ((ck32, "f32"), (ck16, "f16")):
                if name == "f32" and l < 5:
                    with pytest.raises(ls.LSError) as ei:
                        ls.ls_ckpt_replay(ctx, ck, fw, l)
                    assert ei.value.code == ls.LS_ERR_ARG
                    continue
                ls.ls_ckpt_replay(ctx, ck, fw, l)
                assert ls.ls_table_info(fw)["locus"] == l
                ls.ls_table_read(fw, state=A)
                ls.ls_posterior(ctx, fw, bw, P)
                torch.cuda.synchronize()
                a, p = A.cpu().numpy(), P.cpu().numpy()
                ra, rp = ref["alpha"][:, k, :], ref["post"][:, k, :]
                if name == "f32":
                    assert rel_err(a, ra) <= TAB_RTOL, (l, rel_err(a, ra))
                    assert rel_err(p, rp, floor=1e-12) <= TAB_RTOL, (l, rel_err(p, rp, 1e-12))
                else:
                    # rounding of the snapshot, carried forward: relative 2^-11 on the
                    # posterior mass, far below the distance tolerance of the sparse path
                    assert l1_rel(a, ra) <= 2 * U16, (l, l1_rel(a, ra))
                    assert float(np.max(np.abs(p - rp))) <= 2 * U16, (l, float(np.max(np.abs(p - rp))))
                errs[name] = max(errs[name], float(np.max(np.abs(p - rp))))
        print("\nreplay max |p - p_FP64| (%s prior): %s" % (prior, errs))
        for t in (src, fw, bw):
            ls.ls_table_destroy(t)
        ls.ls_ckpt_destroy(ck32)
        ls.ls_ckpt_destroy(ck16)
    finally:
        ls.ls_destroy(ctx)


def test_checkpoint_errors(ls):
    import torch
    w = synth.make_workload("ls_n200_l1000", N=40, L=50, seed=3)
    ctx = make_ctx(ls, w)
    try:
        fw = ls.ls_table_create(ctx, ls.LS_FWD, 0, 40)
        bw = ls.ls_table_create(ctx, ls.LS_BWD, 0, 40)
        ls.ls_forward(ctx, fw, 20)
        with pytest.raises(ls.LSError) as ei:
            ls.ls_checkpoints(ctx, fw, 10, 30)  # table already beyond a
        assert ei.value.code == ls.LS_ERR_DIRECTION
        with pytest.raises(ls.LSError) as ei:
            ls.ls_checkpoints(ctx, fw, 25, 24)
        assert ei.value.code == ls.LS_ERR_ARG
        with pytest.raises(ls.LSError) as ei:
            ls.ls_checkpoints(ctx, fw, 25, 30, 7)
        assert ei.value.code == ls.LS_ERR_ARG
        with pytest.raises(ls.LSError) as ei:
            ls.ls_checkpoints(ctx, bw, 25, 30)
        assert ei.value.code == ls.LS_ERR_ARG
        ck = ls.ls_checkpoints(ctx, fw, 20, 20)  # a == b: one snapshot, the table stays
        info = ls.ls_ckpt_info(ck)
        assert info["n"] == 1 and list(info["loci"]) == [20]
        other = ls.ls_table_create(ctx, ls.LS_FWD, 0, 39)
        with pytest.raises(ls.LSError) as ei:
            ls.ls_ckpt_replay(ctx, ck, other, 30)
        assert ei.value.code == ls.LS_ERR_RANGE
        with pytest.raises(ls.LSError) as ei:
            ls.ls_ckpt_read(ck, 1, torch.empty((40, 40), device="cuda"))
        assert ei.value.code == ls.LS_ERR_ARG
        ls.ls_set_params(ctx, w["rho"] * 0.5, w["mu"])
        with pytest.raises(ls.LSError) as ei:
            ls.ls_ckpt_replay(ctx, ck, fw, 30)
        assert ei.value.code == ls.LS_ERR_PARAM_MISMATCH
        ls.ls_ckpt_destroy(ck)
        for t in (fw, bw, other):
            ls.ls_table_destroy(t)
    finally:
        ls.ls_destroy(ctx)


def test_checkpoints_n20000_l50000_f16_vs_f32(ls):
    """Dense LS at scale (N = 20000, L = 50000, Gamma(2, 1) prior): the ceil(log2 L) = 16
    snapshots of 16 consecutive targets in FP32 and binary16, each against FP64 alpha, and a
    replay to a locus between snapshots."""
    import torch
    w = synth.make_workload("ls_n20000_l50000")
    N, L = w["N"], w["L"]
    rho_gpu = ls.ls_calc_rho(w["gaps"], w["Ne"], 1.0)
    rho_ref = oracle.calc_rho(w["gaps"], w["Ne"], 1.0)
    Pi = synth.gamma_prior_f32(w["pi_seed"], N)
    t0, t1 = 9000, 9016
    T = t1 - t0
    loci = bisection_loci(0, L - 1)
    assert len(loci) == 16
    probe = 30000
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, rho_gpu, w["mu"], torch.from_numpy(Pi).cuda())
        cks = {}
        for dt in (ls.LS_CKPT_F32, ls.LS_CKPT_F16):
            fw = ls.ls_table_create(ctx, ls.LS_FWD, t0, t1)
            cks[dt] = ls.ls_checkpoints(ctx, fw, 0, L - 1, dt)
            ls.ls_table_destroy(fw)
        bw = ls.ls_table_create(ctx, ls.LS_BWD, t0, t1)
        ls.ls_backward(ctx, bw, probe)
        fw = ls.ls_table_create(ctx, ls.LS_FWD, t0, t1)
        A = torch.empty((T, N), dtype=torch.float32, device="cuda")
        P = torch.empty((T, N), dtype=torch.float32, device="cuda")
        snaps, posts = {}, {}
        for dt, name in ((ls.LS_CKPT_F32, "f32"), (ls.LS_CKPT_F16, "f16")):
            snaps[name] = []
            for k in range(len(loci)):
                ls.ls_ckpt_read(cks[dt], k, A)
                torch.cuda.synchronize()
                snaps[name].append(A.cpu().numpy())
            ls.ls_ckpt_replay(ctx, cks[dt], fw, probe)
            ls.ls_posterior(ctx, fw, bw, P)
            torch.cuda.synchronize()
            posts[name] = P.cpu().numpy()
        for ck in cks.values():
            ls.ls_ckpt_destroy(ck)
        ls.ls_table_destroy(fw)
        ls.ls_table_destroy(bw)
    finally:
        ls.ls_destroy(ctx)
    targets = np.arange(t0, t1)
    ref = oracle.run(w["h"], rho_ref, w["mu"], loci + [probe], targets=targets, Pi=Pi, want=("alpha", "post"))
    del Pi
    report = {}
    for name in ("f32", "f16"):
        l1 = max(l1_rel(snaps[name][k], ref["alpha"][:, k, :]) for k in range(len(loci)))
        pe = float(np.max(np.abs(posts[name] - ref["post"][:, -1, :])))
        report[name] = dict(snapshot_l1_rel=l1, replay_max_abs_p=pe)
        for k in range(len(loci)):
            if name == "f32":
                assert rel_err(snaps[name][k], ref["alpha"][:, k, :]) <= TAB_RTOL
            else:
                assert f16_excess(snaps[name][k], ref["alpha"][:, k, :]) <= 1.0
        assert pe <= (TAB_RTOL if name == "f32" else 2 * U16)
    print("\ncheckpoints N=20000 L=50000 vs FP64:", report)
