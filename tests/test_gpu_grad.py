"""Adjoint gradient of the PAC log-likelihood (ls_pac_grad and the autograd wrapper) against the
FP64 oracle's Fisher-identity gradient and against central finite differences (h = 1e-4) of the
oracle's PAC log-likelihood.

Tolerance.  Each group gradient is a difference of two terms of similar size: the posterior
expectation sum_i E[sum_m B_m / (1-rho_m)] (computed in FP32 per target, summed in FP64) and the
constant T sum_m rho_m / (1-rho_m).  Its error is held to 1e-5 of the magnitude of those terms:
the per-target expectations are FP32 recursions over up to L loci (relative error about 1e-6
at L = 10000); the same form is used for d/dlog mu.  The PAC log-likelihood uses the log
tolerance of the parity tests.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2212_11403_gb300 import synth

pytestmark = pytest.mark.gpu

G_RTOL = 1e-5


@pytest.fixture(scope="module")
def ls():
    import torch
    torch.cuda.set_device(0)
    from paper_2212_11403_gb300 import ls as _ls
    return _ls


def magnitudes(rho, mu, L, iv, K, T):
    """T * sum rho/(1-rho) per group and T * sum_l mu/(1-mu): the size of the subtracted terms."""
    c = np.zeros(K)
    np.add.at(c, iv, rho / (1.0 - rho))
    return T * c, T * L * mu / (1.0 - mu)


def check_grad(pac, gm, gr, ref, rho, mu, L, iv, K, T, N):
    rpac, rgm, rgr = ref
    cr, cm = magnitudes(rho, mu, L, iv, K, T)
    assert abs(pac - rpac) <= 1e-6 * abs(rpac) + 2e-7 * L * math.sqrt(T), (pac, rpac)
    assert abs(gm - rgm) <= G_RTOL * (abs(rgm) + cm), (gm, rgm, cm)
    err = np.abs(gr - rgr) / (np.abs(rgr) + cr + 1e-300)
    assert np.all(err <= G_RTOL), (float(err.max()), int(err.argmax()))
    return float(err.max()), abs(gm - rgm) / (abs(rgm) + cm)


@pytest.mark.parametrize("N,L,K", [(200, 1000, 100), (7, 40, 5), (33, 300, 7), (517, 200, 100), (2, 10, 3)])
def test_pac_grad_matches_oracle(ls, N, L, K):
    w = synth.make_workload("ls_n10000_l10000", N=N, L=L, seed=60 + N)
    iv = synth.rho_intervals(L, K)
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        rc, pac, gm, gr = ls.ls_pac_grad(ctx, iv, K)
    finally:
        ls.ls_destroy(ctx)
    assert rc == 0
    ref = oracle.pac_grad(w["h"], w["rho"], w["mu"], iv, K)
    e = check_grad(pac, gm, gr, ref, w["rho"], w["mu"], L, iv, K, N, N)
    print("\nN=%d L=%d K=%d: max group err %.2e, mu err %.2e" % (N, L, K, e[0], e[1]))


def test_pac_grad_vector_mu_and_target_range(ls):
    w = synth.make_workload("ls_n10000_l10000", N=150, L=400, seed=5)
    L, K = w["L"], 9
    mu = np.random.default_rng(3).uniform(1e-5, 1e-3, size=L)
    iv = synth.rho_intervals(L, K)
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], mu)
        rc, pac, gm, gr = ls.ls_pac_grad(ctx, iv, K, t_from=40, t_to=90)
    finally:
        ls.ls_destroy(ctx)
    ref = oracle.pac_grad(w["h"], w["rho"], mu, iv, K, targets=np.arange(40, 90))
    rpac, rgm, rgr = ref
    c = np.zeros(K)
    np.add.at(c, iv, w["rho"] / (1.0 - w["rho"]))
    cm = 50 * float(np.sum(mu / (1.0 - mu)))
    assert abs(pac - rpac) <= 1e-6 * abs(rpac) + 2e-7 * L * math.sqrt(50)
    assert abs(gm - rgm) <= G_RTOL * (abs(rgm) + cm)
    assert np.all(np.abs(gr - rgr) <= G_RTOL * (np.abs(rgr) + 50 * c))


def test_pac_grad_against_oracle_finite_differences(ls):
    """central differences (h = 1e-4) of the FP64 PAC log-likelihood in log mu and three
    interval log-scales, against the GPU adjoint."""
    w = synth.make_workload("ls_n10000_l10000", N=200, L=1000, seed=8)
    L, K = w["L"], 100
    iv = synth.rho_intervals(L, K)
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        _, pac, gm, gr = ls.ls_pac_grad(ctx, iv, K)
    finally:
        ls.ls_destroy(ctx)
    h = 1e-4

    def pac_at(dlmu=0.0, k=None, d=0.0):
        rho = w["rho"].copy()
        if k is not None:
            rho[iv == k] *= math.exp(d)
        return float(oracle.run(w["h"], rho, w["mu"] * math.exp(dlmu), [0], want=("llf",))["llf"].sum())

    fd_mu = (pac_at(dlmu=h) - pac_at(dlmu=-h)) / (2 * h)
    cr, cm = magnitudes(w["rho"], w["mu"], L, iv, K, 200)
    # FD truncation error O(h^2) and FP64 cancellation ~1e-16 |PAC| / h
    fd_tol = 1e-12 * abs(pac) / h
    assert abs(gm - fd_mu) <= G_RTOL * (abs(fd_mu) + cm) + fd_tol, (gm, fd_mu)
    for k in (0, 37, 99):
        fd = (pac_at(k=k, d=h) - pac_at(k=k, d=-h)) / (2 * h)
        assert abs(gr[k] - fd) <= G_RTOL * (abs(fd) + cr[k]) + fd_tol, (k, gr[k], fd)


def test_autograd_function_backward(ls):
    import torch
    from paper_2212_11403_gb300.autograd import pac_loglik
    w = synth.make_workload("ls_n10000_l10000", N=120, L=300, seed=12)
    L, K = w["L"], 10
    iv = synth.rho_intervals(L, K)
    ctx = ls.ls_create(w["h"])
    try:
        log_mu = torch.tensor(math.log(w["mu"]), dtype=torch.float64, requires_grad=True)
        delta = torch.zeros(K, dtype=torch.float64, requires_grad=True)
        out = pac_loglik(log_mu, delta, ctx, w["rho"], iv)
        (2.0 * out).backward()
    finally:
        ls.ls_destroy(ctx)
    rpac, rgm, rgr = oracle.pac_grad(w["h"], w["rho"], w["mu"], iv, K)
    cr, cm = magnitudes(w["rho"], w["mu"], L, iv, K, 120)
    assert abs(float(out.detach()) - rpac) <= 1e-6 * abs(rpac) + 2e-7 * L * math.sqrt(120)
    assert abs(float(log_mu.grad) - 2 * rgm) <= 2 * G_RTOL * (abs(rgm) + cm)
    assert np.all(np.abs(delta.grad.numpy() - 2 * rgr) <= 2 * G_RTOL * (np.abs(rgr) + cr))


def test_pac_grad_errors(ls):
    import torch
    w = synth.make_workload("ls_n10000_l10000", N=30, L=20, seed=2)
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        bad = synth.rho_intervals(20, 4)[::-1].copy()
        with pytest.raises(ls.LSError) as ei:
            ls.ls_pac_grad(ctx, bad, 4)  # decreasing interval map
        assert ei.value.code == ls.LS_ERR_ARG
        with pytest.raises(ls.LSError) as ei:
            ls.ls_pac_grad(ctx, synth.rho_intervals(20, 4), 3)  # index beyond K
        assert ei.value.code == ls.LS_ERR_ARG
        Pi = torch.full((30, 30), 1.0 / 29, dtype=torch.float32, device="cuda")
        Pi.fill_diagonal_(0.0)
        ls.ls_set_params(ctx, w["rho"], w["mu"], Pi)
        with pytest.raises(ls.LSError) as ei:
            ls.ls_pac_grad(ctx, synth.rho_intervals(20, 4), 4)
        assert ei.value.code == ls.LS_ERR_UNSUPPORTED
    finally:
        ls.ls_destroy(ctx)


def test_pac_grad_n10000_l10000_sampled_targets(ls):
    """Differentiation workload at its full size (N = L = 10000, K = 100): the adjoint over all
    targets runs to completion, and over a block of 16 targets it matches the oracle's gradient
    and finite differences of the oracle's PAC log-likelihood."""
    w = synth.make_workload("ls_n10000_l10000")
    N, L, K = w["N"], w["L"], 100
    iv = synth.rho_intervals(L, K)
    t0, t1 = 4000, 4016
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        rc, pac_all, gm_all, gr_all = ls.ls_pac_grad(ctx, iv, K)
        assert rc == 0 and math.isfinite(pac_all) and np.all(np.isfinite(gr_all)) and math.isfinite(gm_all)
        rc, pac, gm, gr = ls.ls_pac_grad(ctx, iv, K, t_from=t0, t_to=t1)
    finally:
        ls.ls_destroy(ctx)
    targets = np.arange(t0, t1)
    ref = oracle.pac_grad(w["h"], w["rho"], w["mu"], iv, K, targets=targets, nthreads=4)
    e = check_grad(pac, gm, gr, ref, w["rho"], w["mu"], L, iv, K, 16, N)
    print("\nN=L=10000 K=100 16 targets: max group err %.2e, mu err %.2e" % e)
    h = 1e-4

    def pac_at(dlmu=0.0, k=None, d=0.0):
        rho = w["rho"].copy()
        if k is not None:
            rho[iv == k] *= math.exp(d)
        r = oracle.run(w["h"], rho, w["mu"] * math.exp(dlmu), [0], targets=targets, want=("llf",))
        return float(r["llf"].sum())

    cr, cm = magnitudes(w["rho"], w["mu"], L, iv, K, 16)
    fd_tol = 1e-12 * abs(pac) / h
    fd_mu = (pac_at(dlmu=h) - pac_at(dlmu=-h)) / (2 * h)
    assert abs(gm - fd_mu) <= G_RTOL * (abs(fd_mu) + cm) + fd_tol, (gm, fd_mu)
    for k in (3, 71):
        fd = (pac_at(k=k, d=h) - pac_at(k=k, d=-h)) / (2 * h)
        assert abs(gr[k] - fd) <= G_RTOL * (abs(fd) + cr[k]) + fd_tol, (k, gr[k], fd)


def test_pac_grad_in_target_blocks_matches_one_block(ls):
    """the gradient's scratch ceiling (LS_GRAD_BUDGET_MB) splits the targets into blocks: with a
    ceiling that forces blocks of 13 targets the result matches the single-block run (each target's
    FP32 recursions may run in another launch configuration, so the sums agree to the gradient
    tolerance, not bit for bit) and the oracle."""
    import os
    N, L, K = 517, 200, 100
    w = synth.make_workload("ls_n10000_l10000", N=N, L=L, seed=77)
    iv = synth.rho_intervals(L, K)
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        rc0, pac0, gm0, gr0 = ls.ls_pac_grad(ctx, iv, K)
        os.environ["LS_GRAD_BUDGET_MB"] = "8"   # (3 x 100 + 2) x 517 x 4 bytes = 0.62 MB per target
        try:
            rc1, pac1, gm1, gr1 = ls.ls_pac_grad(ctx, iv, K)
        finally:
            del os.environ["LS_GRAD_BUDGET_MB"]
    finally:
        ls.ls_destroy(ctx)
    assert rc0 == rc1 == 0
    ref = oracle.pac_grad(w["h"], w["rho"], w["mu"], iv, K)
    check_grad(pac0, gm0, gr0, ref, w["rho"], w["mu"], L, iv, K, N, N)
    check_grad(pac1, gm1, gr1, ref, w["rho"], w["mu"], L, iv, K, N, N)
    cr, cm = magnitudes(w["rho"], w["mu"], L, iv, K, N)
    assert abs(pac1 - pac0) <= 1e-9 * abs(pac0)
    assert abs(gm1 - gm0) <= 1e-6 * (abs(gm0) + cm)
    assert np.all(np.abs(gr1 - gr0) <= 1e-6 * (np.abs(gr0) + cr))
