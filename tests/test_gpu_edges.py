"""Edge cases of the method through ls_run_all, against the FP64 oracle (pytest -m gpu).

The oracle pins these cases on the CPU (closed forms for rho = 0 and rho = 1, identical donors,
per-locus mu); here the CUDA path must reproduce the oracle on them.  Distances are held to the
per-entry bound max |d_gpu - d_ref| / max(|d_ref|, 1) <= 1e-5 on every entry (all targets, or all
entries among sampled targets at the largest N), log-likelihoods as in test_gpu_parity.py.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2212_11403_gb300 import synth

pytestmark = pytest.mark.gpu

D_TOL = 1e-5


def d_err(dg, dr):
    dg = np.asarray(dg, dtype=np.float64)
    dr = np.asarray(dr, dtype=np.float64)
    return float(np.max(np.abs(dg - dr) / np.maximum(np.abs(dr), 1.0)))


def log_close(got, ref, L, n=1):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return bool(np.all(np.abs(got - ref) <= 1e-6 * np.abs(ref) + 2e-7 * L * math.sqrt(n)))


@pytest.fixture(scope="module")
def ls():
    import torch
    torch.cuda.set_device(0)
    from paper_2212_11403_gb300 import ls as _ls
    return _ls


def run_all(ls, h, rho, mu, loci):
    import torch
    L, N = h.shape
    ctx = ls.ls_create(h)
    try:
        ls.ls_set_params(ctx, rho, mu)
        d = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
        st = torch.zeros(N, dtype=torch.int32, device="cuda")
        rc, pac = ls.ls_run_all(ctx, loci, d, status_out=st)
        torch.cuda.synchronize()
        return rc, pac, d.cpu().numpy(), st.cpu().numpy()
    finally:
        ls.ls_destroy(ctx)


def check_all_entries(ls, h, rho, mu, loci):
    L, N = h.shape
    rc, pac, d, st = run_all(ls, h, rho, mu, loci)
    assert rc == 0 and not st.any()
    ref = oracle.run(h, rho, mu, loci, want=("post", "llf"), nthreads=0)
    errs = []
    for k in range(len(loci)):
        dref = oracle.distance_block(ref["post"][:, k, :], np.arange(N))
        errs.append(d_err(d[k], dref))
        assert np.all(np.diag(d[k]) == 0.0)
    assert max(errs) <= D_TOL, errs
    assert log_close(pac, ref["llf"].sum(), L, N), (pac, ref["llf"].sum())
    return d, ref


@pytest.mark.parametrize("kind", ["one", "mixed"])
def test_rho_edge_values(ls, kind):
    """rho = 1 everywhere (independent loci) and a mix of 0, 1 and ordinary values, on a
    founder-mosaic panel."""
    w = synth.make_workload("ls_n200_l1000", N=150, L=240, seed=61)
    rng = np.random.default_rng(62)
    rho = {"one": np.ones(w["L"] - 1), "mixed": rng.choice([0.0, 1.0, 0.3, 1e-3, 0.02], size=w["L"] - 1)}[kind]
    check_all_entries(ls, w["h"], rho, w["mu"], np.array([0, 77, 160, 239], dtype=np.int32))


def test_rho_zero_within_fp32_range(ls):
    """rho = 0 everywhere: no recombination, so every target copies one donor throughout and the
    posterior is the same at every locus.  Without the recombination floor a donor's scaled alpha
    (or beta) is the mismatch ratio mu/(1-mu) to the power of its extra mismatches on the prefix
    (suffix); FP32 represents that only while the power stays above about 1e-38.  With mu = 0.05 and
    L = 16 every such power is above 19^-16 = 3e-21, so the FP32 path must match the oracle on every
    entry.  (Longer panels at small mu leave FP32's range: the copied donor's alpha flushes to 0.)"""
    w = synth.make_workload("ls_n200_l1000", N=150, L=16, seed=61)
    check_all_entries(ls, w["h"], np.zeros(15), 0.05, np.array([0, 7, 15], dtype=np.int32))


def test_paper_default_mu(ls):
    """mu = 1e-8, the paper's default (Sec. 3.3): 1 - mu rounds to 1 in FP32."""
    w = synth.make_workload("ls_n200_l1000", N=140, L=300, seed=63)
    check_all_entries(ls, w["h"], w["rho"], 1e-8, np.array([0, 150, 299], dtype=np.int32))


def test_per_locus_mu(ls):
    """mu given per locus (Table tab:pars: a vector of length L), through the fused pipeline."""
    w = synth.make_workload("ls_n200_l1000", N=160, L=260, seed=64)
    mu = np.random.default_rng(65).uniform(1e-6, 2e-2, size=w["L"])
    check_all_entries(ls, w["h"], w["rho"], mu, np.array([3, 100, 259], dtype=np.int32))


def test_identical_donors(ls):
    """three identical haplotypes: every other target copies them with equal posterior, so their
    distance columns agree, and the GPU path matches the oracle on all entries."""
    w = synth.make_workload("ls_n200_l1000", N=120, L=200, seed=66)
    h = w["h"].copy()
    h[:, 41] = h[:, 40]
    h[:, 42] = h[:, 40]
    d, ref = check_all_entries(ls, h, w["rho"], w["mu"], np.array([0, 99, 199], dtype=np.int32))
    others = [i for i in range(120) if i not in (40, 41, 42)]
    for k in range(3):
        np.testing.assert_allclose(d[k][others, 41], d[k][others, 40], rtol=2e-6, atol=2e-6)
        np.testing.assert_allclose(d[k][others, 42], d[k][others, 40], rtol=2e-6, atol=2e-6)


@pytest.mark.parametrize("N", [20480, 40960, 40961, 57344])
def test_planner_boundaries_sampled(ls, N):
    """N at the boundaries between kernel families (the largest register-tile N, the last N of the
    first shared-memory group, the first of the second, the largest N served): all entries among
    16 sampled targets against the oracle."""
    import torch
    L = 32
    w = synth.make_workload("ls_n50000_l20000", N=N, L=L, seed=700 + N % 89, founders=N // 25)
    loci = np.array([0, 17, L - 1], dtype=np.int32)
    targets = np.sort(np.random.default_rng(N + 1).choice(N, size=16, replace=False))
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        d = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
        rc, pac = ls.ls_run_all(ctx, loci, d)
        ti = torch.from_numpy(targets.astype(np.int64)).cuda()
        sub = d[:, ti][:, :, ti].cpu().numpy()
        del d
        torch.cuda.synchronize()
    finally:
        ls.ls_destroy(ctx)
    assert rc == 0
    ref = oracle.run(w["h"], w["rho"], w["mu"], loci, targets=targets, want=("post", "llf"))
    for k in range(len(loci)):
        dref = oracle.distance_block(ref["post"][:, k, :], targets)
        assert d_err(sub[k], dref) <= D_TOL, (N, k, d_err(sub[k], dref))


@pytest.mark.parametrize("N", [57345, 100000, 114688])
def test_cluster_kernel_run_all_sampled(ls, N):
    """N beyond one CTA's registers and shared memory: each target is split over a cluster of two
    CTAs (distributed shared memory for the per-locus sum).  The fused pipeline at one decode
    locus (an N x N float matrix: up to 52 GB), all entries among 16 sampled targets against the
    oracle, and the PAC log-likelihood against the forward tables' log F."""
    import torch
    L = 16
    w = synth.make_workload("ls_n50000_l20000", N=N, L=L, seed=800 + N % 83, founders=N // 25)
    loci = np.array([9], dtype=np.int32)
    targets = np.sort(np.random.default_rng(N + 2).choice(N, size=16, replace=False))
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        d = torch.empty((1, N, N), dtype=torch.float32, device="cuda")
        rc, pac = ls.ls_run_all(ctx, loci, d)
        ti = torch.from_numpy(targets.astype(np.int64)).cuda()
        sub = d[:, ti][:, :, ti].cpu().numpy()
        del d
        torch.cuda.synchronize()
    finally:
        ls.ls_destroy(ctx)
    assert rc == 0
    ref = oracle.run(w["h"], w["rho"], w["mu"], loci, targets=targets, want=("post", "llf"))
    dref = oracle.distance_block(ref["post"][:, 0, :], targets)
    assert d_err(sub[0], dref) <= D_TOL, (N, d_err(sub[0], dref))


def test_n100000_tables_sampled(ls):
    """the paper's large-table regime (Sec. 5: a 100000 x 100000 forward table): forward and
    backward tables of 64 targets at N = 100000 moved to a middle locus, posterior rows against the
    oracle's, log F and log G against the oracle's, distances among the 64 targets."""
    import torch
    N, L, t0, T = 100000, 24, 31000, 64
    w = synth.make_workload("ls_n50000_l20000", N=N, L=L, seed=801, founders=N // 25)
    l = 11
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        fw = ls.ls_table_create(ctx, ls.LS_FWD, t0, t0 + T)
        bw = ls.ls_table_create(ctx, ls.LS_BWD, t0, t0 + T)
        ls.ls_forward(ctx, fw, 5)
        ls.ls_forward(ctx, fw, l)       # resumed: the state goes through the table
        ls.ls_backward(ctx, bw, l)
        P = torch.empty((T, N), dtype=torch.float32, device="cuda")
        ls.ls_posterior(ctx, fw, bw, P)
        lf = torch.empty(T, dtype=torch.float64, device="cuda")
        lg = torch.empty(T, dtype=torch.float64, device="cuda")
        ls.ls_table_read(fw, logscale=lf)
        ls.ls_table_read(bw, logscale=lg)
        torch.cuda.synchronize()
        P, lf, lg = P.cpu().numpy().astype(np.float64), lf.cpu().numpy(), lg.cpu().numpy()
        ls.ls_table_destroy(fw)
        ls.ls_table_destroy(bw)
    finally:
        ls.ls_destroy(ctx)
    targets = np.arange(t0, t0 + T)
    ref = oracle.run(w["h"], w["rho"], w["mu"], [l], targets=targets, want=("post", "logF", "logG"))
    rp = ref["post"][:, 0, :]
    m = rp > 1e-12
    assert float(np.max(np.abs(P[m] - rp[m]) / rp[m])) <= 2e-4
    assert log_close(lf, ref["logF"][:, 0], l + 1)
    assert log_close(lg, ref["logG"][:, 0], L - l)
    dg = oracle.distance_block(P, targets)
    dref = oracle.distance_block(rp, targets)
    assert d_err(dg, dref) <= D_TOL
