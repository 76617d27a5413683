"""ls_run_all_noalloc, the allocation-free pipeline, checked against ls_run_all through the C ABI.

The allocation-free entry point is for callers that must not allocate device memory while they
run the pipeline (code captured into a CUDA graph, code inside a fixed device-memory budget,
loops where cudaMalloc's implicit synchronisation is unacceptable).  Its scratch is one fixed area
inside the library that every call reuses, so the checks here run it twice in a row on the same
inputs and then on a different context, and compare each result with ls_run_all.  Both entry
points plan their launches with the same planner and so run the same kernels on the same targets:
distances and status words must be bit-identical (the PAC sums are taken in different orders, so
they are held to the log tolerance).  N = 5000 gives a two-launch plan (full waves plus a tail).

This file is named so that pytest collects it last: a run that stops at its first failure has
then already run every other test.
"""
import math

import numpy as np
import pytest

from paper_2212_11403_gb300 import synth

pytestmark = pytest.mark.gpu

D_TOL = 1e-5


def d_err(dg, dr):
    """per-entry error of distances: max over entries of |d_gpu - d_ref| / max(|d_ref|, 1)."""
    dg = np.asarray(dg, dtype=np.float64)
    dr = np.asarray(dr, dtype=np.float64)
    return float(np.max(np.abs(dg - dr) / np.maximum(np.abs(dr), 1.0)))


def pac_close(a, b, L, N):
    return abs(a - b) <= 1e-6 * abs(b) + 2e-7 * L * math.sqrt(N)


@pytest.fixture(scope="module")
def ls():
    import torch
    torch.cuda.set_device(0)
    from paper_2212_11403_gb300 import ls as _ls
    return _ls


def reference(ls, ctx, loci, N):
    import torch
    d = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
    st = torch.zeros(N, dtype=torch.int32, device="cuda")
    rc, pac = ls.ls_run_all(ctx, loci, d, status_out=st)
    torch.cuda.synchronize()
    return rc, pac, d.cpu().numpy(), st.cpu().numpy()


def noalloc(ls, ctx, loci, N):
    import torch
    d = torch.full((len(loci), N, N), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    rc, pac = ls.ls_run_all_noalloc(ctx, loci, d, status_out=st)
    torch.cuda.synchronize()
    return rc, pac, d.cpu().numpy(), st.cpu().numpy()


def test_noalloc_matches_run_all_on_repeated_calls(ls):
    w = synth.make_workload("ls_n200_l1000", N=300, L=400, seed=31)
    v = synth.make_workload("ls_n5000_l20000", N=517, L=300, seed=32)
    u = synth.make_workload("ls_n5000_l20000", N=5000, L=120, seed=33)
    contexts = []
    try:
        for wk in (w, v, u):
            ctx = ls.ls_create(wk["h"])
            contexts.append(ctx)
            ls.ls_set_params(ctx, wk["rho"], wk["mu"])
        runs = [(contexts[0], w), (contexts[0], w), (contexts[1], v), (contexts[2], u), (contexts[2], u),
                (contexts[0], w)]
        for ctx, wk in runs:
            N, L, loci = wk["N"], wk["L"], wk["loci"]
            rc0, pac0, d0, st0 = reference(ls, ctx, loci, N)
            rc1, pac1, d1, st1 = noalloc(ls, ctx, loci, N)
            assert rc1 == rc0
            assert not np.isnan(d1).any()
            assert d_err(d1, d0) <= D_TOL
            np.testing.assert_array_equal(d1, d0)
            assert pac_close(pac1, pac0, L, N), (pac1, pac0)
            np.testing.assert_array_equal(st1, st0)
    finally:
        for ctx in contexts:
            ls.ls_destroy(ctx)


@pytest.mark.parametrize("fmt", ["fp32", "bf16"])
def test_noalloc_matches_run_all_with_a_prior_matrix(ls, fmt):
    """the prior-matrix variants (FP32 or bfloat16 prior values in shared memory), planned by the
    same planner: bit-identical distances and status words"""
    import torch
    wk = synth.make_workload("ls_n5000_l20000", N=700, L=150, seed=34)
    N, L, loci = wk["N"], wk["L"], wk["loci"]
    Pi = torch.from_numpy(synth.gamma_prior_f32(35, N)).cuda()
    ctx = ls.ls_create(wk["h"])
    try:
        if fmt == "bf16":
            ls.ls_set_prior_format(ctx, ls.LS_PRIOR_BF16)
        ls.ls_set_params(ctx, wk["rho"], wk["mu"], Pi)
        rc0, pac0, d0, st0 = reference(ls, ctx, loci, N)
        rc1, pac1, d1, st1 = noalloc(ls, ctx, loci, N)
    finally:
        ls.ls_destroy(ctx)
    assert rc1 == rc0 == 0
    np.testing.assert_array_equal(d1, d0)
    np.testing.assert_array_equal(st1, st0)
    assert pac_close(pac1, pac0, L, N), (pac1, pac0)


def test_noalloc_rejects_n_beyond_its_scratch(ls):
    import torch
    N = ls.LS_NOALLOC_MAX_N + 1
    h = np.zeros((2, N), dtype=np.uint8)
    h[:, ::3] = 1
    ctx = ls.ls_create(h)
    try:
        ls.ls_set_params(ctx, np.array([0.01]), 1e-3)
        tiny = torch.empty(1, dtype=torch.float32, device="cuda")
        with pytest.raises(ls.LSError) as ei:
            ls.ls_run_all_noalloc(ctx, np.array([0], dtype=np.int32), tiny)
        assert ei.value.code == ls.LS_ERR_UNSUPPORTED
        assert "LS_NOALLOC_MAX_N" in str(ei.value)
    finally:
        ls.ls_destroy(ctx)
