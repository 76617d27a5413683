"""Timings of the secondary workloads through the library (one JSON line each).

    python -m paper_2212_11403_gb300.measure prior   # N=20000, L=50000, Gamma(2,1) prior matrix, checkpoints
    python -m paper_2212_11403_gb300.measure grad    # N=L=10000, gradient over 100 rho intervals
    python -m paper_2212_11403_gb300.measure sparse  # learned sparse path against dense (N=20000) and at N=50000
    python -m paper_2212_11403_gb300.measure table   # ls_forward throughput against Delta-l (N=10000, N=100000)
    python -m paper_2212_11403_gb300.measure scaling # fused pipeline time against N and against L
    python -m paper_2212_11403_gb300.measure mlp     # the network's tensor-core scorer alone

CUDA events around each call on the current stream, after one warm-up call; inputs resident in
device memory.  These are measurements of the library only; the accuracy of each path against the
FP64 oracle is established by the GPU tests.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import ls, proposal, synth

P_FP32 = 2 * 128 * 152 * 2070e6  # FP32 FMA pipe, FLOP/s at the maximum SM clock
D_TRUST = float("inf")  # distance bound of the sparse path's trusted entries


def timed(fn, reps=1):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3


def measure_prior():
    import torch
    w = synth.make_workload("ls_n20000_l50000")
    N, L, loci = w["N"], w["L"], w["loci"]
    rho = ls.ls_calc_rho(w["gaps"], w["Ne"], 1.0)
    Pi = torch.from_numpy(synth.gamma_prior_f32(w["pi_seed"], N)).cuda()
    ctx = ls.ls_create(w["h"])
    out = []
    try:
        ls.ls_set_params(ctx, rho, w["mu"], Pi)
        d = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
        t = timed(lambda: ls.ls_run_all(ctx, loci, d, want_pac=False))
        cells = float(N) * N * L
        # matrix prior: 5 FLOP per cell and direction (one more multiply than the uniform prior)
        out.append(dict(workload="ls_n20000_l50000", path="dense fwd+bwd+distance, Gamma(2,1) prior matrix", D=len(loci),
                        seconds=t, cell_updates_per_s=cells / t, flop_per_cell=10,
                        frac_fp32=10 * cells / t / P_FP32))
        for dt, name in ((ls.LS_CKPT_F32, "f32"), (ls.LS_CKPT_F16, "f16")):
            fw = ls.ls_table_create(ctx, ls.LS_FWD, 0, N)
            box = {}

            def run():
                ls.ls_table_reset(fw)
                if "ck" in box:
                    ls.ls_ckpt_destroy(box.pop("ck"))
                box["ck"] = ls.ls_checkpoints(ctx, fw, 0, L - 1, dt)
            t = timed(run)
            info = ls.ls_ckpt_info(box["ck"])
            # replay to the middle of the widest gap between snapshots
            probe = (int(info["loci"][0]) + int(info["loci"][1])) // 2
            fw2 = ls.ls_table_create(ctx, ls.LS_FWD, 0, N)
            tr = timed(lambda: ls.ls_ckpt_replay(ctx, box["ck"], fw2, probe))
            out.append(dict(workload="ls_n20000_l50000", path="forward with %d %s checkpoints" % (info["n"], name),
                            seconds=t, checkpoint_bytes=info["device_bytes"], replay_to_locus=probe,
                            replay_seconds=tr, cell_updates_per_s=float(N) * N * L / t))
            ls.ls_ckpt_destroy(box["ck"])
            ls.ls_table_destroy(fw)
            ls.ls_table_destroy(fw2)
    finally:
        ls.ls_destroy(ctx)
    return out


def measure_prior_bf16():
    """A prior matrix in the BF16 format: the register-tile kernel at N = 20000 (FP32 and BF16
    formats) and the large-N kernels at N = 50000 (one CTA per target) and N = 100000 (clusters of
    two), fused fwd + bwd + distance at one decode locus over a short stretch of the cfg3 map
    (L = 400 for timing; the per-locus cost does not depend on L)."""
    import torch
    out = []
    for N, fmt in ((20000, ls.LS_PRIOR_FP32), (20000, ls.LS_PRIOR_BF16), (50000, ls.LS_PRIOR_BF16),
                   (100000, ls.LS_PRIOR_BF16)):
        L = 400
        w = synth.make_workload("ls_n50000_l20000", N=N, L=L, seed=77 + N, founders=N // 25)
        loci = np.array([L // 2], dtype=np.int32)
        Pi = synth.gamma_prior_torch(N + 1, N)
        ctx = ls.ls_create(w["h"])
        try:
            ls.ls_set_prior_format(ctx, fmt)
            ls.ls_set_params(ctx, w["rho"], w["mu"], Pi)
            del Pi
            torch.cuda.empty_cache()
            d = torch.empty((1, N, N), dtype=torch.float32, device="cuda")
            t = timed(lambda: ls.ls_run_all(ctx, loci, d, want_pac=False), reps=2)
            del d
        finally:
            ls.ls_destroy(ctx)
        cells = float(N) * N * L
        out.append(dict(workload="ls_n50000_l20000 generator with a Gamma(2,1) prior matrix", N=N, L=L, D=1,
                        prior_format="bf16" if fmt == ls.LS_PRIOR_BF16 else "fp32",
                        path="dense fwd+bwd+distance, prior matrix", seconds=t, cell_updates_per_s=cells / t,
                        flop_per_cell=10, frac_fp32=10 * cells / t / P_FP32))
        torch.cuda.empty_cache()
    return out


def measure_grad():
    import torch
    w = synth.make_workload("ls_n10000_l10000")
    N, L, K = w["N"], w["L"], 100
    iv = synth.rho_intervals(L, K)
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        tg = timed(lambda: ls.ls_pac_grad(ctx, iv, K))
        d = torch.empty((1, N, N), dtype=torch.float32, device="cuda")
        tp = timed(lambda: ls.ls_run_all(ctx, np.array([L // 2], dtype=np.int32), d, want_pac=True))
    finally:
        ls.ls_destroy(ctx)
    cells = float(N) * N * L
    return [dict(workload="ls_n10000_l10000", path="PAC log-likelihood + gradient (log mu, 100 log rho groups)",
                 seconds=tg, cell_updates_per_s=cells / tg, plain_fwd_bwd_seconds=tp, ratio_to_plain=tg / tp)]


def error_stats(ds, dd, tm, N, rows=2048):
    """trusted fraction and, against dense, |d_sparse - d_dense| over trusted entries and over the
    estimated ones, in row blocks (bounded memory at N = 50000)."""
    import torch
    n_tr = n_all = n_le = 0
    mx = 0.0
    smp, smp_est = [], []
    g = torch.Generator(device=ds.device).manual_seed(11)
    for k in range(ds.shape[0]):
        for r0 in range(0, N, rows):
            r1 = min(N, r0 + rows)
            tr = ls.trust_bits(tm[k:k + 1, r0:r1], N)[0]
            n_tr += int(tr.sum())
            n_all += (r1 - r0) * N
            if dd is None:
                continue
            e = (ds[k, r0:r1] - dd[k, r0:r1]).abs()
            et = e[tr]
            if et.numel():
                mx = max(mx, float(et.max()))
                n_le += int((et <= 1e-3).sum())
                smp.append(et[torch.randint(et.numel(), (min(et.numel(), 20000),), device=e.device, generator=g)])
            est = e[~tr]
            smp_est.append(est[torch.randint(est.numel(), (20000,), device=e.device, generator=g)])
    out = dict(trusted=n_tr / n_all)
    if dd is not None and smp:
        q = torch.quantile(torch.cat(smp), torch.tensor([0.5, 0.9, 0.99], device=ds.device)).tolist()
        qe = torch.quantile(torch.cat(smp_est), torch.tensor([0.5, 0.9], device=ds.device)).tolist()
        out.update(dd_q50=q[0], dd_q90=q[1], dd_q99=q[2], dd_max=mx, frac_within_1e3=n_le / max(n_tr, 1),
                   estimated_dd_q50=qe[0], estimated_dd_q90=qe[1])
    return out


def measure_sparse():
    import torch
    out = []
    C, K = 1024, 512
    # training on dense posteriors of an N = 5000 instance of the same generator (founders N/25)
    Nt, Lt = 5000, 20000
    wt = synth.make_workload("ls_n50000_l20000", N=Nt, L=Lt, seed=5001, founders=Nt // 25)
    ctx = ls.ls_create(wt["h"])
    wins = list(range(0, (Lt + 255) // 256, 8))
    t0 = time.time()
    try:
        ls.ls_set_params(ctx, wt["rho"], wt["mu"])
        X, y = proposal.training_set(ctx, Nt, Lt, C, wins)
    finally:
        ls.ls_destroy(ctx)
    net, loss = proposal.train(X, y, steps=1500, batch=16384, lr=1e-3, seed=3)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    del X, y
    for N, with_dense in ((20000, True), (50000, True)):
        w = synth.make_workload("ls_n50000_l20000", N=N, seed=6000 + N, founders=N // 25)
        L = w["L"]
        loci = synth.decode_loci(L, 4)
        Wn = (L + 255) // 256
        ctx = ls.ls_create(w["h"])
        try:
            ls.ls_set_params(ctx, w["rho"], w["mu"])
            rec = dict(workload="ls_n50000_l20000 generator at N=%d" % N, N=N, L=L, D=4, K=K, C=C,
                       train_seconds=t_train, train_loss=loss)
            idx = torch.empty((N, Wn, K), dtype=torch.int32, device="cuda")
            ds = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
            tm = torch.empty((len(loci), N, (N + 31) // 32), dtype=torch.int32, device="cuda")
            for name, m in (("raw", None), ("mlp", net)):
                tp = timed(lambda: ls.ls_propose(ctx, C, K, m, idx))
                ts = timed(lambda: ls.ls_sparse_run_all(ctx, idx, K, 256, loci, ds, d_trust=D_TRUST, trust_out=tm))
                rec[name] = dict(propose_seconds=tp, sparse_seconds=ts, total_seconds=tp + ts, d_trust=D_TRUST)
                if with_dense and "dense_seconds" not in rec:
                    dd = torch.empty_like(ds)
                    rec["dense_seconds"] = timed(lambda: ls.ls_run_all(ctx, loci, dd, want_pac=False))
                rec[name].update(error_stats(ds, dd if with_dense else None, tm, N))
                if with_dense:
                    rec[name]["speedup"] = rec["dense_seconds"] / (tp + ts)
            out.append(rec)
            del ds
            if with_dense:
                del dd
        finally:
            ls.ls_destroy(ctx)
    ls.ls_mlp_destroy(net)
    return out


def measure_sparse_case(N, L, K=512):
    """one sparse forward + backward + distance (raw sets, D = 4) on the N = 50000 generator at a
    smaller size: the profiling case of the sparse kernels."""
    import torch
    w = synth.make_workload("ls_n50000_l20000", N=N, L=L, seed=6000 + N, founders=N // 25)
    loci = synth.decode_loci(L, 4)
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        idx = torch.empty((N, (L + 255) // 256, K), dtype=torch.int32, device="cuda")
        ls.ls_propose(ctx, K, K, None, idx)
        ds = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
        t = timed(lambda: ls.ls_sparse_run_all(ctx, idx, K, 256, loci, ds))
    finally:
        ls.ls_destroy(ctx)
    return [dict(workload="ls_n50000_l20000 generator at N=%d L=%d" % (N, L), path="sparse, raw sets", K=K,
                 seconds=t)]


def measure_table(big_L=10000):
    """The paper's single-step table API at scale (Sec. 5, the Delta-L figures): ls_forward of a
    table over all N targets by Delta-l loci, throughput N^2 Delta-l / t, at N = 10000 (L = 10000)
    for Delta-l from 1 to 9999; then one forward of a 100000 x 100000 table over big_L loci."""
    import torch
    out = []
    w = synth.make_workload("ls_n10000_l10000")
    N, L = w["N"], w["L"]
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        fw = ls.ls_table_create(ctx, ls.LS_FWD, 0, N)
        for dl in (1, 2, 4, 16, 64, 256, 1024, 4096, L - 1):
            def run():
                ls.ls_table_reset(fw)
                ls.ls_forward(ctx, fw, 0)       # initialise at locus 0 (outside the timed call)
            run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ls.ls_forward(ctx, fw, dl)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            cells = float(N) * N * dl
            out.append(dict(workload="ls_n10000_l10000", path="ls_forward over Delta-l loci, table of all targets",
                            N=N, delta_l=dl, seconds=t, cell_updates_per_s=cells / t,
                            frac_fp32=4 * cells / t / P_FP32))
        ls.ls_table_destroy(fw)
    finally:
        ls.ls_destroy(ctx)
    N = 100000
    w = synth.make_workload("ls_n50000_l20000", N=N, L=big_L, seed=7100, founders=N // 25)
    ctx = ls.ls_create(w["h"])
    try:
        ls.ls_set_params(ctx, w["rho"], w["mu"])
        fw = ls.ls_table_create(ctx, ls.LS_FWD, 0, N)
        for dl in (1, 16, 256, big_L - 1):
            ls.ls_table_reset(fw)
            ls.ls_forward(ctx, fw, 0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ls.ls_forward(ctx, fw, dl)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            cells = float(N) * N * dl
            out.append(dict(workload="ls_n50000_l20000 generator at N=100000, L=%d" % big_L,
                            path="ls_forward over Delta-l loci, 100000 x 100000 FP32 table (40 GB)", N=N,
                            delta_l=dl, seconds=t, cell_updates_per_s=cells / t, frac_fp32=4 * cells / t / P_FP32))
        ls.ls_table_destroy(fw)
    finally:
        ls.ls_destroy(ctx)
    return out


def measure_scaling():
    """The paper's scaling experiment (Sec. 5, fig:perfscaling: cost against N and against L) on
    the dense fused pipeline: time of ls_run_all (forward + backward + distance at 4 loci) over a
    grid of N at L = 4000 and of L at N = 5000, on the bench workload's generator."""
    import torch
    out = []
    grid = [(N, 4000) for N in (500, 1000, 2000, 5000, 10000, 20000)] + [(5000, L) for L in (500, 1000, 2000, 8000, 16000)]
    for N, L in grid:
        w = synth.make_workload("ls_n5000_l20000", N=N, L=L, seed=3000 + N + L)
        loci = synth.decode_loci(L, 4)
        ctx = ls.ls_create(w["h"])
        try:
            ls.ls_set_params(ctx, w["rho"], w["mu"])
            d = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
            t = timed(lambda: ls.ls_run_all(ctx, loci, d, want_pac=False), reps=2)
        finally:
            ls.ls_destroy(ctx)
        cells = float(N) * N * L
        out.append(dict(workload="ls_n5000_l20000 generator", path="dense fwd+bwd+distance, D = 4", N=N, L=L,
                        seconds=t, cell_updates_per_s=cells / t, frac_fp32=8 * cells / t / P_FP32))
    return out


def measure_mlp(n=1 << 25):
    """The proposal network's tensor-core scorer alone: ls_mlp_forward on n random feature rows
    (the call converts the rows to BF16 first, inside the timed region)."""
    import torch
    rng = np.random.default_rng(1)
    p = (rng.normal(0, 1, ls.LS_MLP_PARAMS) * 0.1).astype(np.float32)
    m = ls.ls_mlp_create(p)
    try:
        X = torch.rand((n, 8), device="cuda")
        X[:, 7] = 0
        s = torch.empty(n, device="cuda")
        t = timed(lambda: ls.ls_mlp_forward(m, X, s), reps=3)
    finally:
        ls.ls_mlp_destroy(m)
    flop = 2.0 * n * (7 * 256 + 256 * 256 + 256)
    return [dict(path="ls_mlp_forward (BF16 tcgen05 scorer)", rows=n, seconds=t, rows_per_s=n / t,
                 tflops=flop / t / 1e12)]


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["prior", "prior_bf16", "grad", "sparse", "sparse_case", "table", "scaling", "mlp"])
    ap.add_argument("--N", type=int, default=20000, help="sparse_case: haplotypes")
    ap.add_argument("--L", type=int, default=2000, help="sparse_case: loci")
    ap.add_argument("--rows", type=int, default=1 << 25, help="mlp: feature rows")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    if a.what == "sparse_case":
        recs = measure_sparse_case(a.N, a.L)
    elif a.what == "mlp":
        recs = measure_mlp(a.rows)
    else:
        recs = dict(prior=measure_prior, prior_bf16=measure_prior_bf16, grad=measure_grad, sparse=measure_sparse, table=measure_table,
                    scaling=measure_scaling)[a.what]()
    for rec in recs:
        print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main()
