"""Seeded synthetic workloads for the LS all-vs-all path.

This module only draws random inputs; it contains none of the method's arithmetic (no emission,
recursion or rho-from-map conversion).  Both the CUDA path and the FP64 oracle consume its
output, so it is the one piece of code the two sides share.

Haplotypes are founder mosaics: F founder haplotypes are drawn with a per-variant allele
frequency p_l ~ U(0.01, 0.5); each of the N haplotypes starts on a uniformly chosen founder and
at every variant switches, with probability `switch`, to a uniformly chosen *other* founder;
finally every allele flips with probability `flip`.  Seeds are 1000 + the workload number.
"""
from __future__ import annotations

import numpy as np

# Workloads: the five synthetic configurations the benchmark and the parity tests use.
WORKLOADS = {
    # plain LS, full oracle parity: N=200, L=1000, d at 10 evenly spaced loci
    "ls_n200_l1000": dict(num=1, N=200, L=1000, founders=20, switch=0.01, flip=1e-3, rho="uniform",
                          rho_lo=1e-4, rho_hi=1e-2, mu=1e-4, Pi="uniform", D=10),
    # dense FP32 LS: N=5000, L=20000, d at 16 loci
    "ls_n5000_l20000": dict(num=2, N=5000, L=20000, founders=200, switch=5e-3, flip=5e-4, rho="loguniform",
                            rho_lo=1e-5, rho_hi=1e-2, mu=1e-5, Pi="uniform", D=16),
    # dense LS at scale with checkpoints and a Gamma(2,1) prior matrix
    "ls_n20000_l50000": dict(num=3, N=20000, L=50000, founders=1000, switch=2e-3, flip=5e-4, rho="map",
                             gap_mean=1e-4, Ne_tilde=1e4, mu=1e-6, Pi="gamma", D=16),
    # differentiation workload (config-2 generator at N=L=10000)
    "ls_n10000_l10000": dict(num=4, N=10000, L=10000, founders=200, switch=5e-3, flip=5e-4, rho="loguniform",
                             rho_lo=1e-5, rho_hi=1e-2, mu=1e-5, Pi="uniform", D=16, K=100),
    # learned donor proposal workload
    "ls_n50000_l20000": dict(num=5, N=50000, L=20000, founders=2000, switch=1e-3, flip=1e-4, rho="loguniform",
                             rho_lo=1e-5, rho_hi=1e-2, mu=1e-5, Pi="uniform", D=16),
}


def mosaic_haplotypes(rng: np.random.Generator, N: int, L: int, founders: int, switch: float, flip: float,
                      chunk: int = 512) -> np.ndarray:
    """uint8 [L, N] founder-mosaic haplotypes (variant-major, 0/1)."""
    F = founders
    af = rng.uniform(0.01, 0.5, size=L)
    h = np.empty((L, N), dtype=np.uint8)
    cur = rng.integers(0, F, size=N)
    for l0 in range(0, L, chunk):
        l1 = min(L, l0 + chunk)
        fnd = (rng.random((l1 - l0, F)) < af[l0:l1, None]).astype(np.uint8)
        for l in range(l0, l1):
            if l > 0:
                sw = rng.random(N) < switch
                if F > 1 and sw.any():
                    k = int(sw.sum())
                    cur[sw] = (cur[sw] + rng.integers(1, F, size=k)) % F
            row = fnd[l - l0, cur]
            fl = rng.random(N) < flip
            h[l] = row ^ fl.astype(np.uint8)
    return h


def decode_loci(L: int, D: int) -> np.ndarray:
    """D evenly spaced 0-based loci including both ends: floor(k (L-1) / (D-1))."""
    if D == 1:
        return np.array([0], dtype=np.int32)
    return np.array([(k * (L - 1)) // (D - 1) for k in range(D)], dtype=np.int32)


def rho_intervals(L: int, K: int) -> np.ndarray:
    """interval index k of each of the L-1 inter-locus gaps, K equal-width intervals."""
    m = np.arange(L - 1, dtype=np.int64)
    return np.minimum((m * K) // max(L - 1, 1), K - 1).astype(np.int32)


def gamma_prior(rng: np.random.Generator, N: int, rows=None) -> np.ndarray:
    """float64 [len(rows), N] prior rows: entries ~ Gamma(2, 1) off the diagonal, diagonal 0, each
    recipient row normalised to sum 1 (recipient-major: row i = recipient i)."""
    rows = np.arange(N) if rows is None else np.asarray(rows)
    out = rng.gamma(2.0, 1.0, size=(len(rows), N))
    out[np.arange(len(rows)), rows] = 0.0
    out /= out.sum(axis=1, keepdims=True)
    return out


def gamma_prior_f32(seed: int, N: int, chunk: int = 1024) -> np.ndarray:
    """float32 [N, N] prior matrix of the Gamma(2, 1) workloads, drawn and normalised in float64
    chunks of recipient rows (bounded host memory at N = 20000), then rounded to float32."""
    rng = np.random.default_rng(seed)
    out = np.empty((N, N), dtype=np.float32)
    for r0 in range(0, N, chunk):
        rows = np.arange(r0, min(N, r0 + chunk))
        out[rows] = gamma_prior(rng, N, rows).astype(np.float32)
    return out


def gamma_prior_torch(seed: int, N: int, device="cuda", chunk: int = 1024):
    """float32 [N, N] torch tensor on `device`: the Gamma(2, 1) prior of gamma_prior (each entry the
    sum of two unit exponentials, diagonal 0, rows normalised in float64), drawn by torch's
    generator on the device, for N too large for a host matrix.  Rows of it for an oracle are
    copied back from the tensor."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = torch.empty((N, N), dtype=torch.float32, device=device)
    for r0 in range(0, N, chunk):
        r1 = min(N, r0 + chunk)
        x = torch.empty((r1 - r0, N), dtype=torch.float64, device=device).exponential_(generator=g)
        x += torch.empty((r1 - r0, N), dtype=torch.float64, device=device).exponential_(generator=g)
        idx = torch.arange(r0, r1, device=device)
        x[idx - r0, idx] = 0.0
        x /= x.sum(dim=1, keepdim=True)
        out[r0:r1] = x.to(torch.float32)
    return out


def make_workload(name: str, N: int | None = None, L: int | None = None, seed: int | None = None,
                  founders: int | None = None) -> dict:
    """Draw the inputs of a workload (optionally shrunk to N x L for tests).

    Returns dict(h uint8 [L, N], rho float64 [L-1] or None, gaps float64 [L-1] (Morgans) and
    Ne for map-based workloads, mu float, Pi None or 'gamma', loci int32 [D], name, N, L).
    """
    cfg = dict(WORKLOADS[name])
    N = int(cfg["N"] if N is None else N)
    L = int(cfg["L"] if L is None else L)
    seed = 1000 + cfg["num"] if seed is None else seed
    rng = np.random.default_rng(seed)
    F = min(cfg["founders"] if founders is None else founders, N)
    h = mosaic_haplotypes(rng, N, L, F, cfg["switch"], cfg["flip"])
    out = dict(name=name, N=N, L=L, h=h, mu=float(cfg["mu"]), loci=decode_loci(L, min(cfg["D"], L)), seed=seed)
    if cfg["rho"] == "uniform":
        out["rho"] = rng.uniform(cfg["rho_lo"], cfg["rho_hi"], size=L - 1)
    elif cfg["rho"] == "loguniform":
        out["rho"] = np.exp(rng.uniform(np.log(cfg["rho_lo"]), np.log(cfg["rho_hi"]), size=L - 1))
    else:
        out["rho"] = None
        out["gaps"] = rng.exponential(cfg["gap_mean"], size=L - 1)
        out["Ne"] = 4.0 * cfg["Ne_tilde"] / N  # N_e = 4 Ne~ / N (Sec. 2.1)
    out["Pi"] = None if cfg["Pi"] == "uniform" else "gamma"
    out["pi_seed"] = seed + 7
    if "K" in cfg:
        out["K"] = cfg["K"]
    return out


def random_tiny(rng: np.random.Generator, N: int, L: int, rho_kind: str = "random", mu_kind: str = "scalar",
                pi_kind: str = "uniform") -> dict:
    """Small random instances for exhaustive checks (any N >= 2, L >= 1)."""
    h = (rng.random((L, N)) < 0.4).astype(np.uint8)
    if rho_kind == "zero":
        rho = np.zeros(L - 1)
    elif rho_kind == "one":
        rho = np.ones(L - 1)
    elif rho_kind == "mixed":
        rho = rng.choice([0.0, 1.0, 0.3, 1e-3], size=L - 1)
    else:
        rho = rng.uniform(0.01, 0.6, size=L - 1)
    mu = rng.uniform(0.01, 0.2) if mu_kind == "scalar" else rng.uniform(0.01, 0.2, size=L)
    Pi = None
    if pi_kind == "matrix":
        Pi = rng.gamma(2.0, 1.0, size=(N, N))
        np.fill_diagonal(Pi, 0.0)
        Pi /= Pi.sum(axis=1, keepdims=True)
    return dict(h=h, rho=rho, mu=mu, Pi=Pi, N=N, L=L)
