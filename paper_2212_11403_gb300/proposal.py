"""Learned donor proposal: training data from the dense path's posteriors, training through the
library's MLP kernels, and the proposal / sparse pipeline.

Labels.  For target i, window w and stage-1 candidate j the label is the dense posterior p_ij at
the window's middle locus on a log scale, y = 1 + log10(max(p, 1e-12)) / 12 (1 for p = 1, 0 at
1e-12 and below), so the network ranks candidates by predicted posterior mass.  The posteriors,
the features, the labels and every step of training run in libls; this module moves tensors
between the calls (dropping padded candidates).
"""
from __future__ import annotations

import numpy as np

from . import ls

WS = 256


def window_mid(L: int, w: int) -> int:
    return min(WS * w + WS // 2, L - 1)


def dense_posteriors(ctx, N: int, loci):
    """Dense posteriors [len(loci), N, N] (CUDA float32) at increasing loci."""
    import torch
    loci = [int(l) for l in loci]
    A = torch.empty((len(loci), N, N), dtype=torch.float32, device="cuda")
    P = torch.empty_like(A)
    B = torch.empty((N, N), dtype=torch.float32, device="cuda")
    fw = ls.ls_table_create(ctx, ls.LS_FWD, 0, N)
    bw = ls.ls_table_create(ctx, ls.LS_BWD, 0, N)
    try:
        ls.ls_forward(ctx, fw, loci[-1], loci, A)
        for k in range(len(loci) - 1, -1, -1):
            ls.ls_backward(ctx, bw, loci[k])
            ls.ls_table_read(bw, state=B)
            ls.ls_posterior_rows(ctx, A[k], B, 0, P[k])
        torch.cuda.synchronize()
    finally:
        ls.ls_table_destroy(fw)
        ls.ls_table_destroy(bw)
    del A
    return P


def training_set(ctx, N: int, L: int, C: int, wins, P=None):
    """(X [n, 8], y [n]) CUDA float32 over the stage-1 candidates of the windows `wins`; P are the
    dense posteriors at their middle loci (computed when None)."""
    import torch
    if P is None:
        P = dense_posteriors(ctx, N, [window_mid(L, w) for w in wins])
    Xs, ys = [], []
    cand = torch.empty((N, C), dtype=torch.int32, device="cuda")
    feat = torch.empty((N, C, 8), dtype=torch.float32, device="cuda")
    yw = torch.empty((N, C), dtype=torch.float32, device="cuda")
    for k, w in enumerate(wins):
        ls.ls_propose_window(ctx, C, int(w), cand, feat)
        ls.ls_propose_labels(ctx, P[k], cand, C, yw)
        valid = cand >= 0
        Xs.append(feat[valid])
        ys.append(yw[valid])
    return torch.cat(Xs).contiguous(), torch.cat(ys).contiguous()


def train(X, y, steps=400, batch=4096, lr=1e-3, seed=1, init_seed=7):
    """A new network trained by Adam on (X, y); returns (handle, final minibatch loss)."""
    m = ls.ls_mlp_create(None, init_seed)
    loss = ls.ls_mlp_train(m, X, y, steps, batch, lr, seed)
    return m, loss


def set_mass(idx, P, wins):
    """Posterior mass of each target's set: [len(wins), N] (CUDA) for sets idx [N, Wn, K] and dense
    posteriors P at the windows' middle loci."""
    import torch
    out = []
    for k, w in enumerate(wins):
        s = idx[:, int(w), :]
        pm = torch.gather(P[k], 1, s.clamp(min=0).long()) * (s >= 0)
        out.append(pm.sum(dim=1))
    return torch.stack(out)
