"""Oracle of the learned donor proposal (plain numpy, float64 unless stated).

TEST INFRASTRUCTURE ONLY: the product library never imports, links or runs anything here.

The proposal is an extension of the paper's method (the paper runs every target against all
donors, Sec. 2.1) and has no counterpart there; these are its definitions, written here first and
pinned by brute force, by the dense oracle where the restricted chain must reduce to it exactly
(full sets; identical outside donors, an exact lumping), and by an enumeration of the pooled
chain's paths (tests/test_oracle_proposal.py):
  * window w holds loci [256 w, min(256 (w+1), L)); the mismatch count of haplotypes i, j in w is
    the number of loci of the window where they differ, stored as min(count, 255);
  * stage 1 keeps for target i the C donors j != i with the smallest sum of mismatch counts over
    the windows w-1, w, w+1 that exist, ties to the lower j, in ascending j;
  * the features of a candidate are the match fractions 1 - count / n of windows w-3..w+3, window
    indices clamped to [0, Wn-1], then one zero;
  * the network maps 8 inputs through 256 and 256 ReLU units to one score; the loss is half the
    mean squared error;
  * the training label of a candidate is its dense posterior on a log scale,
    y = 1 + log10(max(p, 1e-12)) / 12 (pinned by its closed-form values).
"""
from __future__ import annotations

import numpy as np

WS = 256
P_W1, P_B1 = 0, 8 * 256
P_W2 = P_B1 + 256
P_B2 = P_W2 + 256 * 256
P_W3 = P_B2 + 256
P_B3 = P_W3 + 256
N_PARAMS = P_B3 + 1


def windows(L):
    return (L + WS - 1) // WS


def mismatch_counts(h, w):
    """[N, N] int: min(#loci of window w where h_i and h_j differ, 255)."""
    L = h.shape[0]
    hw = h[WS * w:min(WS * (w + 1), L)].astype(np.int64)      # [n, N]
    d = hw.T @ (1 - hw) + (1 - hw).T @ hw                      # differing loci per pair
    return np.minimum(d, 255)


def stage1(h, w, C):
    """(cand [N, C] int, -1 padded; feat [N, C, 8] float64) of window w."""
    L, N = h.shape
    Wn = windows(L)
    M = {v: mismatch_counts(h, v) for v in range(max(0, w - 3), min(Wn, w + 4))}
    score = sum(M[v] for v in (w - 1, w, w + 1) if 0 <= v < Wn)
    n_of = {v: min(WS, L - WS * v) for v in M}
    cand = -np.ones((N, C), dtype=np.int64)
    feat = np.zeros((N, C, 8))
    for i in range(N):
        js = [j for j in range(N) if j != i]
        js.sort(key=lambda j: (score[i, j], j))
        keep = sorted(js[:C])
        cand[i, :len(keep)] = keep
        for q, j in enumerate(keep):
            for d in range(7):
                v = min(max(w + d - 3, 0), Wn - 1)
                feat[i, q, d] = 1.0 - M[v][i, j] / n_of[v]
    return cand, feat


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    W1 = p[P_W1:P_B1].reshape(8, 256)
    b1 = p[P_B1:P_W2]
    W2 = p[P_W2:P_B2].reshape(256, 256)
    b2 = p[P_B2:P_W3]
    w3 = p[P_W3:P_B3]
    b3 = p[P_B3]
    return W1, b1, W2, b2, w3, b3


def mlp_forward(p, X):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    H1 = np.maximum(X @ W1 + b1, 0.0)
    H2 = np.maximum(H1 @ W2 + b2, 0.0)
    return H2 @ w3 + b3


def bf16(x):
    """round float64 values to bfloat16 (via float32, nearest even) and back to float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def mlp_forward_bf16(p, X):
    """The inference kernel's arithmetic: inputs, W1, W2 and the first hidden layer rounded to
    bfloat16, everything else exact (float64 here)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    b1_32, b2_32 = np.float32(b1).astype(np.float64), np.float32(b2).astype(np.float64)
    H1 = bf16(np.maximum(bf16(X) @ bf16(W1) + b1_32, 0.0))
    H2 = np.maximum(H1 @ bf16(W2) + b2_32, 0.0)
    return H2 @ np.float32(w3).astype(np.float64) + float(np.float32(b3))


def mlp_loss_grad(p, X, y):
    """(loss, grad [N_PARAMS]) of sum_r (s_r - y_r)^2 / (2n), by the chain rule."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    n = X.shape[0]
    Z1 = X @ W1 + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2 + b2
    H2 = np.maximum(Z2, 0.0)
    s = H2 @ w3 + b3
    r = s - y
    loss = 0.5 * float(np.sum(r * r)) / n
    ds = r / n
    g = np.zeros(N_PARAMS)
    g[P_W3:P_B3] = H2.T @ ds
    g[P_B3] = ds.sum()
    dZ2 = np.outer(ds, w3) * (Z2 > 0)
    g[P_W2:P_B2] = (H1.T @ dZ2).reshape(-1)
    g[P_B2:P_W3] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2.T) * (Z1 > 0)
    g[P_W1:P_B1] = (X.T @ dZ1).reshape(-1)
    g[P_B1:P_W2] = dZ1.sum(axis=0)
    return loss, g


def labels(P, cand):
    """y [N, C]: 1 + log10(max(P[i, cand[i, c]], 1e-12)) / 12 for a candidate, 0 for padding (-1)."""
    P = np.asarray(P, dtype=np.float64)
    cand = np.asarray(cand)
    y = np.zeros(cand.shape)
    for i in range(cand.shape[0]):
        for c in range(cand.shape[1]):
            j = int(cand[i, c])
            if j >= 0:
                y[i, c] = 1.0 + np.log10(max(P[i, j], 1e-12)) / 12.0
    return y


def lookahead_sets(S, span=1):
    """U[i, w] = S[i, w] u S[i, w+1] (span 1) or S[i, w-1] u S[i, w] u S[i, w+1] (span 2),
    ascending, -1 padded to (span + 1) K."""
    N, Wn, K = S.shape
    U = -np.ones((N, Wn, (span + 1) * K), dtype=np.int64)
    for i in range(N):
        for w in range(Wn):
            u = set(int(j) for j in S[i, w] if j >= 0)
            if w + 1 < Wn:
                u |= set(int(j) for j in S[i, w + 1] if j >= 0)
            if span >= 2 and w > 0:
                u |= set(int(j) for j in S[i, w - 1] if j >= 0)
            u = sorted(u)
            U[i, w, :len(u)] = u
    return U


def sparse_posteriors(h, rho, mu, sets, ws, loci, pool=False):
    """Posteriors [N, len(loci), N] of the chains restricted to per-window donor sets (sets
    [N, Wn, K], ascending, -1 padded), prior 1/(N-1) kept, continuation only for donors in the sets
    of both loci.

    pool=False drops the recombination mass that goes to donors outside the set; posteriors are
    normalised over the set and are 0 outside it.

    pool=True carries the outside donors as one aggregate state o with their average emission at
    each locus (count of outside donors sharing the target's allele), o <- theta_out c o
    + r sum_out theta, adds o to the normalisers, moves the mass of leaving donors into o and starts
    entering donors at o's average.  The posterior is that of the pooled chain over its states (the
    set's donors and the pool): the normaliser adds the pool's forward mass times its donors' mean
    backward value, and every outside donor receives an equal share of the pool's posterior mass."""
    L, N = h.shape
    pi = 1.0 / (N - 1)
    mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), (L,))
    out = np.zeros((N, len(loci), N))
    slot = {int(l): k for k, l in enumerate(loci)}
    ones = h.sum(axis=1).astype(np.int64)

    def theta(l, i, j):
        return 1.0 - mu[l] if h[l, j] == h[l, i] else mu[l]

    def out_sum(l, i, setl):
        """(sum of theta over the outside donors, their count) at locus l."""
        nout = N - 1 - len(setl)
        mtot = (ones[l] if h[l, i] else N - ones[l]) - 1
        mset = sum(1 for j in setl if h[l, j] == h[l, i])
        mout = min(max(mtot - mset, 0), nout)
        return (1.0 - mu[l]) * mout + mu[l] * (nout - mout), nout

    def move(vals, old, new, o):
        """values on the set `new` from those on `old`, and the pool after the change."""
        mapped = sum(vals[j] for j in old if j in new)
        nout_old = N - 1 - len(old)
        fill = o / nout_old if (pool and nout_old > 0) else 0.0
        entering = [j for j in new if j not in old]
        res = {j: (vals[j] if j in old else fill) for j in new}
        if pool:
            o = max(o + (sum(vals.values()) - mapped) - len(entering) * fill, 0.0)
        return res, o

    for i in range(N):
        setof = [[int(j) for j in sets[i, l // ws] if j >= 0] for l in range(L)]
        alpha = [None] * L
        apool = [0.0] * L   # forward pool mass at each locus (pool=True)
        # forward
        a = {j: theta(0, i, j) * pi for j in setof[0]}
        ts, no = out_sum(0, i, setof[0])
        o = pi * ts if pool else 0.0
        tot = sum(a.values()) + o
        alpha[0] = a
        apool[0] = o
        for l in range(1, L):
            if setof[l] != setof[l - 1]:
                a, o = move(a, setof[l - 1], setof[l], o)
            c, r = (1 - rho[l - 1]) / tot, rho[l - 1] * pi
            a = {k: theta(l, i, k) * (c * a[k] + r) for k in setof[l]}
            if pool:
                ts, no = out_sum(l, i, setof[l])
                o = (ts / no if no > 0 else 0.0) * (c * o) + r * ts
            tot = sum(a.values()) + o
            alpha[l] = a
            apool[l] = o
        # backward (t = theta beta)
        t = {j: theta(L - 1, i, j) for j in setof[L - 1]}
        beta = {j: 1.0 for j in setof[L - 1]}
        ts, no = out_sum(L - 1, i, setof[L - 1])
        o = ts if pool else 0.0
        tot = sum(t.values()) + o
        for l in range(L - 1, -1, -1):
            nout = N - 1 - len(setof[l])
            bpool = 1.0   # mean backward value of the outside donors at l
            if l < L - 1:
                if setof[l] != setof[l + 1]:
                    t, o = move(t, setof[l + 1], setof[l], o)
                c, r = (1 - rho[l]) / (pi * tot), rho[l]
                beta = {j: c * t[j] + r for j in setof[l]}
                bpool = c * (o / nout if nout > 0 else 0.0) + r
                t = {j: theta(l, i, j) * beta[j] for j in setof[l]}
                if pool:
                    ts, no = out_sum(l, i, setof[l])
                    o = (ts / no if no > 0 else 0.0) * (c * o) + r * ts
                tot = sum(t.values()) + o
            if l in slot:
                zp = apool[l] * bpool if (pool and nout > 0) else 0.0
                z = sum(alpha[l][j] * beta[j] for j in setof[l]) + zp
                for j in setof[l]:
                    out[i, slot[l], j] = alpha[l][j] * beta[j] / z
                if pool and nout > 0:
                    share = zp / (z * nout)
                    inset = set(setof[l])
                    for j in range(N):
                        if j != i and j not in inset:
                            out[i, slot[l], j] = share
    return out
