"""Brute-force enumeration of copying paths for tiny LS instances (pins the oracle).

Written directly from the model definition (Sec. 2.1): the copying prior Pi, the emission
kernel (Eq. emission, the two-case form, not the App. A.3 rewrite) and the transition kernel
(Eq. transition, with rho[l] the probability of the interval between loci l and l+1).  It sums
over all (N-1)^L hidden paths, so it shares no recursion with the oracle.
"""
import itertools
import math

import numpy as np


def _prior(Pi, N, i, j):
    if j == i:
        return 0.0
    return 1.0 / (N - 1) if Pi is None else float(Pi[i, j])


def _mu(mu, l):
    mu = np.atleast_1d(mu)
    return float(mu[0] if mu.size == 1 else mu[l])


def enumerate_target(h, rho, mu, Pi, i):
    """(log P(h_i | h_-i), marginals [L, N]) by summing over every copying path."""
    L, N = h.shape
    donors = [j for j in range(N) if j != i]

    def theta(l, j):
        m = _mu(mu, l)
        return 1.0 - m if h[l, j] == h[l, i] else m

    def trans(l, j, k):  # X^{l-1} = j -> X^l = k, interval l-1
        r = float(rho[l - 1])
        return r * _prior(Pi, N, i, k) + (1.0 - r) * (1.0 if k == j else 0.0)

    total = 0.0
    marg = np.zeros((L, N))
    for path in itertools.product(donors, repeat=L):
        p = _prior(Pi, N, i, path[0]) * theta(0, path[0])
        for l in range(1, L):
            if p == 0.0:
                break
            p *= trans(l, path[l - 1], path[l]) * theta(l, path[l])
        if p == 0.0:
            continue
        total += p
        for l in range(L):
            marg[l, path[l]] += p
    return math.log(total), marg / total


def loglik(h, rho, mu, Pi, i):
    return enumerate_target(h, rho, mu, Pi, i)[0]


def enumerate_pooled(h, rho, mu, sets_of_locus, i):
    """Marginals of the pooled restricted chain of target i by summing over every path.

    The chain is written out as an explicit inhomogeneous HMM, not as recursions: at locus l its
    states are the donors of the set S^l (sets_of_locus[l], a list without i) plus one pool state
    'o' standing for the n_out(l) = N-1-|S^l| donors outside the set.
      * start: pi = 1/(N-1) per set donor, n_out(0) pi for the pool;
      * emission: theta of the donor for a set donor; for the pool the mean of theta over the
        outside donors, computed from their haplotypes;
      * from locus l-1 to l, when the set changes, a boundary map first: a donor kept in the set
        stays, a donor that leaves goes to the pool, and the pool sends each entering donor a
        1/n_out(l-1) share (it keeps the rest); then the copying transition over S^l and the pool:
        set donor -> set donor k: (1 - rho) [same] + rho pi; -> pool: rho pi n_out(l);
        pool -> set donor k: rho pi; pool -> pool: (1 - rho) + rho pi n_out(l).
    Returns {l: {state: posterior}} with the states of S^l and 'o'."""
    L, N = h.shape
    pi = 1.0 / (N - 1)
    mus = np.broadcast_to(np.asarray(mu, dtype=np.float64), (L,))

    def theta(l, j):
        return 1.0 - mus[l] if h[l, j] == h[l, i] else mus[l]

    def outside(l):
        s = set(sets_of_locus[l])
        return [j for j in range(N) if j != i and j not in s]

    def emit(l, z):
        if z == "o":
            out = outside(l)
            return sum(theta(l, j) for j in out) / len(out) if out else 0.0
        return theta(l, z)

    def boundary(l, a, b):  # locus l-1 -> l: weight of moving from a (state of l-1) to b (of l)
        old, new = set(sets_of_locus[l - 1]), set(sets_of_locus[l])
        if old == new:
            return 1.0 if a == b else 0.0
        n_old = N - 1 - len(old)
        if a == "o":
            if n_old == 0:
                return 0.0
            entering = [k for k in new if k not in old]
            if b == "o":
                return 1.0 - len(entering) / n_old
            return 1.0 / n_old if b in entering else 0.0
        if a in new:
            return 1.0 if b == a else 0.0
        return 1.0 if b == "o" else 0.0

    def trans(l, a, b):  # copying transition at the states of locus l (interval l-1)
        r = float(rho[l - 1])
        n_out = len(outside(l))
        if b == "o":
            return ((1.0 - r) if a == "o" else 0.0) + r * pi * n_out
        return ((1.0 - r) if a == b else 0.0) + r * pi

    states = [list(sets_of_locus[l]) + ["o"] for l in range(L)]

    def step(l, a, b):  # state a at l-1 -> state b at l
        return sum(boundary(l, a, m) * trans(l, m, b) for m in states[l])

    total = 0.0
    marg = [dict() for _ in range(L)]
    for path in itertools.product(*states):
        z0 = path[0]
        p = (pi * len(outside(0)) if z0 == "o" else pi) * emit(0, z0)
        for l in range(1, L):
            if p == 0.0:
                break
            p *= step(l, path[l - 1], path[l]) * emit(l, path[l])
        if p == 0.0:
            continue
        total += p
        for l in range(L):
            marg[l][path[l]] = marg[l].get(path[l], 0.0) + p
    return [{z: v / total for z, v in m.items()} for m in marg]
