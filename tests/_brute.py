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
