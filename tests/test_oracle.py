"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign, an
off-by-one rho index, a transposed prior) fails at least one of them:
  * brute-force enumeration of copying paths (model definition, Sec. 2.1) -> likelihood and
    every posterior marginal;
  * the raw recursions (Eq. raw_forward / raw_backward) against the rescaled ones (App. A.1/A.2);
  * closed forms at rho = 0 (one copied donor for the whole sequence) and rho = 1 (independent
    loci);
  * invariants: posteriors sum to one, forward and backward likelihoods agree, the
    forward-backward product identity holds at every locus, alpha <= 2 (App. A.3), distances are
    symmetric and non-negative;
  * values printed in the paper (CalcRho, the uniform prior, the packed cache size);
  * the Fisher-identity gradient against finite differences of the brute-force likelihood.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2212_11403_gb300 import synth
from tests import _brute

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- values printed in the paper
def test_calc_rho_matches_paper_print():
    rows = _read_golden("calc_rho_sec3_3.txt")
    x = np.array([float(r[0]) for r in rows])
    want = np.array([float(r[1]) for r in rows])
    tol = np.array([float(r[2]) for r in rows])
    got = oracle.calc_rho(x, Ne=1.0, gamma=1.0)
    assert np.all(np.abs(got - want) <= tol * want), (got, want)


def test_calc_rho_scale_and_power():
    # Eq. rho with Ne and gamma: 1 - exp(-Ne m^gamma); series for small arguments, exact at large
    m = np.array([1e-9, 3e-6, 0.01, 0.5, 2.0])
    for Ne, g in [(1.0, 1.0), (2.0, 1.0), (4.0, 0.5), (0.3, 1.7)]:
        z = Ne * m ** g
        got = oracle.calc_rho(m, Ne=Ne, gamma=g)
        series = z - z ** 2 / 2 + z ** 3 / 6 - z ** 4 / 24
        small = z < 1e-3
        assert np.allclose(got[small], series[small], rtol=1e-12, atol=0)
        assert np.allclose(got[~small], 1 - np.exp(-z[~small]), rtol=1e-13, atol=0)


def test_packed_cache_size_matches_paper():
    vals = dict((r[0], float(r[1])) for r in _read_golden("paper_printed_values.txt"))
    h = np.zeros((400, 300), dtype=np.uint8)
    nbytes, _ = oracle.pack_paper_layout(h)
    assert nbytes == int(vals["packed_cache_bytes_n300_l400"])


def test_packed_layout_bit_order():
    rng = np.random.default_rng(5)
    h = (rng.random((7, 70)) < 0.5).astype(np.uint8)
    _, words = oracle.pack_paper_layout(h)
    for l in range(7):
        for i in range(70):
            assert ((int(words[l, i // 32]) >> (i % 32)) & 1) == h[l, i]
        # padding bits beyond N are zero
        assert (int(words[l, 2]) >> (70 - 64)) == 0


def test_uniform_prior_value_matches_paper():
    vals = dict((r[0], float(r[1])) for r in _read_golden("paper_printed_values.txt"))
    # with every haplotype identical at locus 0, alpha~^0_j = theta pi_j = (1 - mu) / (N - 1)
    N = 300
    h = np.zeros((1, N), dtype=np.uint8)
    mu = 1e-8
    A, F = oracle.raw_forward_target(h, np.zeros(0), mu, 3)
    assert A[0, 3] == 0.0
    np.testing.assert_allclose(A[0, 0] / (1 - mu), vals["uniform_prior_n300"], rtol=1e-14)
    np.testing.assert_allclose(F[0], 1 - mu, rtol=1e-14)


# ---------------------------------------------------------------- brute force
CASES = []
for seed in range(6):
    for (N, L) in [(3, 1), (3, 4), (4, 3), (5, 2), (4, 5), (3, 6)]:
        CASES.append((seed, N, L))


@pytest.mark.parametrize("seed,N,L", CASES)
def test_oracle_matches_brute_force(seed, N, L):
    rng = np.random.default_rng(100 + seed * 31 + N * 7 + L)
    kinds = ["random", "zero", "one", "mixed"]
    inst = synth.random_tiny(rng, N, L, rho_kind=kinds[seed % 4], mu_kind=["scalar", "vector"][seed % 2],
                             pi_kind=["uniform", "matrix"][(seed // 2) % 2])
    h, rho, mu, Pi = inst["h"], inst["rho"], inst["mu"], inst["Pi"]
    loci = list(range(L))
    res = oracle.run(h, rho, mu, loci, Pi=Pi, want=("post", "llf", "llb"))
    for i in range(N):
        ll, marg = _brute.enumerate_target(h, rho, mu, Pi, i)
        assert abs(res["llf"][i] - ll) <= 1e-12 * max(1.0, abs(ll))
        assert abs(res["llb"][i] - ll) <= 1e-12 * max(1.0, abs(ll))
        np.testing.assert_allclose(res["post"][i], marg, rtol=1e-10, atol=1e-14)


def test_prior_rows_form_equals_the_matrix_form():
    """oracle.run with only the targets' prior rows (for N too large for a host matrix) gives the
    same results as with the full matrix, bit for bit, and with a row permuted it does not."""
    rng = np.random.default_rng(12)
    N, L = 11, 30
    inst = synth.random_tiny(rng, N, L, mu_kind="vector", pi_kind="matrix")
    h, rho, mu, Pi = inst["h"], inst["rho"], inst["mu"], inst["Pi"]
    targets = np.array([7, 0, 3, 10])
    loci = [0, 13, L - 1]
    want = ("alpha", "beta", "post", "logF", "logG", "llf", "llb")
    full = oracle.run(h, rho, mu, loci, targets=targets, Pi=Pi, want=want)
    rows = oracle.run(h, rho, mu, loci, targets=targets, Pi_rows=Pi[targets], want=want)
    for k in want:
        np.testing.assert_array_equal(rows[k], full[k])
    swapped = Pi[targets][[1, 0, 2, 3]]
    other = oracle.run(h, rho, mu, loci, targets=targets, Pi_rows=swapped, want=("llf",))
    assert abs(other["llf"][0] - full["llf"][0]) > 1e-9


# ---------------------------------------------------------------- raw vs rescaled recursions
@pytest.mark.parametrize("pi_kind", ["uniform", "matrix"])
def test_rescaled_equals_raw(pi_kind):
    rng = np.random.default_rng(7)
    N, L = 9, 25
    inst = synth.random_tiny(rng, N, L, mu_kind="vector", pi_kind=pi_kind)
    h, rho, mu, Pi = inst["h"], inst["rho"], inst["mu"], inst["Pi"]
    loci = list(range(L))
    for i in (0, 4, 8):
        At, F = oracle.raw_forward_target(h, rho, mu, i, Pi=Pi)
        Bt, G = oracle.raw_backward_target(h, rho, mu, i, Pi=Pi)
        A, lF, llf = oracle.forward_target(h, rho, mu, i, loci, Pi=Pi)
        B, lG, llb = oracle.backward_target(h, rho, mu, i, loci, Pi=Pi)
        # alpha^l = alpha~^l / F^{l-1}  (App. A.1),  beta^l = beta~^l / G^l  (App. A.2)
        for l in range(L):
            Fprev = 1.0 if l == 0 else F[l - 1]
            np.testing.assert_allclose(A[l], At[l] / Fprev, rtol=1e-11, atol=1e-300)
            ref = Bt[l] / G[l]
            ref[i] = 0.0
            np.testing.assert_allclose(B[l], ref, rtol=1e-11, atol=1e-300)
            np.testing.assert_allclose(lF[l], math.log(F[l]), rtol=1e-12)
        # log G at locus l = log G^l (G at the last locus = 1)
        np.testing.assert_allclose(lG, np.log(G), rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(llf, math.log(F[L - 1]), rtol=1e-12)
        # P = sum_j beta~^0_j theta^0_j pi_j  (Eq. G one step past locus 0)
        np.testing.assert_allclose(llb, llf, rtol=1e-12)


# ---------------------------------------------------------------- closed forms
def test_rho_zero_closed_form():
    # no recombination: the hidden donor never changes, p_ji = pi_ji mu^m (1-mu)^(L-m) / Z at every
    # locus, m = number of mismatches between h_i and h_j over all loci
    rng = np.random.default_rng(11)
    N, L = 12, 40
    inst = synth.random_tiny(rng, N, L, rho_kind="zero", pi_kind="matrix")
    h, rho, mu, Pi = inst["h"], inst["rho"], inst["mu"], inst["Pi"]
    res = oracle.run(h, rho, mu, [0, 17, L - 1], Pi=Pi, want=("post", "llf"))
    for i in range(N):
        m = (h != h[:, [i]]).sum(axis=0)
        w = Pi[i] * mu ** m * (1 - mu) ** (L - m)
        w[i] = 0.0
        for k in range(3):
            np.testing.assert_allclose(res["post"][i, k], w / w.sum(), rtol=1e-10, atol=1e-300)
        np.testing.assert_allclose(res["llf"][i], math.log(w.sum()), rtol=1e-12)


def test_rho_one_closed_form():
    # full recombination at every interval: loci independent, p^l_ji = pi_ji theta^l_ji / Z^l and
    # log P = sum_l log sum_j pi_ji theta^l_ji
    rng = np.random.default_rng(12)
    N, L = 10, 30
    inst = synth.random_tiny(rng, N, L, rho_kind="one", mu_kind="vector", pi_kind="matrix")
    h, rho, mu, Pi = inst["h"], inst["rho"], inst["mu"], inst["Pi"]
    loci = list(range(L))
    res = oracle.run(h, rho, mu, loci, Pi=Pi, want=("post", "llf"))
    for i in range(N):
        ll = 0.0
        for l in range(L):
            th = np.where(h[l] == h[l, i], 1 - mu[l], mu[l])
            w = Pi[i] * th
            w[i] = 0.0
            ll += math.log(w.sum())
            np.testing.assert_allclose(res["post"][i, l], w / w.sum(), rtol=1e-11, atol=1e-300)
        np.testing.assert_allclose(res["llf"][i], ll, rtol=1e-12)


# ---------------------------------------------------------------- invariants at realistic size
@pytest.fixture(scope="module")
def small_workload():
    return synth.make_workload("ls_n200_l1000", N=60, L=300)


def test_posterior_sums_to_one_and_diag_zero(small_workload):
    w = small_workload
    res = oracle.run(w["h"], w["rho"], w["mu"], w["loci"], want=("post",))
    p = res["post"]
    np.testing.assert_allclose(p.sum(axis=2), 1.0, rtol=1e-12)
    for i in range(w["N"]):
        assert np.all(p[i, :, i] == 0.0)
    assert np.all(p >= 0)


def test_forward_backward_likelihoods_agree(small_workload):
    w = small_workload
    res = oracle.run(w["h"], w["rho"], w["mu"], [0], want=("llf", "llb"))
    np.testing.assert_allclose(res["llf"], res["llb"], rtol=1e-12)


def test_product_identity_constant_over_loci(small_workload):
    # log sum_j alpha^l beta^l + log F^{l-1} + log G^l = log P for every l
    w = small_workload
    L = w["L"]
    loci = list(range(0, L, 7)) + [L - 1]
    res = oracle.run(w["h"], w["rho"], w["mu"], loci, targets=[0, 13, 59],
                     want=("alpha", "beta", "logF", "logG", "llf"))
    for t in range(3):
        for k, l in enumerate(loci):
            s = float(np.sum(res["alpha"][t, k] * res["beta"][t, k]))
            logF_prev = res["logF"][t, k] - math.log(res["alpha"][t, k].sum())
            val = math.log(s) + logF_prev + res["logG"][t, k]
            np.testing.assert_allclose(val, res["llf"][t], rtol=1e-12)


def test_alpha_bound_and_nonnegative(small_workload):
    w = small_workload
    res = oracle.run(w["h"], w["rho"], w["mu"], list(range(0, w["L"], 3)), targets=[1, 2, 3], want=("alpha", "beta"))
    assert res["alpha"].max() <= 2.0 and res["alpha"].min() >= 0.0  # App. A.3: alpha <= 2
    assert res["beta"].min() >= 0.0


def test_distance_symmetry_and_clamp(small_workload):
    w = small_workload
    N = w["N"]
    res = oracle.run(w["h"], w["rho"], w["mu"], [w["L"] // 2], want=("post",))
    d = oracle.distance_block(res["post"][:, 0, :], np.arange(N))
    np.testing.assert_array_equal(d, d.T)
    assert np.all(np.diag(d) == 0.0)
    assert np.all(d >= 0.0)
    eps = np.finfo(np.float64).eps
    assert d.max() <= -math.log(eps) + 1e-12
    # p below eps is clamped to eps (Eq. distmat)
    assert oracle.distance_pair(0.0, 0.0) == pytest.approx(-math.log(eps))
    assert oracle.distance_pair(0.5, 0.25) == pytest.approx(-(math.log(0.5) + math.log(0.25)) / 2)


def test_identical_donors_have_equal_posterior():
    rng = np.random.default_rng(3)
    N, L = 8, 50
    inst = synth.random_tiny(rng, N, L)
    h = inst["h"].copy()
    h[:, 5] = h[:, 2]  # donors 2 and 5 identical
    res = oracle.run(h, inst["rho"], inst["mu"], [0, 20, 49], targets=[0, 1, 7], want=("post",))
    np.testing.assert_allclose(res["post"][:, :, 2], res["post"][:, :, 5], rtol=1e-12)


def test_total_underflow_gives_nan_columns():
    # mu = 0 and a private allele: every theta is 0 at that locus, so sum_j alpha = 0 there (total
    # underflow, App. A.3): log F becomes -inf and the next column is NaN except the diagonal (0)
    N, L = 5, 4
    h = np.zeros((L, N), dtype=np.uint8)
    h[2, 0] = 1
    A, lF, ll = oracle.forward_target(h, np.full(L - 1, 0.1), 0.0, 0, loci=[1, 2, 3])
    assert np.isfinite(lF[0]) and lF[1] == -math.inf
    assert A[2, 0] == 0.0 and np.all(np.isnan(A[2, 1:]))
    assert math.isnan(ll)


# ---------------------------------------------------------------- gradient
def test_gradient_matches_brute_force_finite_differences():
    rng = np.random.default_rng(21)
    N, L, K = 4, 5, 2
    inst = synth.random_tiny(rng, N, L)
    h, rho, mu = inst["h"], inst["rho"], float(inst["mu"])
    iv = synth.rho_intervals(L, K)
    eps = 1e-6
    for i in range(N):
        ll, gmu, grho = oracle.grad_target(h, rho, mu, i, iv, K)
        assert abs(ll - _brute.loglik(h, rho, mu, None, i)) < 1e-12
        fd_mu = (_brute.loglik(h, rho, mu * math.exp(eps), None, i) -
                 _brute.loglik(h, rho, mu * math.exp(-eps), None, i)) / (2 * eps)
        assert abs(gmu - fd_mu) < 1e-7 * max(1, abs(fd_mu))
        for k in range(K):
            sc = np.where(iv == k, math.exp(eps), 1.0)
            fd = (_brute.loglik(h, rho * sc, mu, None, i) - _brute.loglik(h, rho / sc, mu, None, i)) / (2 * eps)
            assert abs(grho[k] - fd) < 1e-7 * max(1, abs(fd))


def test_pac_gradient_matches_oracle_finite_differences():
    w = synth.make_workload("ls_n200_l1000", N=20, L=60)
    K = 4
    iv = synth.rho_intervals(w["L"], K)
    pac, gmu, grho = oracle.pac_grad(w["h"], w["rho"], w["mu"], iv, K)
    llf = oracle.run(w["h"], w["rho"], w["mu"], [0], want=("llf",))["llf"]
    assert abs(pac - llf.sum()) < 1e-9 * abs(pac)

    def pac_at(rho, mu):
        return oracle.run(w["h"], rho, mu, [0], want=("llf",))["llf"].sum()

    e = 1e-5
    fd_mu = (pac_at(w["rho"], w["mu"] * math.exp(e)) - pac_at(w["rho"], w["mu"] * math.exp(-e))) / (2 * e)
    assert abs(gmu - fd_mu) < 1e-5 * max(1, abs(fd_mu))
    for k in range(K):
        sc = np.where(iv == k, math.exp(e), 1.0)
        fd = (pac_at(w["rho"] * sc, w["mu"]) - pac_at(w["rho"] / sc, w["mu"])) / (2 * e)
        assert abs(grho[k] - fd) < 1e-5 * max(1, abs(fd))
