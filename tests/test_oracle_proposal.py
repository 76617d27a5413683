"""Pins of the proposal oracle (oracle/proposal.py): brute force on tiny inputs and finite
differences of the network loss."""
import numpy as np

from oracle import proposal as op


def test_mismatch_counts_brute_force():
    rng = np.random.default_rng(1)
    L, N = 600, 9
    h = (rng.random((L, N)) < 0.3).astype(np.uint8)
    for w in range(op.windows(L)):
        M = op.mismatch_counts(h, w)
        lo, hi = 256 * w, min(256 * (w + 1), L)
        for i in range(N):
            for j in range(N):
                assert M[i, j] == min(sum(int(h[l, i] != h[l, j]) for l in range(lo, hi)), 255)


def test_mismatch_counts_saturate_at_255():
    h = np.zeros((256, 2), dtype=np.uint8)
    h[:, 1] = 1
    assert op.mismatch_counts(h, 0)[0, 1] == 255


def test_stage1_selection_by_brute_force():
    rng = np.random.default_rng(2)
    L, N, C = 900, 12, 5
    h = (rng.random((L, N)) < 0.4).astype(np.uint8)
    Wn = op.windows(L)
    for w in range(Wn):
        cand, feat = op.stage1(h, w, C)
        for i in range(N):
            sc = {}
            for j in range(N):
                if j == i:
                    continue
                s = 0
                for v in (w - 1, w, w + 1):
                    if 0 <= v < Wn:
                        lo, hi = 256 * v, min(256 * (v + 1), L)
                        s += min(int(np.sum(h[lo:hi, i] != h[lo:hi, j])), 255)
                sc[j] = s
            best = sorted(sorted(sc, key=lambda j: (sc[j], j))[:C])
            assert list(cand[i]) == best
            # features: match fractions of windows w-3..w+3 (clamped), then 0
            j = best[0]
            for d in range(7):
                v = min(max(w + d - 3, 0), Wn - 1)
                lo, hi = 256 * v, min(256 * (v + 1), L)
                assert abs(feat[i, 0, d] - (1 - np.sum(h[lo:hi, i] != h[lo:hi, j]) / (hi - lo))) < 1e-15
            assert feat[i, 0, 7] == 0.0


def test_stage1_pads_when_fewer_donors_than_c():
    h = (np.random.default_rng(3).random((300, 4)) < 0.5).astype(np.uint8)
    cand, _ = op.stage1(h, 0, 6)
    assert np.all(cand[:, 3:] == -1) and np.all(cand[:, :3] >= 0)


def test_labels_closed_form_values():
    # p = 1 -> 1, p = 1e-6 -> 1/2, p = 1e-12 and below (0 too) -> 0, padding -> 0; the row of
    # each candidate is its own target's
    P = np.array([[1.0, 1e-6, 1e-12], [0.0, 1e-3, 1e-15]])
    cand = np.array([[0, 1, 2, -1], [0, 1, 2, -1]])
    y = op.labels(P, cand)
    np.testing.assert_allclose(y, [[1.0, 0.5, 0.0, 0.0], [0.0, 0.75, 0.0, 0.0]], rtol=0, atol=1e-15)


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    p = rng.normal(0, 0.2, op.N_PARAMS)
    X = rng.random((40, 8))
    X[:, 7] = 0.0
    y = rng.random(40)
    loss, g = op.mlp_loss_grad(p, X, y)
    assert abs(loss - 0.5 * np.mean((op.mlp_forward(p, X) - y) ** 2)) < 1e-12
    h = 1e-6
    for k in list(rng.choice(op.N_PARAMS, 40, replace=False)) + [op.P_B3, op.P_W1, op.P_B1 + 3, op.P_W3 + 7]:
        e = np.zeros(op.N_PARAMS)
        e[k] = h
        fd = (op.mlp_loss_grad(p + e, X, y)[0] - op.mlp_loss_grad(p - e, X, y)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_bf16_rounding_matches_definition():
    # nearest-even rounding to 8 significant bits
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -9, -2.5, 3.0e-3])
    r = op.bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # half an ulp (2^-7): tie to even
    assert r[3] == 1.0                      # a quarter ulp rounds down
    assert r[2] == 1.0 + 2 ** -7            # three quarters of an ulp rounds up
    assert r[4] == -2.5
    assert abs(r[5] - 3.0e-3) <= 3.0e-3 * 2 ** -8


def test_sparse_oracle_with_full_sets_is_the_dense_oracle():
    import oracle
    rng = np.random.default_rng(9)
    L, N = 40, 6
    h = (rng.random((L, N)) < 0.4).astype(np.uint8)
    rho = rng.uniform(0.01, 0.3, L - 1)
    mu = 0.05
    ws = 7
    Wn = (L + ws - 1) // ws
    sets = np.array([[[j for j in range(N) if j != i]] * Wn for i in range(N)])
    loci = [0, 13, 39]
    p = op.sparse_posteriors(h, rho, mu, sets, ws, loci)
    ref = oracle.run(h, rho, mu, loci, want=("post",))["post"]
    assert float(np.max(np.abs(p - ref))) < 1e-12


def test_lookahead_sets_union():
    S = np.array([[[1, 3, -1], [2, 3, 5], [0, -1, -1]]])
    U = op.lookahead_sets(S)
    assert list(U[0, 0]) == [1, 2, 3, 5, -1, -1]
    assert list(U[0, 1]) == [0, 2, 3, 5, -1, -1]
    assert list(U[0, 2]) == [0, -1, -1, -1, -1, -1]
    V = op.lookahead_sets(S, 2)
    assert list(V[0, 0]) == [1, 2, 3, 5] + [-1] * 5
    assert list(V[0, 1]) == [0, 1, 2, 3, 5] + [-1] * 4
    assert list(V[0, 2]) == [0, 2, 3, 5] + [-1] * 5


def test_pooled_sparse_oracle_with_full_sets_is_the_dense_oracle():
    """with every donor in every set the pool is empty and the pooled chain is the dense one."""
    import oracle
    rng = np.random.default_rng(19)
    L, N = 35, 7
    h = (rng.random((L, N)) < 0.4).astype(np.uint8)
    rho = rng.uniform(0.01, 0.3, L - 1)
    sets = np.array([[[j for j in range(N) if j != i]] * 5 for i in range(N)])
    p = op.sparse_posteriors(h, rho, 0.05, sets, 7, [0, 20, 34], pool=True)
    ref = oracle.run(h, rho, 0.05, [0, 20, 34], want=("post",))["post"]
    assert float(np.max(np.abs(p - ref))) < 1e-12


def test_pooled_sparse_oracle_is_exact_when_outside_donors_are_identical():
    """donors outside the set that are all identical to each other (and so share one emission at
    every locus) are represented exactly by the pool: posteriors of set donors equal the dense
    oracle's when the outside donors never enter the set."""
    import oracle
    rng = np.random.default_rng(23)
    L, N = 40, 8
    h = (rng.random((L, N)) < 0.4).astype(np.uint8)
    h[:, 5] = h[:, 6]
    h[:, 7] = h[:, 6]
    rho = rng.uniform(0.01, 0.3, L - 1)
    i = 0
    sets = -np.ones((N, 4, 4), dtype=np.int64)
    sets[i, :, :] = [1, 2, 3, 4]   # outside: 5, 6, 7 (identical)
    for j in range(1, N):
        sets[j, :, :N - 1 if N - 1 <= 4 else 4] = [k for k in range(N) if k != j][:4]
    p = op.sparse_posteriors(h, rho, 0.05, sets, 10, [0, 17, 39], pool=True)
    ref = oracle.run(h, rho, 0.05, [0, 17, 39], targets=[i], want=("post",))["post"][0]
    # the pool holds the outside mass exactly and shares its posterior equally among identical
    # donors, so every donor's posterior is the dense one
    np.testing.assert_allclose(p[i], ref, rtol=1e-12, atol=1e-300)


def _changing_sets(N, Wn, base, extra_choices, i, rng):
    """sets [N, Wn, K] for target i: base donors plus, per window, a different subset of
    extra_choices (never i); other targets get all donors but themselves (unused)."""
    K = N - 1
    sets = -np.ones((N, Wn, K), dtype=np.int64)
    for t in range(N):
        sets[t, :, :N - 1] = [k for k in range(N) if k != t]
    for w in range(Wn):
        pick = [j for j in extra_choices if j != i and rng.random() < 0.5]
        s = sorted(set(j for j in base if j != i) | set(pick))
        sets[i, w, :] = -1
        sets[i, w, :len(s)] = s
    return sets


def test_pooled_chain_is_an_exact_lumping_with_changing_sets():
    """Donors outside the set all identical (one shared haplotype, hence one emission at every
    locus): by symmetry the dense chain gives them equal alpha and beta, so the pool holds their
    mass exactly, a donor that leaves hands its mass to the pool, and an entering donor's
    pool share is its dense value.  The pooled chain is then an exact lumping of the dense chain
    even as donors of the identical group enter and leave the set between windows, and the set
    donors' posteriors equal the dense ones, and so do the outside donors' equal shares of the
    pool's posterior mass."""
    import oracle
    rng = np.random.default_rng(41)
    L, N, ws = 36, 10, 4
    Wn = (L + ws - 1) // ws
    h = (rng.random((L, N)) < 0.45).astype(np.uint8)
    G = [5, 6, 7, 8, 9]
    for g in G[1:]:
        h[:, g] = h[:, G[0]]
    rho = rng.uniform(0.02, 0.4, L - 1)
    mu = 0.07
    loci = [0, 3, 4, 9, 17, 26, 35]
    for i in (0, 2, 6):   # targets outside and inside the identical group
        sets = _changing_sets(N, Wn, [0, 1, 2, 3, 4], G, i, rng)
        changes = sum(1 for w in range(1, Wn) if list(sets[i, w]) != list(sets[i, w - 1]))
        assert changes >= 3
        p = op.sparse_posteriors(h, rho, mu, sets, ws, loci, pool=True)[i]
        ref = oracle.run(h, rho, mu, loci, targets=[i], want=("post",))["post"][0]
        np.testing.assert_allclose(p, ref, rtol=1e-12, atol=1e-300)


def test_pooled_chain_matches_brute_force_of_its_definition():
    """Arbitrary haplotypes (the pool is then only an approximation of the dense chain): the
    oracle's pooled recursions, window changes included, against an enumeration of every path
    of the pooled chain written out as an explicit HMM (tests/_brute.py)."""
    from tests._brute import enumerate_pooled
    rng = np.random.default_rng(43)
    for trial in range(4):
        L, N, ws = 6, 5, 2
        Wn = 3
        h = (rng.random((L, N)) < 0.5).astype(np.uint8)
        rho = rng.uniform(0.05, 0.6, L - 1)
        mu = rng.uniform(0.02, 0.2)
        i = trial % N
        others = [j for j in range(N) if j != i]
        sets = -np.ones((N, Wn, N - 1), dtype=np.int64)
        for t in range(N):
            sets[t, :, :N - 1] = [k for k in range(N) if k != t]
        chosen = [[others[0], others[1]], [others[1], others[2]], [others[0], others[3]]]
        for w in range(Wn):
            sets[i, w, :] = -1
            sets[i, w, :2] = sorted(chosen[w])
        loci = list(range(L))
        p = op.sparse_posteriors(h, rho, mu, sets, ws, loci, pool=True)[i]
        marg = enumerate_pooled(h, rho, mu, [[int(j) for j in sets[i, l // ws] if j >= 0] for l in range(L)], i)
        for l in range(L):
            S = [int(j) for j in sets[i, l // ws] if j >= 0]
            out = [j for j in range(N) if j != i and j not in S]
            for j in S:
                assert abs(p[l, j] - marg[l].get(j, 0.0)) <= 1e-12, (trial, l, j)
            for j in out:   # an equal share of the pool state's posterior
                assert abs(p[l, j] - marg[l].get("o", 0.0) / len(out)) <= 1e-12, (trial, l, j)
            assert abs(p[l].sum() - 1.0) <= 1e-12
