"""Pins of the oracle's product-matrix MBR code (Sec. 2 parameters, Sec. 3.2
systematic Psi = [I; Psi''], Sec. 4.2 operations) against facts the paper
and the mathematics fix: the MBR point alpha = d, k Delta = k(2d-k+1)/2; the
product form C = Psi M with M = [S T; T^t 0] symmetric; the systematic
nodes holding message symbols verbatim; exact repair from every helper set
and exact reconstruction from every k-subset (small n), sampled at n=16."""
import itertools

import numpy as np
import pytest

import oracle as O


def mul(a, b):
    """GF(2^8) product by shift and reduce (modulus 0x11D), independent of
    the oracle's log tables."""
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        if a & 0x100:
            a ^= 0x11D
        b >>= 1
    return r


CASES = [(5, 3, 4), (6, 3, 4), (6, 3, 5), (7, 4, 6), (8, 4, 6), (8, 4, 7)]


@pytest.mark.parametrize("n,k,d", CASES + [(16, 8, 14), (16, 8, 15), (32, 16, 30)])
def test_mbr_point_parameters(n, k, d):
    """Sec. 2: MBR codes have alpha = d and k Delta message blocks with
    Delta = (2d-k+1)/2, all of them placed in M exactly as S (symmetric
    k x k) and T (k x (d-k))."""
    a, B = O.mbr_params(n, k, d)
    assert a == d
    assert 2 * B == k * (2 * d - k + 1)
    L = O.mbr_index_matrix(k, d)
    assert (L == L.T).all()                            # M is symmetric
    assert (L[k:, k:] == -1).all()                     # the zero block
    assert (L[:k, :] >= 0).all()
    assert sorted(set(L[L >= 0].tolist())) == list(range(B))


def test_mbr_rejects_points_off_the_mbr_range():
    for n, k, d in [(6, 3, 2), (6, 3, 6), (4, 0, 2)]:
        with pytest.raises(O.OracleError):
            O.mbr_params(n, k, d)


@pytest.mark.parametrize("n,k,d", [(6, 3, 4), (8, 4, 7), (16, 8, 14)])
def test_mbr_generator_is_the_product_form(n, k, d):
    """G X equals Psi M(X) computed as a matrix product (Sec. 3.1 applied to
    the MBR message matrix)."""
    a, B = O.mbr_params(n, k, d)
    rng = np.random.default_rng(1)
    X = rng.integers(0, 256, (B, 3), dtype=np.uint8)
    Y = O.mbr_encode(n, k, d, X)
    Psi = O.mbr_psi(n, k, d)
    L = O.mbr_index_matrix(k, d)
    for t in range(X.shape[1]):
        M = np.where(L >= 0, X[np.maximum(L, 0), t], 0)
        for i in range(n):
            for j in range(a):
                acc = 0
                for l in range(d):
                    acc ^= mul(int(Psi[i, l]), int(M[l, j]))
                assert Y[a * i + j, t] == acc, (i, j, t)


@pytest.mark.parametrize("n,k,d", CASES + [(16, 8, 14)])
def test_mbr_systematic_nodes_store_symbols(n, k, d):
    """Psi = [I; Psi''] (Sec. 3.2): node i < k stores row i of M verbatim, so
    every message symbol sits on the systematic nodes."""
    a, B = O.mbr_params(n, k, d)
    X = np.random.default_rng(2).integers(0, 256, (B, 5), dtype=np.uint8)
    Y = O.mbr_encode(n, k, d, X)
    L = O.mbr_index_matrix(k, d)
    seen = set()
    for i in range(k):
        for j in range(a):
            assert np.array_equal(Y[a * i + j], X[L[i, j]])
            seen.add(int(L[i, j]))
    assert seen == set(range(B))


def _rank(A):
    A = [list(map(int, r)) for r in A]
    rows, cols, r = len(A), len(A[0]), 0
    for c in range(cols):
        p = next((i for i in range(r, rows) if A[i][c]), None)
        if p is None:
            continue
        A[r], A[p] = A[p], A[r]
        inv = next(x for x in range(1, 256) if mul(A[r][c], x) == 1)
        A[r] = [mul(v, inv) for v in A[r]]
        for i in range(rows):
            if i != r and A[i][c]:
                f = A[i][c]
                A[i] = [v ^ mul(f, w) for v, w in zip(A[i], A[r])]
        r += 1
    return r


@pytest.mark.parametrize("n,k,d", [(6, 3, 4), (7, 4, 6), (8, 4, 6)])
def test_mbr_psi_rank_conditions(n, k, d):
    """Any d rows of Psi and any k rows of Phi (its first k columns) are
    independent: the two conditions PM-MBR repair and reconstruction need."""
    Psi = O.mbr_psi(n, k, d)
    for rows in itertools.combinations(range(n), d):
        assert _rank(Psi[list(rows)]) == d, rows
    for rows in itertools.combinations(range(n), k):
        assert _rank(Psi[list(rows), :k]) == k, rows


def test_mbr_parity_rows_are_sparse():
    """Each parity row touches only column j of M: d symbols for j < k, k for
    j >= k (the paper's "naturally sparse" MBR encode, Sec. 4.2)."""
    n, k, d = 16, 8, 14
    a, B = O.mbr_params(n, k, d)
    G = O.mbr_generator(n, k, d)
    for i in range(k, n):
        for j in range(a):
            assert int((G[a * i + j] != 0).sum()) == (d if j < k else k)


def _repair_ok(n, k, d, X, Y, f, H):
    a = d
    sent = np.stack([O.mbr_repair_helper(n, k, d, f, Y[a * h:a * h + a]) for h in H])
    got = O.mbr_repair_newcomer(n, k, d, f, H, sent)
    return np.array_equal(got, Y[a * f:a * f + a])


@pytest.mark.parametrize("n,k,d", CASES)
def test_mbr_repair_every_node_every_helper_set(n, k, d):
    a, B = O.mbr_params(n, k, d)
    X = np.random.default_rng(3).integers(0, 256, (B, 4), dtype=np.uint8)
    Y = O.mbr_encode(n, k, d, X)
    for f in range(n):
        others = [h for h in range(n) if h != f]
        for H in itertools.combinations(others, d):
            assert _repair_ok(n, k, d, X, Y, f, list(H)), (f, H)


@pytest.mark.parametrize("n,k,d", CASES)
def test_mbr_decode_every_k_subset(n, k, d):
    a, B = O.mbr_params(n, k, d)
    X = np.random.default_rng(4).integers(0, 256, (B, 4), dtype=np.uint8)
    Y = O.mbr_encode(n, k, d, X)
    for S in itertools.combinations(range(n), k):
        rows = [a * i + j for i in S for j in range(a)]
        assert np.array_equal(O.mbr_decode(n, k, d, list(S), Y[rows]), X), S


def test_mbr_k8_sampled_repair_and_decode():
    n, k, d = 16, 8, 14
    a, B = O.mbr_params(n, k, d)
    X = np.random.default_rng(5).integers(0, 256, (B, 3), dtype=np.uint8)
    Y = O.mbr_encode(n, k, d, X)
    rng = np.random.default_rng(6)
    for _ in range(6):
        f = int(rng.integers(0, n))
        H = rng.permutation([h for h in range(n) if h != f])[:d].tolist()
        assert _repair_ok(n, k, d, X, Y, f, H)
    for _ in range(6):
        S = rng.permutation(rng.choice(n, k, replace=False)).tolist()
        rows = [a * i + j for i in S for j in range(a)]
        assert np.array_equal(O.mbr_decode(n, k, d, S, Y[rows]), X)
