"""Pins of the oracle's Reed-Solomon baseline (the paper's comparison code,
Sec. 4) against the definitions: non-systematic codeword symbols are the
message polynomial evaluated at g^i (Horner with an independent multiply);
the systematic form has the identity on top (Sec. 3.2); the code is MDS
(every k-subset decodes, every node repairs from any k others)."""
import itertools

import numpy as np
import pytest

import oracle as O


def mul(a, b):
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        if a & 0x100:
            a ^= 0x11D
        b >>= 1
    return r


def gpow(e):
    r = 1
    for _ in range(e):
        r = mul(r, 2)
    return r


@pytest.mark.parametrize("n,k", [(6, 3), (9, 6), (16, 8)])
def test_rs_is_polynomial_evaluation(n, k):
    Z = np.random.default_rng(1).integers(0, 256, (k, 4), dtype=np.uint8)
    Y = O.rs_encode(n, k, False, Z)
    for t in range(Z.shape[1]):
        for i in range(n):
            x, acc = gpow(i), 0
            for j in reversed(range(k)):          # Horner
                acc = mul(acc, x) ^ int(Z[j, t])
            assert Y[i, t] == acc, (i, t)


@pytest.mark.parametrize("n,k", [(6, 3), (16, 8), (32, 16)])
def test_rs_systematic_top_is_identity(n, k):
    G = O.rs_generator(n, k, True)
    assert np.array_equal(G[:k], np.eye(k, dtype=np.uint8))
    X = np.random.default_rng(2).integers(0, 256, (k, 5), dtype=np.uint8)
    assert np.array_equal(O.rs_encode(n, k, True, X)[:k], X)


@pytest.mark.parametrize("systematic", [False, True])
@pytest.mark.parametrize("n,k", [(5, 2), (6, 3), (8, 4)])
def test_rs_mds_every_subset_and_every_repair(n, k, systematic):
    X = np.random.default_rng(3).integers(0, 256, (k, 6), dtype=np.uint8)
    Y = O.rs_encode(n, k, systematic, X)
    for S in itertools.combinations(range(n), k):
        assert np.array_equal(O.rs_decode(n, k, systematic, list(S), Y[list(S)]), X), S
    for f in range(n):
        for H in itertools.combinations([h for h in range(n) if h != f], k):
            got = O.rs_repair(n, k, systematic, f, list(H), Y[list(H)])
            assert np.array_equal(got, Y[f]), (f, H)


def test_rs_k8_sampled():
    n, k = 16, 8
    X = np.random.default_rng(4).integers(0, 256, (k, 3), dtype=np.uint8)
    Y = O.rs_encode(n, k, True, X)
    rng = np.random.default_rng(5)
    for _ in range(10):
        S = rng.permutation(rng.choice(n, k, replace=False)).tolist()
        assert np.array_equal(O.rs_decode(n, k, True, S, Y[S]), X)
        f = int(rng.integers(0, n))
        H = rng.permutation([h for h in range(n) if h != f])[:k].tolist()
        assert np.array_equal(O.rs_repair(n, k, True, f, H, Y[H]), Y[f])
