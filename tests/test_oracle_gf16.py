"""Pins of the oracle's GF(2^16) variant (Sec. 3.3 checks the sparse
construction in GF(2^16) for k up to 64) against facts fixed by the field's
definition and by the mathematics of the code: the quadratic extension
GF(2^8)[y]/(y^2 + y + w) is a field (w has trace 1, so the polynomial has no
root), the oracle's table multiply equals the extension's multiplication
rule computed here with an independent shift-and-reduce GF(2^8) multiply,
g has order exactly 65535; the code built over it is linearized exactly,
repairs every node from every helper set and decodes from every k-subset."""
import itertools

import numpy as np
import pytest

import oracle as O


def mul8(a, b):
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        if a & 0x100:
            a ^= 0x11D
        b >>= 1
    return r


W = O.gf16_omega()


def mul16(x, z):
    a0, a1, b0, b1 = x & 255, x >> 8, z & 255, z >> 8
    hh = mul8(a1, b1)
    return (mul8(a0, b0) ^ mul8(W, hh)) | ((mul8(a1, b0) ^ mul8(a0, b1) ^ hh) << 8)


def test_extension_polynomial_is_irreducible():
    t, s = W, W
    for _ in range(7):
        t = mul8(t, t)
        s ^= t
    assert s == 1                                            # absolute trace 1
    assert all(mul8(y, y) ^ y ^ W for y in range(256))       # no root in GF(2^8)
    # w is the smallest element of trace 1
    for a in range(1, W):
        t, s = a, a
        for _ in range(7):
            t = mul8(t, t)
            s ^= t
        assert s == 0


def test_table_multiply_equals_extension_rule():
    rng = np.random.default_rng(1)
    xs = rng.integers(0, 65536, 4000)
    zs = rng.integers(0, 65536, 4000)
    for x, z in zip(xs.tolist(), zs.tolist()):
        assert O.gf16_mul(x, z) == mul16(x, z), (x, z)
    for x in (0, 1, 255, 256, 65535):
        for z in (0, 1, 2, 0x104, 65535):
            assert O.gf16_mul(x, z) == mul16(x, z)


def test_field_axioms_sampled_and_inverses():
    rng = np.random.default_rng(2)
    for x, y, z in rng.integers(0, 65536, (1500, 3)).tolist():
        assert mul16(x, y) == mul16(y, x)
        assert mul16(mul16(x, y), z) == mul16(x, mul16(y, z))
        assert mul16(x, y ^ z) == mul16(x, y) ^ mul16(x, z)
    for x in rng.integers(1, 65536, 3000).tolist():
        assert mul16(x, O.gf16_inv(x)) == 1


def test_generator_has_order_65535():
    g = O.gf16_primitive()
    p, order = 1, 0
    for i in range(1, 65536):
        p = mul16(p, g)
        if p == 1:
            order = i
            break
    assert order == 65535


@pytest.mark.parametrize("k", [2, 3, 8, 16, 32, 64])
def test_sparse_lambda_distinct_up_to_k64(k):
    """Sec. 3.3: in GF(2^16) the sparse construction is checked up to
    k = 64 (n = 2k - 1); its lambda values are distinct and its Cauchy
    points g^(i+alpha), g^(j-1) never collide."""
    n = 2 * k - 1
    phi, lam = O.gf16_phi_lambda(n, k, O.SPARSE)
    assert len(set(lam.tolist())) == n
    a = k - 1
    g = O.gf16_primitive()
    def gp(e):
        r = 1
        for _ in range(e):
            r = mul16(r, g)
        return r
    pts_x = [gp(i + a) for i in range(a + 1, n + 1)]
    pts_y = [gp(j - 1) for j in range(1, a + 1)]
    assert len(set(pts_x)) == len(pts_x) and not set(pts_x) & set(pts_y)


def test_vanilla_k16_n32_is_valid_in_gf16():
    """In GF(2^8) the vanilla code at k=16, n=32 repeats lambda; in GF(2^16)
    (65535 = 3 * 5 * 17 * 257) it does not."""
    phi, lam = O.gf16_phi_lambda(32, 16, O.VANILLA)
    assert len(set(lam.tolist())) == 32


@pytest.mark.parametrize("cons", [O.VANILLA, O.SPARSE])
@pytest.mark.parametrize("n,k", [(5, 3), (8, 4)])
def test_gf16_linearization_equals_product_form(n, k, cons):
    d, a = O.params(n, k)
    X = np.random.default_rng(3).integers(0, 256, (k * a, 6), dtype=np.uint8)
    Y = O.gf16_encode(n, k, cons, False, X)
    Psi = O.gf16_psi(n, k, cons)
    L = O.index_matrix(k)
    h = X.shape[1] // 2
    for t in range(h):
        sym = [int(X[r, t]) | (int(X[r, h + t]) << 8) for r in range(k * a)]
        for i in range(n):
            for j in range(a):
                acc = 0
                for l in range(d):
                    acc ^= mul16(int(Psi[i, l]), sym[L[l, j]])
                assert (int(Y[a * i + j, t]) | (int(Y[a * i + j, h + t]) << 8)) == acc


@pytest.mark.parametrize("systematic", [False, True])
@pytest.mark.parametrize("cons", [O.VANILLA, O.SPARSE])
@pytest.mark.parametrize("n,k", [(5, 3), (6, 3), (8, 4)])
def test_gf16_repair_and_decode_exhaustive(n, k, cons, systematic):
    d, a = O.params(n, k)
    X = np.random.default_rng(4).integers(0, 256, (k * a, 8), dtype=np.uint8)
    Y = O.gf16_encode(n, k, cons, systematic, X)
    if systematic:
        assert np.array_equal(Y[:k * a], X)
    tried = ok = 0
    for f in range(n):
        coef = O.gf16_helper_coefficients(n, k, cons, f)
        for H in itertools.combinations([h for h in range(n) if h != f], d):
            tried += 1
            try:
                D = O.gf16_newcomer_matrix(n, k, cons, f, list(H))
            except O.OracleError:
                # singular only for the sparse code at n = 2k, both left-out
                # nodes among the alpha identity rows
                left = [x for x in range(n) if x != f and x not in H]
                assert cons == O.SPARSE and n == 2 * k and all(x < a for x in left), (f, H)
                continue
            ok += 1
            sent = np.concatenate([O.gf16_region_apply(coef[None, :], Y[a * h:a * h + a])
                                   for h in H])
            assert np.array_equal(O.gf16_region_apply(D, sent), Y[a * f:a * f + a]), (f, H)
    assert ok > 0.8 * tried
    for S in itertools.combinations(range(n), k):
        R = O.gf16_decode_matrix(n, k, cons, systematic, list(S))
        rows = [a * i + j for i in S for j in range(a)]
        assert np.array_equal(O.gf16_region_apply(R, Y[rows]), X), S
