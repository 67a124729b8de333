"""GPU parity of the GF(2^16) variant (pmrc_create_field(..., 16)): encode,
repair (helper projections + newcomer) and decode through the C ABI, on
blocks of two byte planes, byte for byte against the CPU oracle."""
import itertools

import numpy as np
import pytest

import oracle as O
import paper_1412_3022_gb300 as P
from paper_1412_3022_gb300 import inputs
from test_gpu_parity import Blocks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.mark.parametrize("form", [P.PMRC_NONSYSTEMATIC, P.PMRC_SYSTEMATIC])
@pytest.mark.parametrize("cons", [P.PMRC_VANILLA, P.PMRC_SPARSE])
@pytest.mark.parametrize("n,k", [(6, 3), (8, 4), (16, 8)])
def test_gf16_encode_matches_oracle(n, k, cons, form):
    c = P.Code(n, k, cons, form, field_bits=16)
    a, K = k - 1, k * (k - 1)
    for nbytes, shift in ((3 * 8192 + 78, 0), (1000, 2), (2, 0)):
        X = inputs.blocks(K, nbytes, seed=nbytes + 7 * k)
        xin = Blocks(K, nbytes, shift, X)
        nout = (n - k) * a if form else n * a
        y = Blocks(nout, nbytes, shift)
        c.encode(xin.ptrs(), y.ptrs(), nbytes)
        assert y.guards_intact()
        Y = O.gf16_encode(n, k, cons, bool(form), X)
        assert np.array_equal(y.get(), Y[K:] if form else Y), (nbytes, shift)


def test_gf16_vanilla_k16_systematic_encode():
    n, k = 32, 16
    c = P.Code(n, k, P.PMRC_VANILLA, P.PMRC_SYSTEMATIC, field_bits=16)
    K, nbytes = 240, 4096 + 2
    X = inputs.blocks(K, nbytes, seed=70)
    xin = Blocks(K, nbytes, 0, X)
    y = Blocks(K, nbytes)
    c.encode(xin.ptrs(), y.ptrs(), nbytes)
    assert np.array_equal(y.get(), O.gf16_encode(n, k, O.VANILLA, True, X)[K:])


def _repair(c, f, H, Y, nbytes):
    a, d = c.alpha, c.d
    hin = Blocks(d * a, nbytes, 0, np.concatenate([Y[a * h:a * h + a] for h in H]))
    recv = Blocks(d, nbytes)
    out = Blocks(a, nbytes)
    c.repair_helpers(f, H, hin.ptrs(), recv.ptrs(), nbytes)
    c.repair_newcomer(f, H, recv.ptrs(), out.ptrs(), nbytes)
    assert recv.guards_intact() and out.guards_intact()
    return out.get()


@pytest.mark.parametrize("cons", [P.PMRC_VANILLA, P.PMRC_SPARSE])
def test_gf16_repair_every_node_and_helper_set_k3(cons):
    n, k, nbytes = 6, 3, 4096 + 10
    c = P.Code(n, k, cons, P.PMRC_SYSTEMATIC, field_bits=16)
    a = k - 1
    X = inputs.blocks(k * a, nbytes, seed=71)
    Y = O.gf16_encode(n, k, cons, True, X)
    done = 0
    for f in range(n):
        for H in itertools.combinations([h for h in range(n) if h != f], 2 * k - 2):
            try:
                got = _repair(c, f, list(H), Y, nbytes)
            except P.PMRCError as e:
                assert e.rc == P.PMRC_ESINGULAR and cons == P.PMRC_SPARSE
                continue
            assert np.array_equal(got, Y[a * f:a * f + a]), (f, H)
            done += 1
    assert done > 0


def test_gf16_repair_k8_every_node():
    n, k, nbytes = 16, 8, 2 * 8192 + 4
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC, field_bits=16)
    a = k - 1
    X = inputs.blocks(k * a, nbytes, seed=72)
    Y = O.gf16_encode(n, k, O.SPARSE, True, X)
    for f in range(n):
        got = _repair(c, f, c.default_helpers(f), Y, nbytes)
        assert np.array_equal(got, Y[a * f:a * f + a]), f


@pytest.mark.parametrize("form", [P.PMRC_NONSYSTEMATIC, P.PMRC_SYSTEMATIC])
def test_gf16_decode_subsets(form):
    for (n, k, nbytes, sub) in ((6, 3, 4096 + 6, None), (16, 8, 3 * 8192 + 2, 6)):
        c = P.Code(n, k, P.PMRC_SPARSE, form, field_bits=16)
        a, K = k - 1, k * (k - 1)
        X = inputs.blocks(K, nbytes, seed=73 + k)
        Y = O.gf16_encode(n, k, O.SPARSE, bool(form), X)
        subsets = list(itertools.combinations(range(n), k))
        if sub:
            rng = np.random.default_rng(74)
            subsets = [rng.permutation(rng.choice(n, k, replace=False)).tolist() for _ in range(sub)]
        for S in subsets:
            S = list(S)
            rows = [a * i + j for i in S for j in range(a)]
            yin = Blocks(K, nbytes, 0, Y[rows])
            xout = Blocks(K, nbytes)
            ptrs = xout.ptrs()
            if form:   # lazy: present data blocks stay where they are
                for pos, i in enumerate(S):
                    if i < k:
                        for j in range(a):
                            ptrs[a * i + j] = yin.ptr(a * pos + j)
            c.decode(S, yin.ptrs(), ptrs, nbytes)
            assert xout.guards_intact()
            got = xout.get()
            for r in range(K):
                if ptrs[r] == xout.ptr(r):
                    assert np.array_equal(got[r], X[r]), (S, r)
