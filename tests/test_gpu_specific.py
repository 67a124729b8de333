"""GPU parity of the "specific" product-matrix algorithms (the data collector
and the systematic encode by decoding then encoding), called through the C
ABI, against the CPU oracle and the data itself.  Integer work: bit-exact."""
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


def workspace(c, nbytes):
    nb = c.specific_workspace_bytes(nbytes)
    return torch.full((nb,), 0x5A, dtype=torch.uint8, device="cuda"), nb


def decode_specific(c, S, Y, nbytes, shift=0, out_null=None):
    a, K = c.alpha, c.k * c.alpha
    rows = [a * i + j for i in S for j in range(a)]
    yin = Blocks(K, nbytes, shift, Y[rows])
    xout = Blocks(K, nbytes, shift)
    ptrs = xout.ptrs()
    if out_null is not None:
        for r in out_null:
            ptrs[r] = None
    ws, nb = workspace(c, nbytes)
    c.decode_specific(S, yin.ptrs(), ptrs, nbytes, ws, nb)
    assert xout.guards_intact()
    return xout.get()


@pytest.mark.parametrize("form", [P.PMRC_NONSYSTEMATIC, P.PMRC_SYSTEMATIC])
@pytest.mark.parametrize("cons", [P.PMRC_VANILLA, P.PMRC_SPARSE])
def test_data_collector_every_subset_k3(cons, form):
    n, k, B = 6, 3, 3 * 4096 + 77
    c = P.Code(n, k, cons, form)
    X = inputs.blocks(k * (k - 1), B, seed=31)
    Y = O.encode(n, k, cons, bool(form), X)
    for S in itertools.combinations(range(n), k):
        S = list(S)
        got = decode_specific(c, S, Y, B)
        assert np.array_equal(got, X), S


@pytest.mark.parametrize("cons,form", [(P.PMRC_SPARSE, P.PMRC_SYSTEMATIC),
                                       (P.PMRC_VANILLA, P.PMRC_NONSYSTEMATIC),
                                       (P.PMRC_SPARSE, P.PMRC_NONSYSTEMATIC)])
def test_data_collector_k8_random_subsets_match_oracle(cons, form):
    n, k, B = 16, 8, 2 * 4096 + 13
    c = P.Code(n, k, cons, form)
    X = inputs.blocks(56, B, seed=32)
    Y = O.encode(n, k, cons, bool(form), X)
    rng = np.random.default_rng(33)
    for t in range(5):
        S = rng.permutation(rng.choice(n, k, replace=False)).tolist()
        got = decode_specific(c, S, Y, B, shift=t % 3)
        a = k - 1
        want = O.decode_specific(n, k, cons, bool(form), S, Y[[a * i + j for i in S for j in range(a)]])
        assert np.array_equal(want, X)
        assert np.array_equal(got, X), S


def test_data_collector_k16_and_full_size_k8():
    c16 = P.Code(32, 16, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    X = inputs.blocks(240, 4096 + 5, seed=34)
    Y = O.encode(32, 16, P.PMRC_SPARSE, True, X)
    for S in (list(range(16, 32)), [0, 31, 2, 29, 4, 27, 6, 25, 8, 23, 10, 21, 12, 19, 14, 17]):
        assert np.array_equal(decode_specific(c16, S, Y, 4096 + 5), X), S
    # n=16 k=8 at 1 MiB blocks, checked on sampled byte columns
    c = P.Code(16, 8, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    B = 1 << 20
    Xd = inputs.device_blocks(56, B, seed=35)
    Yd = torch.empty((112, B), dtype=torch.uint8, device="cuda")
    Yd[:56].copy_(Xd)
    c.encode([Xd[i] for i in range(56)], [Yd[56 + i] for i in range(56)], B)
    S = inputs.node_subset(16, 8, seed=35)
    ins = [Yd[7 * i + j] for i in S for j in range(7)]
    out = torch.empty((56, B), dtype=torch.uint8, device="cuda")
    ws, nb = workspace(c, B)
    c.decode_specific(S, ins, [out[r] for r in range(56)], B, ws, nb)
    torch.cuda.synchronize()
    cols = np.random.default_rng(36).choice(B, 2048, replace=False)
    assert np.array_equal(out.cpu().numpy()[:, cols], Xd.cpu().numpy()[:, cols])


def test_data_collector_lazy_null_and_copied_rows():
    """Aliased systematic rows stay in place, NULL rows are not written,
    present rows that are not aliased are copied."""
    n, k, B = 8, 4, 4096 + 9
    a, K = k - 1, k * (k - 1)
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    X = inputs.blocks(K, B, seed=37)
    Y = O.encode(n, k, P.PMRC_SPARSE, True, X)
    S = [1, 6, 3, 7]                                # data nodes 1 and 3 present
    rows = [a * i + j for i in S for j in range(a)]
    yin = Blocks(K, B, 0, Y[rows])
    xout = Blocks(K, B)
    ptrs = xout.ptrs()
    in_ptrs = yin.ptrs()
    for j in range(a):                              # node 1 aliased in place
        ptrs[a * 1 + j] = in_ptrs[a * 0 + j]
    ptrs[a * 0 + 1] = None                          # one missing row not wanted
    ws, nb = workspace(c, B)
    c.decode_specific(S, in_ptrs, ptrs, B, ws, nb)
    got = xout.get()
    for r in range(K):
        if r == a * 0 + 1 or r // a == 1:
            assert (got[r] == 0xA5).all(), r        # untouched
        else:
            assert np.array_equal(got[r], X[r]), r  # copied (node 3) or decoded
    assert np.array_equal(yin.get(), Y[rows])       # inputs unchanged


@pytest.mark.parametrize("n,k,cons", [(6, 3, P.PMRC_VANILLA), (6, 3, P.PMRC_SPARSE),
                                      (8, 4, P.PMRC_SPARSE), (16, 8, P.PMRC_SPARSE),
                                      (16, 8, P.PMRC_VANILLA), (32, 16, P.PMRC_SPARSE)])
def test_precode_encode_equals_oracle_and_linear_encode(n, k, cons):
    a, K = k - 1, k * (k - 1)
    B = 2 * 4096 + 3
    c = P.Code(n, k, cons, P.PMRC_SYSTEMATIC)
    X = inputs.blocks(K, B, seed=38 + k)
    xin = Blocks(K, B, 1, X)
    par = Blocks((n - k) * a, B, 1)
    lin = Blocks((n - k) * a, B, 1)
    ws, nb = workspace(c, B)
    c.encode_precode(xin.ptrs(), par.ptrs(), B, ws, nb)
    c.encode(xin.ptrs(), lin.ptrs(), B)
    assert par.guards_intact()
    got = par.get()
    assert np.array_equal(got, lin.get())
    assert np.array_equal(got, O.encode_precode(n, k, cons, X))


def test_specific_argument_errors():
    c = P.Code(8, 4, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    cn = P.Code(8, 4, P.PMRC_SPARSE, P.PMRC_NONSYSTEMATIC)
    B = 4096
    blocks = Blocks(12, B)
    ws, nb = workspace(c, B)
    assert c.specific_workspace_bytes(B) == (max(12, 18) + 12 + 12) * 4096
    with pytest.raises(P.PMRCError) as e:
        c.decode_specific([0, 1, 2, 3], blocks.ptrs(), blocks.ptrs(), B, ws, nb - 1)
    assert e.value.rc == P.PMRC_EINVAL
    with pytest.raises(P.PMRCError) as e:
        c.decode_specific([0, 1, 2, 2], blocks.ptrs(), blocks.ptrs(), B, ws, nb)
    assert e.value.rc == P.PMRC_EINVAL
    with pytest.raises(P.PMRCError) as e:
        cn.encode_precode(blocks.ptrs(), blocks.ptrs(), B, ws, nb)
    assert e.value.rc == P.PMRC_EINVAL
