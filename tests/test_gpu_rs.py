"""GPU parity of the Reed-Solomon baseline (construction PMRC_RS, Sec. 4):
encode (bitsliced and generic), repair from k helpers (two-step and fused),
decode, through the C ABI, byte for byte against the CPU oracle."""
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


@pytest.mark.parametrize("form", [P.PMRC_SYSTEMATIC, P.PMRC_NONSYSTEMATIC])
@pytest.mark.parametrize("n,k", [(6, 3), (16, 8), (32, 16)])
def test_rs_encode_matches_oracle(n, k, form):
    c = P.Code(n, k, P.PMRC_RS, form)
    for nbytes, shift in ((3 * 4096 + 77, 0), (64 * 1024 + 32, 0), (999, 5)):
        X = inputs.blocks(k, nbytes, seed=nbytes + k)
        xin = Blocks(k, nbytes, shift, X)
        nout = n - k if form == P.PMRC_SYSTEMATIC else n
        y = Blocks(nout, nbytes, shift)
        c.encode(xin.ptrs(), y.ptrs(), nbytes)
        assert y.guards_intact()
        Y = O.rs_encode(n, k, bool(form), X)
        assert np.array_equal(y.get(), Y[k:] if form == P.PMRC_SYSTEMATIC else Y), nbytes


def test_rs_bitsliced_matches_generic():
    c = P.Code(16, 8, P.PMRC_RS, P.PMRC_SYSTEMATIC)
    nbytes = 128 * 1024 + 40
    X = inputs.blocks(8, nbytes, seed=60)
    xin = Blocks(8, nbytes, 0, X)
    outs = []
    for which in (P.PMRC_KERNEL_BITSLICED, P.PMRC_KERNEL_GENERIC):
        c.set_encode_kernel(which)
        y = Blocks(8, nbytes)
        c.encode(xin.ptrs(), y.ptrs(), nbytes)
        outs.append(y.get())
    c.set_encode_kernel(P.PMRC_KERNEL_AUTO)
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], O.rs_encode(16, 8, True, X)[8:])


def _repair(c, f, H, Y, nbytes):
    k = c.k
    hin = Blocks(k, nbytes, 0, Y[H])
    recv = Blocks(k, nbytes)
    out = Blocks(1, nbytes)
    c.repair_helpers(f, H, hin.ptrs(), recv.ptrs(), nbytes)
    c.repair_newcomer(f, H, recv.ptrs(), out.ptrs(), nbytes)
    fo = Blocks(1, nbytes)
    c.repair(f, H, hin.ptrs(), fo.ptrs(), nbytes)
    assert out.guards_intact() and fo.guards_intact()
    return out.get()[0], fo.get()[0]


def test_rs_repair_every_node_every_helper_set_and_k8():
    n, k, nbytes = 6, 3, 4096 + 11
    c = P.Code(n, k, P.PMRC_RS, P.PMRC_SYSTEMATIC)
    X = inputs.blocks(k, nbytes, seed=61)
    Y = O.rs_encode(n, k, True, X)
    for f in range(n):
        for H in itertools.combinations([h for h in range(n) if h != f], k):
            two, fused = _repair(c, f, list(H), Y, nbytes)
            assert np.array_equal(two, Y[f]) and np.array_equal(fused, Y[f]), (f, H)
    n, k, nbytes = 16, 8, 2 * 4096 + 3
    c = P.Code(n, k, P.PMRC_RS, P.PMRC_SYSTEMATIC)
    X = inputs.blocks(k, nbytes, seed=62)
    Y = O.rs_encode(n, k, True, X)
    rng = np.random.default_rng(63)
    for f in range(n):
        H = rng.permutation([h for h in range(n) if h != f])[:k].tolist()
        two, fused = _repair(c, f, H, Y, nbytes)
        assert np.array_equal(two, Y[f]) and np.array_equal(fused, Y[f]), f


def test_rs_decode_every_subset_and_full_size():
    n, k, nbytes = 6, 3, 4096 + 7
    c = P.Code(n, k, P.PMRC_RS, P.PMRC_SYSTEMATIC)
    X = inputs.blocks(k, nbytes, seed=64)
    Y = O.rs_encode(n, k, True, X)
    for S in itertools.combinations(range(n), k):
        yin = Blocks(k, nbytes, 0, Y[list(S)])
        xout = Blocks(k, nbytes)
        c.decode(list(S), yin.ptrs(), xout.ptrs(), nbytes)
        assert xout.guards_intact()
        assert np.array_equal(xout.get(), X), S
    n, k, nb = 16, 8, 7 << 20
    c = P.Code(n, k, P.PMRC_RS, P.PMRC_SYSTEMATIC)
    Xd = inputs.device_blocks(k, nb, seed=65)
    Yd = torch.empty((n, nb), dtype=torch.uint8, device="cuda")
    Yd[:k].copy_(Xd)
    c.encode([Xd[i] for i in range(k)], [Yd[k + i] for i in range(n - k)], nb)
    S = inputs.node_subset(n, k, seed=65)
    out = torch.empty((k, nb), dtype=torch.uint8, device="cuda")
    c.decode(S, [Yd[i] for i in S], [out[r] for r in range(k)], nb)
    torch.cuda.synchronize()
    cols = np.random.default_rng(66).choice(nb, 2048, replace=False)
    Xs = Xd.cpu().numpy()[:, cols]
    assert np.array_equal(Yd.cpu().numpy()[:, cols], O.rs_encode(n, k, True, np.ascontiguousarray(Xs)))
    assert np.array_equal(out.cpu().numpy()[:, cols], Xs)
