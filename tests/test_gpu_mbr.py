"""GPU parity of the PM-MBR code (construction PMRC_MBR): encode, two-step
and fused repair, reconstruction (lazy), batched and served, called through
the C ABI and compared byte for byte with the CPU oracle."""
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


def mbr(n, k, d, form=P.PMRC_SYSTEMATIC):
    return P.Code(n, k, P.PMRC_MBR, form, d=d)


@pytest.mark.parametrize("form", [P.PMRC_SYSTEMATIC, P.PMRC_NONSYSTEMATIC])
@pytest.mark.parametrize("n,k,d", [(6, 3, 4), (8, 4, 7), (16, 8, 14), (32, 16, 30)])
def test_mbr_encode_matches_oracle(n, k, d, form):
    c = mbr(n, k, d, form)
    a, B = O.mbr_params(n, k, d)
    for nbytes, shift in ((3 * 4096 + 77, 0), (1000, 3), (1, 0)):
        X = inputs.blocks(B, nbytes, seed=nbytes + d)
        xin = Blocks(B, nbytes, shift, X)
        nout = (n - k) * a if form == P.PMRC_SYSTEMATIC else n * a
        yout = Blocks(nout, nbytes, shift)
        c.encode(xin.ptrs(), yout.ptrs(), nbytes)
        assert yout.guards_intact()
        Y = O.mbr_encode(n, k, d, X)
        want = Y[k * a:] if form == P.PMRC_SYSTEMATIC else Y
        assert np.array_equal(yout.get(), want), (nbytes, shift)


def _repair_two_step(c, f, H, Y, nbytes):
    a, d = c.alpha, c.d
    hin = Blocks(d * a, nbytes, 0, np.concatenate([Y[a * h:a * h + a] for h in H]))
    recv = Blocks(d, nbytes)
    out = Blocks(a, nbytes)
    c.repair_helpers(f, H, hin.ptrs(), recv.ptrs(), nbytes)
    c.repair_newcomer(f, H, recv.ptrs(), out.ptrs(), nbytes)
    fused = None
    if a <= 16:
        fo = Blocks(a, nbytes)
        c.repair(f, H, hin.ptrs(), fo.ptrs(), nbytes)
        assert fo.guards_intact()
        fused = fo.get()
    assert out.guards_intact()
    return out.get(), fused


@pytest.mark.parametrize("n,k,d", [(6, 3, 4), (8, 4, 6)])
def test_mbr_repair_every_node_every_helper_set(n, k, d):
    c = mbr(n, k, d)
    a, B = O.mbr_params(n, k, d)
    nbytes = 4096 + 33
    X = inputs.blocks(B, nbytes, seed=40)
    Y = O.mbr_encode(n, k, d, X)
    for f in range(n):
        for H in itertools.combinations([h for h in range(n) if h != f], d):
            two, fused = _repair_two_step(c, f, list(H), Y, nbytes)
            assert np.array_equal(two, Y[a * f:a * f + a]), (f, H)
            assert np.array_equal(fused, two), (f, H)


def test_mbr_repair_k8_every_node_and_k16_two_step():
    n, k, d = 16, 8, 14
    c = mbr(n, k, d)
    a, B = O.mbr_params(n, k, d)
    nbytes = 2 * 4096 + 5
    X = inputs.blocks(B, nbytes, seed=41)
    Y = O.mbr_encode(n, k, d, X)
    rng = np.random.default_rng(42)
    for f in range(n):
        H = rng.permutation([h for h in range(n) if h != f])[:d].tolist()
        two, fused = _repair_two_step(c, f, H, Y, nbytes)
        assert np.array_equal(two, Y[a * f:a * f + a]), f
        assert np.array_equal(fused, two), f
    c16 = mbr(32, 16, 30)
    a, B = O.mbr_params(32, 16, 30)
    X = inputs.blocks(B, 1000, seed=43)
    Y = O.mbr_encode(32, 16, 30, X)
    for f in (0, 20):
        H = c16.default_helpers(f)
        two, fused = _repair_two_step(c16, f, H, Y, 1000)
        assert fused is None                      # alpha = 30: two-step only
        assert np.array_equal(two, Y[a * f:a * f + a]), f


def _decode(c, S, Y, nbytes, alias=False):
    a, K = c.alpha, c.data_blocks
    rows = [a * i + j for i in S for j in range(a)]
    yin = Blocks(len(rows), nbytes, 0, Y[rows])
    xout = Blocks(K, nbytes)
    ptrs = xout.ptrs()
    if alias:   # data blocks held verbatim by a listed node stay in place
        L = O.mbr_index_matrix(c.k, c.d)
        for pos, i in enumerate(S):
            if i < c.k:
                for j in range(a):
                    ptrs[int(L[i, j])] = yin.ptr(a * pos + j)
    c.decode(S, yin.ptrs(), ptrs, nbytes)
    assert xout.guards_intact()
    return xout.get(), ptrs, xout


def test_mbr_decode_every_subset_small_and_random_k8():
    for (n, k, d) in ((6, 3, 4), (7, 3, 5)):
        c = mbr(n, k, d)
        a, B = O.mbr_params(n, k, d)
        X = inputs.blocks(B, 4096 + 7, seed=44)
        Y = O.mbr_encode(n, k, d, X)
        for S in itertools.combinations(range(n), k):
            got, _, _ = _decode(c, list(S), Y, 4096 + 7)
            assert np.array_equal(got, X), S
    n, k, d = 16, 8, 14
    c = mbr(n, k, d)
    a, B = O.mbr_params(n, k, d)
    X = inputs.blocks(B, 3 * 4096 + 1, seed=45)
    Y = O.mbr_encode(n, k, d, X)
    rng = np.random.default_rng(46)
    for _ in range(8):
        S = rng.permutation(rng.choice(n, k, replace=False)).tolist()
        got, _, _ = _decode(c, S, Y, 3 * 4096 + 1)
        assert np.array_equal(got, X), S


def test_mbr_lazy_decode_leaves_aliased_blocks():
    n, k, d = 16, 8, 14
    c = mbr(n, k, d)
    a, B = O.mbr_params(n, k, d)
    X = inputs.blocks(B, 4096 + 3, seed=47)
    Y = O.mbr_encode(n, k, d, X)
    S = [0, 3, 9, 12, 5, 15, 7, 10]
    got, ptrs, xout = _decode(c, S, Y, 4096 + 3, alias=True)
    base = xout.ptrs()
    for r in range(B):
        if ptrs[r] == base[r]:
            assert np.array_equal(got[r], X[r]), r   # computed
        else:
            assert (got[r] == 0xA5).all(), r        # left to the alias


def test_mbr_full_size_k8_sampled_columns():
    n, k, d = 16, 8, 14
    c = mbr(n, k, d)
    a, B = O.mbr_params(n, k, d)
    nb = 1 << 20
    X = inputs.device_blocks(B, nb, seed=48)
    Y = torch.empty((n * a, nb), dtype=torch.uint8, device="cuda")
    cn = mbr(n, k, d, P.PMRC_NONSYSTEMATIC)
    cn.encode([X[i] for i in range(B)], [Y[r] for r in range(n * a)], nb)
    f = 11
    H = c.default_helpers(f)
    node = torch.empty((a, nb), dtype=torch.uint8, device="cuda")
    c.repair(f, H, [Y[a * h + j] for h in H for j in range(a)], [node[j] for j in range(a)], nb)
    S = inputs.node_subset(n, k, seed=48)
    Xr = torch.empty((B, nb), dtype=torch.uint8, device="cuda")
    c.decode(S, [Y[a * i + j] for i in S for j in range(a)], [Xr[r] for r in range(B)], nb)
    torch.cuda.synchronize()
    cols = np.random.default_rng(49).choice(nb, 1024, replace=False)
    Xs = X.cpu().numpy()[:, cols]
    Ys = O.mbr_encode(n, k, d, np.ascontiguousarray(Xs))
    assert np.array_equal(Y.cpu().numpy()[:, cols], Ys)
    assert np.array_equal(node.cpu().numpy()[:, cols], Ys[a * f:a * f + a])
    assert np.array_equal(Xr.cpu().numpy()[:, cols], Xs)


def test_mbr_batched_and_served():
    n, k, d = 8, 4, 6
    c = mbr(n, k, d)
    a, B = O.mbr_params(n, k, d)
    nb = 3 * 4096 + 16
    X = inputs.blocks(B, nb, seed=50)
    Y = O.mbr_encode(n, k, d, X)
    xin = Blocks(B, nb, 0, X)
    par = Blocks((n - k) * a, nb)
    f, H = 5, c.default_helpers(5)
    hin = Blocks(d * a, nb, 0, np.concatenate([Y[a * h:a * h + a] for h in H]))
    node = Blocks(a, nb)
    S = [7, 1, 4, 6]
    din = Blocks(k * a, nb, 0, Y[[a * i + j for i in S for j in range(a)]])
    dout = Blocks(B, nb)
    b = P.Batch()
    b.add_encode(c, xin.ptrs(), par.ptrs(), nb)
    b.add_repair(c, f, H, hin.ptrs(), node.ptrs(), nb)
    b.add_decode(c, S, din.ptrs(), dout.ptrs(), nb)
    b.build()
    b.launch()
    assert np.array_equal(par.get(), Y[k * a:])
    assert np.array_equal(node.get(), Y[a * f:a * f + a])
    assert np.array_equal(dout.get(), X)

    srv = P.Server(budget_bytes=64 << 20, max_slots=8)
    pin = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).pin_memory()  # noqa: E731
    q_in = [pin(X), pin(np.concatenate([Y[a * h:a * h + a] for h in H])),
            pin(Y[[a * i + j for i in S for j in range(a)]])]
    q_out = [torch.zeros(((n - k) * a, nb), dtype=torch.uint8).pin_memory(),
             torch.zeros((a, nb), dtype=torch.uint8).pin_memory(),
             torch.zeros((B, nb), dtype=torch.uint8).pin_memory()]
    ids = [srv.submit(P.PMRC_OP_ENCODE, c, nb, q_in[0], q_out[0]),
           srv.submit(P.PMRC_OP_REPAIR, c, nb, q_in[1], q_out[1], failed=f, helpers=H),
           srv.submit(P.PMRC_OP_DECODE, c, nb, q_in[2], q_out[2], nodes=S)]
    for rid in ids:
        assert srv.wait(rid, timeout_ms=30000)[0] == P.PMRC_OK
    assert np.array_equal(q_out[0].numpy(), Y[k * a:])
    assert np.array_equal(q_out[1].numpy(), Y[a * f:a * f + a])
    assert np.array_equal(q_out[2].numpy(), X)
    srv.close()


def test_mbr_bitsliced_encode_matches_generic_and_oracle():
    n, k, d = 16, 8, 14
    c = mbr(n, k, d)
    a, B = O.mbr_params(n, k, d)
    nbytes = 64 * 1024 + 32 + 7          # bitsliced body plus a ragged tail
    X = inputs.blocks(B, nbytes, seed=51)
    xin = Blocks(B, nbytes, 0, X)
    outs = {}
    for which in (P.PMRC_KERNEL_BITSLICED, P.PMRC_KERNEL_GENERIC):
        c.set_encode_kernel(which)
        y = Blocks((n - k) * a, nbytes)
        c.encode(xin.ptrs(), y.ptrs(), nbytes)
        assert y.guards_intact()
        outs[which] = y.get()
    c.set_encode_kernel(P.PMRC_KERNEL_AUTO)
    assert np.array_equal(outs[P.PMRC_KERNEL_BITSLICED], outs[P.PMRC_KERNEL_GENERIC])
    assert np.array_equal(outs[P.PMRC_KERNEL_BITSLICED], O.mbr_encode(n, k, d, X)[k * a:])
