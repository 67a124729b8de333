"""Repairs through bitsliced kernels compiled at run time: the helper
projections (one kernel per failed node) and the fused repair (one kernel per
failed node and helper set), bit-exact against the CPU oracle, the stored
codeword and the split-table kernels.  Covers every failed node at n=16,
k=8 (both constructions, a helper that projects alpha blocks and one that
sends a stored block), k=3 and k=4, ragged block sizes (the tail runs on the
split-table kernels), single-helper calls, misaligned pointers (split-table
only), and the background compilation under AUTO."""
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


def stored(n, k, cons, nbytes, seed):
    X = inputs.blocks(k * (k - 1), nbytes, seed=seed)
    return O.encode(n, k, cons, True, X)


def helpers_gpu(c, f, H, Y, nbytes, shift=0):
    a = c.alpha
    hb = Blocks(len(H) * a, nbytes, shift, np.concatenate([Y[a * h:a * h + a] for h in H]))
    out = Blocks(len(H), nbytes, shift)
    c.repair_helpers(f, H, hb.ptrs(), out.ptrs(), nbytes)
    assert out.guards_intact()
    return out.get()


def fused_gpu(c, f, H, Y, nbytes, shift=0):
    a = c.alpha
    hb = Blocks(len(H) * a, nbytes, shift, np.concatenate([Y[a * h:a * h + a] for h in H]))
    out = Blocks(a, nbytes, shift)
    c.repair(f, H, hb.ptrs(), out.ptrs(), nbytes)
    assert out.guards_intact()
    return out.get()


@pytest.mark.parametrize("cons", [O.SPARSE, O.VANILLA])
def test_runtime_helpers_and_fused_every_node_k8(cons):
    n, k, a = 16, 8, 7
    nbytes = 3 * 1024 + 96 + 13          # four tiles, a partial tile and a ragged tail
    Y = stored(n, k, cons, nbytes, seed=300 + cons)
    c = P.Code(n, k, cons, P.PMRC_SYSTEMATIC)
    c.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    for f in range(n):
        H = c.default_helpers(f)
        sent = np.stack([O.repair_helper(n, k, cons, f, Y[a * h:a * h + a]) for h in H])
        assert np.array_equal(helpers_gpu(c, f, H, Y, nbytes), sent), f
        assert np.array_equal(fused_gpu(c, f, H, Y, nbytes), Y[a * f:a * f + a]), f


@pytest.mark.parametrize("n,k", [(6, 3), (8, 4), (5, 3)])
def test_runtime_fused_every_node_every_helper_order_small(n, k):
    a, d = k - 1, 2 * k - 2
    nbytes = 2048 + 32
    Y = stored(n, k, O.SPARSE, nbytes, seed=310 + n)
    c = P.Code(n, k, O.SPARSE, P.PMRC_SYSTEMATIC)
    c.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    rng = np.random.default_rng(n)
    for f in range(n):
        H = c.default_helpers(f)
        for order in (H, list(reversed(H)), rng.permutation(H).tolist()):
            try:
                got = fused_gpu(c, f, order, Y, nbytes)
            except P.PMRCError as e:   # singular helper sets are refused
                assert e.rc == P.PMRC_ESINGULAR
                continue
            assert np.array_equal(got, Y[a * f:a * f + a]), (f, order)
        assert len(H) == d


def test_runtime_single_helper_and_misaligned_fall_back():
    n, k, a = 16, 8, 7
    nbytes = 8192
    Y = stored(n, k, O.SPARSE, nbytes, seed=320)
    c = P.Code(n, k, O.SPARSE, P.PMRC_SYSTEMATIC)
    c.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    f = 12
    for h in (0, 15, 3):
        blocks = Blocks(a, nbytes, 0, Y[a * h:a * h + a])
        out = Blocks(1, nbytes)
        c.repair_helper(f, h, blocks.ptrs(), out.ptr(0), nbytes)
        assert np.array_equal(out.get()[0], O.repair_helper(n, k, O.SPARSE, f, Y[a * h:a * h + a]))
    H = c.default_helpers(f)
    sent = np.stack([O.repair_helper(n, k, O.SPARSE, f, Y[a * h:a * h + a]) for h in H])
    assert np.array_equal(helpers_gpu(c, f, H, Y, nbytes, shift=3), sent)
    assert np.array_equal(fused_gpu(c, f, H, Y, nbytes, shift=5), Y[a * f:a * f + a])


def test_runtime_repair_matches_split_table_at_1mib():
    """1 MiB blocks as benchmarked, both kernels on the same device data."""
    n, k, a = 16, 8, 7
    nbytes = 1 << 20
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    X = inputs.device_blocks(k * a, nbytes, seed=330)
    Y = torch.empty((n * a, nbytes), dtype=torch.uint8, device="cuda")
    Y[:k * a].copy_(X)
    c.encode([X[i] for i in range(k * a)], [Y[k * a + i] for i in range(k * a)], nbytes)
    outs = {}
    for which in (P.PMRC_KERNEL_BITSLICED, P.PMRC_KERNEL_GENERIC):
        c.set_decode_kernel(which)
        for f in (9, 2):
            H = c.default_helpers(f)
            hb = [Y[a * h + j] for h in H for j in range(a)]
            recv = torch.empty((len(H), nbytes), dtype=torch.uint8, device="cuda")
            c.repair_helpers(f, H, hb, [recv[i] for i in range(len(H))], nbytes)
            node = torch.empty((a, nbytes), dtype=torch.uint8, device="cuda")
            c.repair(f, H, hb, [node[j] for j in range(a)], nbytes)
            outs[(which, f)] = (recv, node)
    torch.cuda.synchronize()
    for f in (9, 2):
        rb, nb_ = outs[(P.PMRC_KERNEL_BITSLICED, f)]
        rg, ng = outs[(P.PMRC_KERNEL_GENERIC, f)]
        assert torch.equal(rb, rg) and torch.equal(nb_, ng)
        assert torch.equal(nb_, Y[a * f:a * f + a])
    # the bitsliced projections of f = 9 on every column, against the oracle
    f = 9
    H = c.default_helpers(f)
    Yh = Y.cpu().numpy()
    sent = np.stack([O.repair_helper(n, k, 1, f, Yh[a * h:a * h + a]) for h in H])
    assert np.array_equal(outs[(P.PMRC_KERNEL_BITSLICED, f)][0].cpu().numpy(), sent)


def test_auto_compiles_repair_kernels_in_the_background():
    n, k, a = 16, 8, 7
    nbytes = 512 << 10
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    X = inputs.device_blocks(k * a, nbytes, seed=340)
    Y = torch.empty((n * a, nbytes), dtype=torch.uint8, device="cuda")
    Y[:k * a].copy_(X)
    c.encode([X[i] for i in range(k * a)], [Y[k * a + i] for i in range(k * a)], nbytes)
    f = 13
    H = c.default_helpers(f)
    hb = [Y[a * h + j] for h in H for j in range(a)]
    nodes = []
    for _ in range(2):     # split-table kernel until the compilation ends, then bitsliced
        node = torch.empty((a, nbytes), dtype=torch.uint8, device="cuda")
        c.repair(f, H, hb, [node[j] for j in range(a)], nbytes)
        nodes.append(node)
        c.wait_kernels()
    ready, pending = c.runtime_kernels()
    assert pending == 0 and ready >= 1
    torch.cuda.synchronize()
    for node in nodes:
        assert torch.equal(node, Y[a * f:a * f + a])
