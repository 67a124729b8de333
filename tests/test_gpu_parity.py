"""GPU parity: every operation of libpmrc, called through its C ABI, against
the CPU oracle on the same seeded inputs.  Integer work, so the bar is
bit-exact equality.  Sizes span several 4 KiB tiles plus a ragged tail; the
full-size workloads are checked on sampled byte columns (every operation is
independent per byte column, so a column slice of the inputs run through the
oracle gives exactly those columns of the output)."""
import itertools

import numpy as np
import pytest

import oracle as O
import paper_1412_3022_gb300 as P
from paper_1412_3022_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

GUARD = 64


class Blocks:
    """`count` device blocks of `nbytes`, each at a 256-byte aligned row
    (plus `shift` bytes), with guard bytes after each block."""

    def __init__(self, count, nbytes, shift=0, fill=None):
        self.count, self.nbytes, self.shift = count, nbytes, shift
        self.stride = ((nbytes + shift + GUARD + 255) // 256) * 256
        self.buf = torch.full((max(count, 1), self.stride), 0xA5, dtype=torch.uint8, device="cuda")
        if fill is not None:
            self.set(fill)

    def set(self, arr):
        self.buf[:self.count, self.shift:self.shift + self.nbytes] = torch.from_numpy(
            np.ascontiguousarray(arr)).cuda()

    def ptrs(self):
        base = self.buf.data_ptr()
        return [base + i * self.stride + self.shift for i in range(self.count)]

    def ptr(self, i):
        return self.buf.data_ptr() + i * self.stride + self.shift

    def get(self):
        torch.cuda.synchronize()
        return self.buf[:self.count, self.shift:self.shift + self.nbytes].cpu().numpy()

    def guards_intact(self):
        torch.cuda.synchronize()
        b = self.buf.cpu().numpy()
        pre = b[:self.count, :self.shift]
        post = b[:self.count, self.shift + self.nbytes:]
        return bool((pre == 0xA5).all() and (post == 0xA5).all())


def code(n, k, cons, form):
    return P.Code(n, k, cons, form)


def run_encode(c, X, shift=0):
    K = c.k * c.alpha
    nbytes = X.shape[1]
    xin = Blocks(K, nbytes, shift, X)
    yout = Blocks(c.n_outputs, nbytes, shift)
    c.encode(xin.ptrs(), yout.ptrs(), nbytes)
    assert yout.guards_intact()
    return yout.get()


def oracle_outputs(n, k, cons, form, X):
    Y = O.encode(n, k, cons, bool(form), X)
    return Y[k * (k - 1):] if form else Y


# ------------------------------------------------------------------ encode
ENCODE_CASES = [(6, 3), (5, 3), (8, 4), (16, 8), (24, 12), (32, 16)]


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("cons", [0, 1])
@pytest.mark.parametrize("n,k", ENCODE_CASES)
def test_encode_parity(n, k, cons, form):
    if cons == 0 and k == 16:
        pytest.skip("vanilla k=16 n=32 is not an MSR code in GF(2^8)")
    nbytes = 3 * 4096 + 37
    X = inputs.blocks(k * (k - 1), nbytes, seed=100 + n * 10 + k + cons)
    c = code(n, k, cons, form)
    assert np.array_equal(run_encode(c, X), oracle_outputs(n, k, cons, form, X))


@pytest.mark.parametrize("nbytes", [1, 2, 15, 16, 17, 31, 4095, 4096, 4097, 65536 + 3])
def test_encode_odd_sizes(nbytes):
    n, k = 16, 8
    X = inputs.blocks(56, nbytes, seed=nbytes)
    c = code(n, k, 1, 1)
    assert np.array_equal(run_encode(c, X), oracle_outputs(n, k, 1, 1, X))


@pytest.mark.parametrize("shift", [1, 3, 4, 8, 15])
def test_encode_misaligned(shift):
    n, k = 16, 8
    X = inputs.blocks(56, 4096 + 100, seed=shift)
    c = code(n, k, 0, 0)
    assert np.array_equal(run_encode(c, X, shift), oracle_outputs(n, k, 0, 0, X))


def test_encode_zero_bytes_and_null_outputs():
    c = code(16, 8, 1, 1)
    xin = Blocks(56, 4096, 0, inputs.blocks(56, 4096, 1))
    yout = Blocks(56, 4096, 0)
    c.encode(xin.ptrs(), yout.ptrs(), 0)  # nothing happens
    assert (yout.get() == 0xA5).all()
    ptrs = yout.ptrs()
    ptrs[5] = 0
    c.encode(xin.ptrs(), ptrs, 4096)
    got = yout.get()
    want = oracle_outputs(16, 8, 1, 1, xin.get())
    assert (got[5] == 0xA5).all()
    assert np.array_equal(np.delete(got, 5, 0), np.delete(want, 5, 0))


def test_systematic_parity_is_a_codeword():
    """Data + parity from the GPU decode back to the data from any k nodes
    (oracle decode), and repair every node (oracle repair)."""
    n, k, a = 16, 8, 7
    X = inputs.blocks(k * a, 257, seed=9)
    Y = np.concatenate([X, run_encode(code(n, k, 1, 1), X)])
    for S in (list(range(8, 16)), [0, 3, 5, 8, 9, 11, 14, 15]):
        rows = [a * i + j for i in S for j in range(a)]
        assert np.array_equal(O.decode(n, k, 1, True, S, Y[rows]), X)


# ------------------------------------------------------------------ repair
def repair_gpu(c, Y, f, H, nbytes, batched=False):
    a = c.alpha
    store = Blocks(c.n * a, nbytes, 0, Y)
    recv = Blocks(len(H), nbytes)
    if batched:
        blocks = [store.ptr(a * h + j) for h in H for j in range(a)]
        c.repair_helpers(f, H, blocks, recv.ptrs(), nbytes)
    else:
        for i, h in enumerate(H):
            c.repair_helper(f, h, [store.ptr(a * h + j) for j in range(a)], recv.ptr(i), nbytes)
    out = Blocks(a, nbytes)
    c.repair_newcomer(f, H, recv.ptrs(), out.ptrs(), nbytes)
    assert recv.guards_intact() and out.guards_intact()
    return recv.get(), out.get()


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("cons", [0, 1])
def test_repair_k3_every_node_every_helper_set(cons, form):
    n, k, a, d = 6, 3, 2, 4
    nbytes = 4096 + 5
    X = inputs.blocks(k * a, nbytes, seed=31 + cons)
    Y = O.encode(n, k, cons, bool(form), X)
    c = code(n, k, cons, form)
    for f in range(n):
        for H in itertools.combinations([i for i in range(n) if i != f], d):
            H = list(H)
            try:
                O.newcomer_matrix(n, k, cons, f, H)
            except O.OracleError:
                with pytest.raises(P.PMRCError) as e:
                    repair_gpu(c, Y, f, H, nbytes)
                assert e.value.rc == P.PMRC_ESINGULAR
                continue
            sent, out = repair_gpu(c, Y, f, H, nbytes)
            want_sent = np.stack([O.repair_helper(n, k, cons, f, Y[a * h:a * h + a]) for h in H])
            assert np.array_equal(sent, want_sent)
            assert np.array_equal(out, O.repair_newcomer(n, k, cons, f, H, want_sent))
            assert np.array_equal(out, Y[a * f:a * f + a])


@pytest.mark.parametrize("cons", [0, 1])
def test_repair_k8_every_node(cons):
    n, k, a = 16, 8, 7
    nbytes = 2 * 4096 + 3
    X = inputs.blocks(k * a, nbytes, seed=77 + cons)
    Y = O.encode(n, k, cons, True, X)
    c = code(n, k, cons, 1)
    for f in range(n):
        H = c.default_helpers(f)
        sent, out = repair_gpu(c, Y, f, H, nbytes, batched=(f % 2 == 0))
        want_sent = np.stack([O.repair_helper(n, k, cons, f, Y[a * h:a * h + a]) for h in H])
        assert np.array_equal(sent, want_sent), f
        assert np.array_equal(out, Y[a * f:a * f + a]), f


def test_sparse_helper_reads_only_nonzero_blocks():
    """For a failed node among the alpha first, a sparse-code helper reads
    one block (Sec. 3.3): the other block pointers may be NULL."""
    n, k, a = 16, 8, 7
    nbytes = 4096
    X = inputs.blocks(k * a, nbytes, seed=5)
    Y = O.encode(n, k, 1, True, X)
    c = code(n, k, 1, 1)
    store = Blocks(n * a, nbytes, 0, Y)
    out = Blocks(1, nbytes)
    f, h = 2, 9
    blocks = [store.ptr(a * h + j) if j == f else 0 for j in range(a)]
    c.repair_helper(f, h, blocks, out.ptr(0), nbytes)
    assert np.array_equal(out.get()[0], O.repair_helper(n, k, 1, f, Y[a * h:a * h + a]))


# ------------------------------------------------------------------ decode
def decode_gpu(c, Y, S, nbytes, alias=False, null_rows=()):
    a = c.alpha
    K = c.k * a
    rows = [a * i + j for i in S for j in range(a)]
    nodes = Blocks(K, nbytes, 0, Y[rows])
    out = Blocks(K, nbytes)
    ptrs = out.ptrs()
    if alias:  # systematic blocks already in place stay where they are
        for pos, i in enumerate(S):
            if i < c.k:
                for j in range(a):
                    ptrs[a * i + j] = nodes.ptr(a * pos + j)
    for r in null_rows:
        ptrs[r] = 0
    c.decode(S, nodes.ptrs(), ptrs, nbytes)
    assert out.guards_intact() and nodes.guards_intact()
    got = out.get()
    if alias:
        nb = nodes.get()
        for pos, i in enumerate(S):
            if i < c.k:
                for j in range(a):
                    got[a * i + j] = nb[a * pos + j]
    return got, out


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("cons", [0, 1])
def test_decode_k3_every_subset(cons, form):
    n, k, a = 6, 3, 2
    nbytes = 4096 + 11
    X = inputs.blocks(k * a, nbytes, seed=55)
    Y = O.encode(n, k, cons, bool(form), X)
    c = code(n, k, cons, form)
    for S in itertools.combinations(range(n), k):
        got, _ = decode_gpu(c, Y, list(S), nbytes)
        assert np.array_equal(got, X), S


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("cons", [0, 1])
def test_decode_k8_random_subsets(cons, form):
    n, k, a = 16, 8, 7
    nbytes = 4096 + 700
    X = inputs.blocks(k * a, nbytes, seed=66)
    Y = O.encode(n, k, cons, bool(form), X)
    c = code(n, k, cons, form)
    for s in range(12):
        S = inputs.node_subset(n, k, seed=s)
        got, _ = decode_gpu(c, Y, S, nbytes, alias=bool(form and s % 2))
        assert np.array_equal(got, X), S


def test_decode_lazy_leaves_present_blocks_and_nulls():
    n, k, a = 16, 8, 7
    nbytes = 1000
    X = inputs.blocks(k * a, nbytes, seed=67)
    Y = O.encode(n, k, 1, True, X)
    c = code(n, k, 1, 1)
    S = [0, 2, 4, 6, 9, 10, 12, 15]
    got, out = decode_gpu(c, Y, S, nbytes, alias=True, null_rows=(7, 8))
    raw = out.get()
    assert (raw[7] == 0xA5).all() and (raw[8] == 0xA5).all()
    for r in range(k * a):
        if r not in (7, 8):
            assert np.array_equal(got[r], X[r]), r
    # blocks of data nodes present in S were not written into the output buffer
    assert (raw[0] == 0xA5).all()


# ------------------------------------------------------------------ full size
def columns(nbytes):
    w = 4096
    return [slice(0, w), slice(nbytes // 2 - 5, nbytes // 2 + w), slice(nbytes - w - 3, nbytes)]


@pytest.mark.parametrize("cons,form", [(1, 1), (0, 0), (0, 1), (1, 0)])
def test_full_size_k8_encode_sampled(cons, form):
    """n=16, k=8, 56 data blocks of 1 MiB, as benchmarked."""
    n, k, a = 16, 8, 7
    nbytes = 1 << 20
    X = inputs.device_blocks(k * a, nbytes, seed=2024)
    c = code(n, k, cons, form)
    Y = torch.empty((c.n_outputs, nbytes), dtype=torch.uint8, device="cuda")
    c.encode([X[i] for i in range(k * a)], [Y[i] for i in range(c.n_outputs)], nbytes)
    torch.cuda.synchronize()
    for cs in columns(nbytes):
        Xc = X[:, cs].cpu().numpy()
        assert np.array_equal(Y[:, cs].cpu().numpy(), oracle_outputs(n, k, cons, form, Xc))


@pytest.mark.parametrize("nbytes", [64 << 10, 1 << 20, 4 << 20])
def test_full_size_k8_repair_and_decode_sampled(nbytes):
    """n=16, k=8 sparse systematic: repair of a seeded failed node from its
    default helpers and reconstruction from a seeded 8-node subset."""
    n, k, a = 16, 8, 7
    c = code(n, k, 1, 1)
    X = inputs.device_blocks(k * a, nbytes, seed=nbytes)
    P_ = torch.empty(((n - k) * a, nbytes), dtype=torch.uint8, device="cuda")
    c.encode([X[i] for i in range(k * a)], [P_[i] for i in range(len(P_))], nbytes)
    Y = torch.cat([X, P_])
    f = inputs.failed_node(n, seed=nbytes)
    H = c.default_helpers(f)
    recv = torch.empty((len(H), nbytes), dtype=torch.uint8, device="cuda")
    c.repair_helpers(f, H, [Y[a * h + j] for h in H for j in range(a)],
                     [recv[i] for i in range(len(H))], nbytes)
    node = torch.empty((a, nbytes), dtype=torch.uint8, device="cuda")
    c.repair_newcomer(f, H, [recv[i] for i in range(len(H))], [node[j] for j in range(a)], nbytes)
    S = inputs.node_subset(n, k, seed=nbytes)
    Xd = torch.empty_like(X)
    c.decode(S, [Y[a * i + j] for i in S for j in range(a)], [Xd[r] for r in range(k * a)], nbytes)
    torch.cuda.synchronize()
    assert torch.equal(node, Y[a * f:a * f + a])
    assert torch.equal(Xd, X)
    for cs in columns(nbytes):
        Yc = Y[:, cs].cpu().numpy()
        sent = np.stack([O.repair_helper(n, k, 1, f, Yc[a * h:a * h + a]) for h in H])
        assert np.array_equal(recv[:, cs].cpu().numpy(), sent)
        assert np.array_equal(node[:, cs].cpu().numpy(), O.repair_newcomer(n, k, 1, f, H, sent))
        rows = [a * i + j for i in S for j in range(a)]
        assert np.array_equal(Xd[:, cs].cpu().numpy(), O.decode(n, k, 1, True, S, Yc[rows]))


def test_cfg1_small_code_end_to_end():
    """n=6, k=3 vanilla generator code, 4 KiB blocks: encode, repair of node
    0 from helpers {1,2,3,4}, reconstruction from nodes {1,2,3}."""
    n, k, a, nbytes = 6, 3, 2, 4096
    X = inputs.blocks(k * a, nbytes, seed=1)
    c = code(n, k, 0, 0)
    Y = run_encode(c, X)
    assert np.array_equal(Y, O.encode(n, k, 0, False, X))
    sent, out = repair_gpu(c, Y, 0, [1, 2, 3, 4], nbytes)
    assert np.array_equal(out, Y[0:2])
    got, _ = decode_gpu(c, Y, [1, 2, 3], nbytes)
    assert np.array_equal(got, X)


def test_gpu_calls_reject_bad_arguments_without_launching():
    c = code(8, 4, 1, 1)
    b = Blocks(12, 64)
    with pytest.raises(P.PMRCError) as e:
        c.repair_newcomer(0, [2, 3, 4, 5, 6, 7], b.ptrs()[:6], b.ptrs()[6:9], 64)
    assert e.value.rc == P.PMRC_ESINGULAR
    with pytest.raises(P.PMRCError) as e:
        c.repair_helper(0, 0, b.ptrs()[:3], b.ptr(3), 64)
    assert e.value.rc == P.PMRC_EINVAL
    with pytest.raises(P.PMRCError) as e:
        c.encode([0] * 12, b.ptrs(), 64)
    assert e.value.rc == P.PMRC_EINVAL


BITSLICED_CODES = [(16, 8, 1, 1), (16, 8, 0, 0), (8, 4, 1, 1), (6, 3, 1, 1), (6, 3, 0, 0),
                   (24, 12, 1, 1), (32, 16, 1, 1)]


@pytest.mark.parametrize("nbytes", [32, 33, 8192, 8192 + 32 + 7, 3 * 8192 + 16, 100000])
@pytest.mark.parametrize("n,k,cons,form", BITSLICED_CODES)
def test_bitsliced_and_generic_encode_agree_with_oracle(n, k, cons, form, nbytes):
    X = inputs.blocks(k * (k - 1), nbytes, seed=nbytes + 7 * k)
    want = oracle_outputs(n, k, cons, form, X)
    for which in (P.PMRC_KERNEL_BITSLICED, P.PMRC_KERNEL_GENERIC):
        c = code(n, k, cons, form)
        c.set_encode_kernel(which)
        assert np.array_equal(run_encode(c, X), want), which


# ------------------------------------------------------------------ fused repair
def fused_repair_gpu(c, Y, f, H, nbytes, shift=0):
    a = c.alpha
    store = Blocks(c.n * a, nbytes, shift, Y)
    out = Blocks(a, nbytes, shift)
    c.repair(f, H, [store.ptr(a * h + j) for h in H for j in range(a)], out.ptrs(), nbytes)
    assert out.guards_intact()
    return out.get()


@pytest.mark.parametrize("n,k,cons,form", [(6, 3, 0, 0), (6, 3, 1, 1), (8, 4, 1, 1),
                                           (16, 8, 1, 1), (16, 8, 0, 0), (24, 12, 1, 1),
                                           (32, 16, 1, 1)])
def test_fused_repair_every_node(n, k, cons, form):
    a = k - 1
    nbytes = 2 * 4096 + 19
    X = inputs.blocks(k * a, nbytes, seed=300 + k)
    Y = O.encode(n, k, cons, bool(form), X)
    c = code(n, k, cons, form)
    for f in range(n):
        H = c.default_helpers(f)
        got = fused_repair_gpu(c, Y, f, H, nbytes, shift=(f % 3) * 4)
        assert np.array_equal(got, Y[a * f:a * f + a]), f


def test_fused_repair_k3_every_helper_set_and_sizes():
    n, k, a, d = 6, 3, 2, 4
    c = code(n, k, 1, 1)
    for nbytes in (1, 17, 4096, 3 * 4096 + 1):
        X = inputs.blocks(k * a, nbytes, seed=nbytes)
        Y = O.encode(n, k, 1, True, X)
        for f in range(n):
            for H in itertools.combinations([i for i in range(n) if i != f], d):
                H = list(H)
                try:
                    O.newcomer_matrix(n, k, 1, f, H)
                except O.OracleError:
                    continue
                assert np.array_equal(fused_repair_gpu(c, Y, f, H, nbytes), Y[a * f:a * f + a])


def test_fused_repair_full_size_sampled():
    n, k, a = 16, 8, 7
    nbytes = 1 << 20
    c = code(n, k, 1, 1)
    X = inputs.device_blocks(k * a, nbytes, seed=99)
    Y = torch.empty((n * a, nbytes), dtype=torch.uint8, device="cuda")
    Y[:k * a].copy_(X)
    c.encode([X[i] for i in range(k * a)], [Y[k * a + i] for i in range((n - k) * a)], nbytes)
    for f in (3, 12):
        H = c.default_helpers(f)
        out = torch.empty((a, nbytes), dtype=torch.uint8, device="cuda")
        c.repair(f, H, [Y[a * h + j] for h in H for j in range(a)], [out[j] for j in range(a)],
                 nbytes)
        torch.cuda.synchronize()
        assert torch.equal(out, Y[a * f:a * f + a])
        for cs in columns(nbytes):
            Yc = Y[:, cs].cpu().numpy()
            sent = np.stack([O.repair_helper(n, k, 1, f, Yc[a * h:a * h + a]) for h in H])
            assert np.array_equal(out[:, cs].cpu().numpy(), O.repair_newcomer(n, k, 1, f, H, sent))


@pytest.mark.parametrize("node", [3, 7])
def test_degraded_read_returns_the_nodes_data(node):
    """A lost systematic node's data, byte ranges included, rebuilt from its
    helpers (node 3 < alpha: one block per helper; node 7: seven)."""
    n, k, a, d = 16, 8, 7, 14
    nbytes = 3 * 4096 + 29
    X = inputs.blocks(k * a, nbytes, seed=98 + node)
    Y = O.encode(n, k, 1, True, X)
    c = code(n, k, 1, 1)
    H = c.default_helpers(node)
    hin = Blocks(d * a, nbytes, 0, np.concatenate([Y[a * h:a * h + a] for h in H]))
    for off, length in ((0, nbytes), (1000, 5003), (nbytes - 17, 17)):
        out = Blocks(a, length)
        c.read_degraded(node, H, hin.ptrs(), out.ptrs(), off, length)
        assert out.guards_intact()
        assert np.array_equal(out.get(), X[a * node:a * node + a, off:off + length]), (off, length)


def test_degraded_read_reed_solomon():
    n, k, nbytes = 16, 8, 4096 + 3
    X = inputs.blocks(k, nbytes, seed=99)
    Y = O.rs_encode(n, k, True, X)
    c = P.Code(n, k, P.PMRC_RS, P.PMRC_SYSTEMATIC)
    node = 5
    H = c.default_helpers(node)
    hin = Blocks(k, nbytes, 0, Y[H])
    out = Blocks(1, nbytes - 100)
    c.read_degraded(node, H, hin.ptrs(), out.ptrs(), 100, nbytes - 100)
    assert np.array_equal(out.get()[0], X[node, 100:])
