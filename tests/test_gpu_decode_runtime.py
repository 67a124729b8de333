"""Reconstruction through bitsliced kernels compiled at run time
(pmrc_set_decode_kernel): bit-exact against the CPU oracle and the data, on
every subset at k=3, random subsets at k=8 (with a ragged tail and lazy
aliasing), Reed-Solomon; refusals when the kernel cannot be built."""
import itertools

import numpy as np
import pytest

import oracle as O
import paper_1412_3022_gb300 as P
from oracle_columns import oracle_columns
from paper_1412_3022_gb300 import inputs
from test_gpu_parity import Blocks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def decode(c, S, Y, nbytes, lazy=False, shift=0):
    a, K = c.alpha, c.data_blocks
    rows = [a * i + j for i in S for j in range(a)]
    yin = Blocks(len(rows), nbytes, shift, Y[rows])
    xout = Blocks(K, nbytes, shift)
    ptrs = xout.ptrs()
    if lazy and c.form == P.PMRC_SYSTEMATIC:
        for pos, i in enumerate(S):
            if i < c.k:
                for j in range(a):
                    ptrs[a * i + j] = yin.ptr(a * pos + j)
    c.decode(S, yin.ptrs(), ptrs, nbytes)
    assert xout.guards_intact()
    got = xout.get()
    return got, [ptrs[r] == xout.ptr(r) for r in range(K)]


@pytest.mark.parametrize("form", [P.PMRC_SYSTEMATIC, P.PMRC_NONSYSTEMATIC])
def test_runtime_decode_every_subset_k3(form):
    n, k, nbytes = 6, 3, 4096 + 7
    c = P.Code(n, k, P.PMRC_SPARSE, form)
    c.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    X = inputs.blocks(6, nbytes, seed=80)
    Y = O.encode(n, k, O.SPARSE, bool(form), X)
    for S in itertools.combinations(range(n), k):
        got, _ = decode(c, list(S), Y, nbytes)
        assert np.array_equal(got, X), S


def test_runtime_decode_k8_random_lazy_and_tail():
    n, k = 16, 8
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    c.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    rng = np.random.default_rng(81)
    for t, nbytes in enumerate((64 * 1024 + 13, 3 * 4096 + 32)):
        X = inputs.blocks(56, nbytes, seed=82 + t)
        Y = O.encode(n, k, O.SPARSE, True, X)
        for _ in range(2):
            S = rng.permutation(rng.choice(n, k, replace=False)).tolist()
            got, computed = decode(c, S, Y, nbytes, lazy=True)
            for r in range(56):
                if computed[r]:
                    assert np.array_equal(got[r], X[r]), (S, r)
                else:
                    assert (got[r] == 0xA5).all(), (S, r)


def test_runtime_decode_matches_generic_and_rs():
    n, k, nbytes = 16, 8, 32 * 1024
    gen = P.Code(n, k, P.PMRC_VANILLA, P.PMRC_NONSYSTEMATIC)
    X = inputs.blocks(56, nbytes, seed=83)
    Y = O.encode(n, k, O.VANILLA, False, X)
    S = [15, 3, 9, 0, 12, 6, 1, 10]
    outs = []
    for which in (P.PMRC_KERNEL_BITSLICED, P.PMRC_KERNEL_GENERIC):
        gen.set_decode_kernel(which)
        outs.append(decode(gen, S, Y, nbytes)[0])
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], X)
    rs = P.Code(16, 8, P.PMRC_RS, P.PMRC_SYSTEMATIC)
    rs.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    X = inputs.blocks(8, nbytes, seed=84)
    Y = O.rs_encode(16, 8, True, X)
    got, _ = decode(rs, [9, 2, 14, 11, 4, 15, 0, 7], Y, nbytes)
    assert np.array_equal(got, X)


def test_runtime_decode_refusals():
    c = P.Code(16, 8, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    c.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    X = inputs.blocks(56, 4096, seed=85)
    Y = O.encode(16, 8, O.SPARSE, True, X)
    with pytest.raises(P.PMRCError) as e:      # misaligned blocks cannot take this path
        decode(c, [8, 9, 10, 11, 12, 13, 14, 15], Y, 4096, shift=3)
    assert e.value.rc == P.PMRC_EUNSUPPORTED
    m = P.Code(16, 8, P.PMRC_MBR, P.PMRC_SYSTEMATIC, d=14)   # 112 inputs per block
    m.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    a, B = O.mbr_params(16, 8, 14)
    Xm = inputs.blocks(B, 4096, seed=86)
    Ym = O.mbr_encode(16, 8, 14, Xm)
    with pytest.raises(P.PMRCError) as e:
        decode(m, [8, 9, 10, 11, 12, 13, 14, 15], Ym, 4096)
    assert e.value.rc == P.PMRC_EUNSUPPORTED
    m.set_decode_kernel(P.PMRC_KERNEL_AUTO)    # AUTO keeps the split-table kernel
    got, _ = decode(m, [8, 9, 10, 11, 12, 13, 14, 15], Ym, 4096)
    assert np.array_equal(got, Xm)


def test_runtime_newcomer_every_node_k8_and_mbr():
    """The newcomer's D compiled at run time per (failed node, helpers)."""
    n, k, nbytes = 16, 8, 64 * 1024 + 20
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    c.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    a, d = 7, 14
    X = inputs.blocks(56, nbytes, seed=87)
    Y = O.encode(n, k, O.SPARSE, True, X)
    for f in range(n):
        H = c.default_helpers(f)
        sent = np.stack([O.repair_helper(n, k, O.SPARSE, f, Y[a * h:a * h + a]) for h in H])
        recv = Blocks(d, nbytes, 0, sent)
        out = Blocks(a, nbytes)
        c.repair_newcomer(f, H, recv.ptrs(), out.ptrs(), nbytes)
        assert out.guards_intact()
        assert np.array_equal(out.get(), Y[a * f:a * f + a]), f
    m = P.Code(16, 8, P.PMRC_MBR, P.PMRC_SYSTEMATIC, d=14)
    m.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    am, B = O.mbr_params(16, 8, 14)
    Xm = inputs.blocks(B, 4096 + 32, seed=88)
    Ym = O.mbr_encode(16, 8, 14, Xm)
    for f in (0, 13):
        H = m.default_helpers(f)
        sent = np.stack([O.mbr_repair_helper(16, 8, 14, f, Ym[am * h:am * h + am]) for h in H])
        recv = Blocks(14, 4096 + 32, 0, sent)
        out = Blocks(am, 4096 + 32)
        m.repair_newcomer(f, H, recv.ptrs(), out.ptrs(), 4096 + 32)
        assert np.array_equal(out.get(), Ym[am * f:am * f + am]), f


def test_runtime_kernels_cached_on_disk(tmp_path, monkeypatch):
    """With PMRC_KERNEL_CACHE set, a compiled schedule is written once and a
    fresh handle meeting the same node set reads it back."""
    monkeypatch.setenv("PMRC_KERNEL_CACHE", str(tmp_path))
    n, k, nbytes = 16, 8, 8192 + 32
    X = inputs.blocks(56, nbytes, seed=97)
    Y = O.encode(n, k, O.SPARSE, True, X)
    S = [15, 0, 9, 2, 11, 4, 13, 6]
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    c.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    got, _ = decode(c, S, Y, nbytes)
    assert np.array_equal(got, X)
    files = list(tmp_path.glob("pmrc-*.cubin"))
    assert len(files) == 1
    stamp = files[0].stat().st_mtime_ns
    c2 = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    c2.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    got, _ = decode(c2, S, Y, nbytes)
    assert np.array_equal(got, X)
    assert list(tmp_path.glob("pmrc-*.cubin")) == files
    assert files[0].stat().st_mtime_ns == stamp     # read back, not rewritten
    assert not list(tmp_path.glob("*.tmp"))


def test_auto_compiles_in_the_background():
    """AUTO: the first reconstruction of a node set starts its compilation
    and runs the split-table kernel; once compiled, the next call loads and
    runs the bitsliced kernel.  Both results are the data."""
    n, k, nbytes = 16, 8, 256 * 1024 + 32
    X = inputs.blocks(56, nbytes, seed=100)
    Y = O.encode(n, k, O.SPARSE, True, X)
    S = [1, 3, 5, 7, 8, 10, 12, 14]
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    got, _ = decode(c, S, Y, nbytes)
    assert np.array_equal(got, X)
    ready, pending = c.runtime_kernels()
    assert ready + pending == 1
    c.wait_kernels()
    assert c.runtime_kernels() == (1, 0)
    got, _ = decode(c, S, Y, nbytes)
    assert np.array_equal(got, X)
    assert c.runtime_kernels() == (1, 0)


def test_forced_bitsliced_compiles_before_it_launches():
    n, k, nbytes = 16, 8, 4096 + 32
    X = inputs.blocks(56, nbytes, seed=101)
    Y = O.encode(n, k, O.SPARSE, True, X)
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    c.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    got, _ = decode(c, [0, 2, 4, 6, 9, 11, 13, 15], Y, nbytes)
    assert np.array_equal(got, X)
    assert c.runtime_kernels() == (1, 0)


def lazy_decode_every_column(c, n, k, S, nbytes, X, Y):
    """Reconstruction of the missing data rows only (present data rows
    alias their node blocks), checked byte for byte against the data."""
    got, computed = decode(c, S, Y, nbytes, lazy=True)
    a = k - 1
    missing = [r for r in range(k * a) if r // a not in S]
    assert [r for r in range(k * a) if computed[r]] == missing
    for r in missing:
        assert np.array_equal(got[r], X[r]), (S, r)


@pytest.mark.parametrize("S,kernels", [([0, 1, 2, 3, 4, 5, 6, 9], None),   # one data node missing
                                       ([0, 1, 4, 5, 7, 8, 11, 12], 2),     # three (the bench's set)
                                       ([15, 2, 9, 4, 13, 0, 11, 6], 2),    # four, out of order
                                       ([1, 3, 5, 8, 9, 10, 12, 14], 2)])   # five
def test_factored_reconstruction_k8_1mib(S, kernels):
    """Lazy reconstructions of 1 MiB blocks: where the reconstruction rows
    are dense (three or more data nodes missing: B^-1 mixes every parity
    block) they take the two-launch factored kernels -- z = the received
    parity blocks plus their present-data terms, stored in plane layout in
    stream-ordered scratch, then the missing rows B^-1 z -- two run-time
    kernels per node set; with one data node missing the rows are about as
    sparse as z and either schedule may be chosen.  The 48-byte ragged tail
    goes to the split-table kernel; every missing row equals the data."""
    n, k = 16, 8
    nbytes = (1 << 20) + 48
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    c.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    X = inputs.blocks(56, nbytes, seed=120)
    Y = oracle_columns(lambda x: O.encode(n, k, O.SPARSE, True, x), [X])
    lazy_decode_every_column(c, n, k, S, nbytes, X, Y)
    first = c.runtime_kernels()
    assert first in ((1, 0), (2, 0)) if kernels is None else first == (kernels, 0)
    lazy_decode_every_column(c, n, k, S, nbytes, X, Y)   # the same kernels again
    assert c.runtime_kernels() == first


def test_factored_reconstruction_k16_where_one_launch_cannot_fit():
    """n=32, k=16: with four data nodes missing, a row of the one-launch
    schedule reads the 240 received blocks, beyond a bitsliced block's 64
    inputs, so the bitsliced reconstruction exists only in factored form (z
    rows grouped by support, B^-1 of 60 rows); with two and three missing
    either form may be chosen.  Lazy reconstructions with a ragged 16-byte
    tail equal the data."""
    n, k = 32, 16
    a = k - 1
    nbytes = (64 << 10) + 16
    X = inputs.blocks(k * a, nbytes, seed=121)
    Y = oracle_columns(lambda x: O.encode(n, k, O.SPARSE, True, x), [X])
    sets = [[0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 16, 31],
            [31, 0, 2, 3, 17, 5, 6, 7, 8, 9, 10, 11, 12, 20, 14, 15],
            [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 18, 19, 22, 25]]
    for S in sets:
        c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
        c.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
        lazy_decode_every_column(c, n, k, S, nbytes, X, Y)
        if sum(1 for i in S if i >= k) == 4:   # 60 dense rows over 240 blocks: factored only
            assert c.runtime_kernels() == (2, 0)
        else:
            assert c.runtime_kernels() in ((1, 0), (2, 0))
