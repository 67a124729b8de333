"""pmrc_repair_noalloc -- the repair entry point for callers that cannot
allocate GPU memory (a library inside a process whose device memory belongs
to another allocator, or a repair path that must not block, synchronize or
fail part-way on an allocation) -- returns the same bytes as pmrc_repair,
as the stored node and as the CPU oracle's repair (the helpers' projections
onto phi_f, then the newcomer matrix, Sec. 2 and 3.3).

Both entry points are called through the C ABI on a codeword the oracle
encoded, twice in a row for each code: the n=16 k=8 sparse code (a failed
node whose helpers project alpha blocks, then one whose helpers send a
stored block as is), the largest PM-MSR code the fixed table area is meant
for (k=16, alpha=15), the n=16 k=8 d=14 PM-MBR code and RS(16, 8).  The bar
is the one every test here uses: byte-for-byte equality.  This file is
collected last so that a run stopping at its first failure has already run
everything else; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import paper_1412_3022_gb300 as P
from oracle_columns import oracle_columns
from paper_1412_3022_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def abi_call(fn, c, f, H, blocks, out, nbytes):
    """Calls a repair entry point of libpmrc directly through ctypes."""
    L = P.lib()
    hs = (ctypes.c_int * len(H))(*H)
    bp = (ctypes.c_void_p * len(blocks))(*[b.data_ptr() for b in blocks])
    op = (ctypes.c_void_p * len(out))(*[o.data_ptr() for o in out])
    stream = torch.cuda.current_stream().cuda_stream
    rc = getattr(L, fn)(ctypes.c_void_p(c.handle), f, hs, bp, op, ctypes.c_size_t(nbytes),
                        ctypes.c_void_p(stream))
    assert rc == P.PMRC_OK, (fn, rc, P.pmrc_last_error())


def compare(c, Yh, f, nbytes, oracle_repair):
    """Runs both entry points for node f from its default helpers and
    checks them against each other, the stored node and oracle_repair(H,
    helper blocks) on every column."""
    a = c.alpha
    Y = torch.from_numpy(Yh).cuda()
    H = c.default_helpers(f)
    blocks = [Y[a * h + j] for h in H for j in range(a)]
    ref = torch.full((a, nbytes), 0x5A, dtype=torch.uint8, device="cuda")
    got = torch.full((a, nbytes), 0xA5, dtype=torch.uint8, device="cuda")
    abi_call("pmrc_repair", c, f, H, blocks, [ref[j] for j in range(a)], nbytes)
    abi_call("pmrc_repair_noalloc", c, f, H, blocks, [got[j] for j in range(a)], nbytes)
    torch.cuda.synchronize()
    assert torch.equal(got, ref), f
    assert np.array_equal(got.cpu().numpy(), Yh[a * f:a * f + a]), f
    helper_blocks = np.concatenate([Yh[a * h:a * h + a] for h in H])
    want = oracle_columns(lambda x: oracle_repair(H, x), [helper_blocks])
    assert np.array_equal(got.cpu().numpy(), want), f


def msr_repair(n, k, f):
    a = k - 1

    def rep(H, x):
        sent = np.stack([O.repair_helper(n, k, O.SPARSE, f, x[a * i:a * i + a])
                         for i in range(len(H))])
        return O.repair_newcomer(n, k, O.SPARSE, f, H, sent)
    return rep


def test_repair_noalloc_matches_repair_and_oracle_on_two_calls_in_a_row():
    n, k = 16, 8
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    nbytes = (1 << 20) + 48
    X = inputs.blocks(k * (k - 1), nbytes, seed=11)
    Yh = oracle_columns(lambda x: O.encode(n, k, O.SPARSE, True, x), [X])
    compare(c, Yh, 12, nbytes, msr_repair(n, k, 12))   # helpers project all alpha blocks
    compare(c, Yh, 3, nbytes, msr_repair(n, k, 3))     # helpers send one stored block


def test_repair_noalloc_matches_repair_for_k16():
    n, k = 32, 16
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    nbytes = (256 << 10) + 5
    X = inputs.blocks(k * (k - 1), nbytes, seed=12)
    Yh = oracle_columns(lambda x: O.encode(n, k, O.SPARSE, True, x), [X])
    compare(c, Yh, 20, nbytes, msr_repair(n, k, 20))
    compare(c, Yh, 31, nbytes, msr_repair(n, k, 31))


def test_repair_noalloc_matches_repair_for_mbr_and_reed_solomon():
    n, k, d = 16, 8, 14
    nbytes = (192 << 10) + 7
    mbr = P.Code(n, k, P.PMRC_MBR, P.PMRC_SYSTEMATIC, d=d)
    a, K = O.mbr_params(n, k, d)
    X = inputs.blocks(K, nbytes, seed=13)
    Yh = oracle_columns(lambda x: O.mbr_encode(n, k, d, x), [X])
    for f in (2, 13):
        def rep(H, x, f=f):
            sent = np.stack([O.mbr_repair_helper(n, k, d, f, x[a * i:a * i + a])
                             for i in range(len(H))])
            return O.mbr_repair_newcomer(n, k, d, f, H, sent)
        compare(mbr, Yh, f, nbytes, rep)
    rs = P.Code(n, k, P.PMRC_RS, P.PMRC_SYSTEMATIC)
    X = inputs.blocks(k, nbytes, seed=14)
    Yr = oracle_columns(lambda x: O.rs_encode(n, k, True, x), [X])
    for f in (3, 12):
        compare(rs, Yr, f, nbytes, lambda H, x, f=f: O.rs_repair(n, k, True, f, H, x)[None, :])
