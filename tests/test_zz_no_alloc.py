"""pmrc_repair_noalloc -- the repair entry point for callers that cannot
allocate GPU memory -- returns the same bytes as pmrc_repair.

Both are called through the C ABI on the same stored codeword, twice in a
row (a failed node whose helpers must project alpha blocks, then one whose
helpers send a stored block as is), and again for the largest code the
fixed table area is meant for (k=16, alpha=15).  The bar is
the one every test here uses: byte-for-byte equality.  This file is
collected last so that a run stopping at its first failure has already run
everything else; it passes alone in a fresh process as well.
"""
import ctypes

import pytest

import paper_1412_3022_gb300 as P
from paper_1412_3022_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def codeword(c, nbytes, seed):
    K = c.k * c.alpha
    X = inputs.device_blocks(K, nbytes, seed=seed)
    Y = torch.empty((c.n * c.alpha, nbytes), dtype=torch.uint8, device="cuda")
    Y[:K].copy_(X)
    c.encode([X[i] for i in range(K)], [Y[K + i] for i in range(Y.shape[0] - K)], nbytes)
    return Y


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


def compare(c, Y, f, nbytes):
    a = c.alpha
    H = c.default_helpers(f)
    blocks = [Y[a * h + j] for h in H for j in range(a)]
    ref = torch.empty((a, nbytes), dtype=torch.uint8, device="cuda")
    got = torch.full((a, nbytes), 0xA5, dtype=torch.uint8, device="cuda")
    abi_call("pmrc_repair", c, f, H, blocks, [ref[j] for j in range(a)], nbytes)
    abi_call("pmrc_repair_noalloc", c, f, H, blocks, [got[j] for j in range(a)], nbytes)
    torch.cuda.synchronize()
    assert torch.equal(got, ref), f
    assert torch.equal(got, Y[a * f:a * f + a]), f


def test_repair_noalloc_matches_repair_on_two_calls_in_a_row():
    c = P.Code(16, 8, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    nbytes = (1 << 20) + 48
    Y = codeword(c, nbytes, seed=11)
    compare(c, Y, 12, nbytes)   # helpers project all alpha blocks
    compare(c, Y, 3, nbytes)    # helpers send one stored block


def test_repair_noalloc_matches_repair_for_k16():
    c = P.Code(32, 16, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    nbytes = (3 << 20) + 5
    Y = codeword(c, nbytes, seed=12)
    compare(c, Y, 20, nbytes)
    compare(c, Y, 31, nbytes)
