"""Encodes of codes without a built-in bitsliced kernel, through a bitsliced
kernel compiled at run time for their encode matrix (pmrc_set_encode_kernel
PMRC_KERNEL_BITSLICED at any size, PMRC_KERNEL_AUTO from 256 KiB blocks for
small matrices):
bit-exact against the CPU oracle, with ragged tails (split-table kernel)
and misaligned blocks (split-table kernel throughout)."""
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


def encode(c, X, nbytes, shift=0):
    xin = Blocks(X.shape[0], nbytes, shift, X)
    y = Blocks(c.n_outputs, nbytes, shift)
    c.encode(xin.ptrs(), y.ptrs(), nbytes)
    assert y.guards_intact() and xin.guards_intact()
    return y.get()


# PM-MSR codes of n = 2k and other n, both constructions and forms; the
# vanilla k = 12 generator takes 33 blocks and 396 block pointers
MSR = [(14, 7, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC), (20, 10, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC),
       (12, 6, P.PMRC_VANILLA, P.PMRC_SYSTEMATIC), (24, 12, P.PMRC_VANILLA, P.PMRC_NONSYSTEMATIC),
       (11, 5, P.PMRC_SPARSE, P.PMRC_NONSYSTEMATIC)]


@pytest.mark.parametrize("n,k,cons,form", MSR)
def test_runtime_encode_forced(n, k, cons, form):
    c = P.Code(n, k, cons, form)
    c.set_encode_kernel(P.PMRC_KERNEL_BITSLICED)
    K = c.data_blocks
    for nbytes, shift in ((64 * 1024 + 32 + 7, 0), (4096, 0), (1000, 4)):
        X = inputs.blocks(K, nbytes, seed=nbytes + n)
        Y = O.encode(n, k, cons, bool(form), X)
        assert np.array_equal(encode(c, X, nbytes, shift), Y[K:] if form else Y), (nbytes, shift)


def test_runtime_encode_auto_from_256k():
    """AUTO compiles the schedule of a small encode matrix (k = 10: 1620
    non-zero coefficients) for blocks of 256 KiB and more."""
    n, k = 20, 10
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    K, nbytes = c.data_blocks, 256 * 1024 + 48
    X = inputs.blocks(K, nbytes, seed=90)
    assert np.array_equal(encode(c, X, nbytes), O.encode(n, k, O.SPARSE, True, X)[K:])


def test_runtime_encode_gf16_and_mbr():
    c = P.Code(16, 8, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC, field_bits=16)
    c.set_encode_kernel(P.PMRC_KERNEL_BITSLICED)
    K, nbytes = c.data_blocks, 2 * (32 * 1024 + 48)   # planes: bitsliced body + 16-byte tail
    X = inputs.blocks(K, nbytes, seed=91)
    assert np.array_equal(encode(c, X, nbytes), O.gf16_encode(16, 8, O.SPARSE, True, X)[K:])
    for n, k, d, form in ((8, 4, 6, P.PMRC_NONSYSTEMATIC), (12, 6, 10, P.PMRC_SYSTEMATIC)):
        c = P.Code(n, k, P.PMRC_MBR, form, d=d)
        c.set_encode_kernel(P.PMRC_KERNEL_BITSLICED)
        a, B = O.mbr_params(n, k, d)
        nbytes = 16 * 1024 + 40
        X = inputs.blocks(B, nbytes, seed=92 + n)
        Y = O.mbr_encode(n, k, d, X)
        assert np.array_equal(encode(c, X, nbytes), Y[k * a:] if form else Y), (n, k, d)
    # PM-MBR n=16 non-systematic: its rows need more than 64 blocks of
    # identical support, or blocks of more than 64 inputs
    c = P.Code(16, 8, P.PMRC_MBR, P.PMRC_NONSYSTEMATIC, d=14)
    with pytest.raises(P.PMRCError) as e:
        c.set_encode_kernel(P.PMRC_KERNEL_BITSLICED)
    assert e.value.rc == P.PMRC_EUNSUPPORTED


def test_runtime_encode_null_output_takes_the_generic_kernel():
    """A NULL output block is skipped by the split-table kernel; the
    bitsliced kernels need every output, so the call takes the former."""
    n, k = 20, 10
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    c.set_encode_kernel(P.PMRC_KERNEL_BITSLICED)
    K, nbytes = c.data_blocks, 8192
    X = inputs.blocks(K, nbytes, seed=93)
    xin = Blocks(K, nbytes, 0, X)
    y = Blocks(c.n_outputs, nbytes)
    ptrs = y.ptrs()
    ptrs[5] = 0
    c.encode(xin.ptrs(), ptrs, nbytes)
    got = y.get()
    Y = O.encode(n, k, O.SPARSE, True, X)[K:]
    assert (got[5] == 0xA5).all()
    for r in range(len(ptrs)):
        if r != 5:
            assert np.array_equal(got[r], Y[r]), r
