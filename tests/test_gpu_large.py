"""GPU parity of codes too large for one region launch: more than 1024 block
pointers per operation (k >= 24 at n = 2k, the paper's evaluation reaches
k = 32), or reconstruction rows over more inputs than one block's split
tables hold in shared memory.  The library runs such operations as several
launches (row sets; input chunks whose later launches XOR into the outputs
of the first); every result is compared byte for byte with the CPU oracle."""
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

NBYTES = 3 * 2048 + 13   # several tiles and a ragged tail


def _encode(c, X, nbytes, shift=0):
    K = X.shape[0]
    xin = Blocks(K, nbytes, shift, X)
    y = Blocks(c.n_outputs, nbytes, shift)
    c.encode(xin.ptrs(), y.ptrs(), nbytes)
    assert y.guards_intact()
    return y.get()


@pytest.mark.parametrize("cons,form", [(P.PMRC_SPARSE, P.PMRC_SYSTEMATIC),
                                       (P.PMRC_VANILLA, P.PMRC_NONSYSTEMATIC)])
def test_k24_encode(cons, form):
    n, k = 48, 24
    a, K = k - 1, k * (k - 1)
    c = P.Code(n, k, cons, form)
    for nbytes, shift in ((NBYTES, 0), (999, 3)):
        X = inputs.blocks(K, nbytes, seed=nbytes + cons)
        Y = O.encode(n, k, cons, bool(form), X)
        assert np.array_equal(_encode(c, X, nbytes, shift), Y[K:] if form else Y), (nbytes, shift)


def test_k24_repair_and_decode():
    n, k = 48, 24
    a, K, d = k - 1, k * (k - 1), 2 * k - 2
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    X = inputs.blocks(K, NBYTES, seed=31)
    Y = O.encode(n, k, O.SPARSE, True, X)
    # repair: d = 46 helpers x 23 blocks read (1058 input pointers)
    for f in (3, 30):
        H = c.default_helpers(f)
        hin = Blocks(d * a, NBYTES, 0, np.concatenate([Y[a * h:a * h + a] for h in H]))
        recv = Blocks(d, NBYTES)
        out = Blocks(a, NBYTES)
        c.repair_helpers(f, H, hin.ptrs(), recv.ptrs(), NBYTES)
        c.repair_newcomer(f, H, recv.ptrs(), out.ptrs(), NBYTES)
        assert recv.guards_intact() and out.guards_intact()
        assert np.array_equal(out.get(), Y[a * f:a * f + a]), f
    # reconstruction from 12 data and 12 parity nodes: 276 missing rows,
    # each over ~550 inputs (more than one block's tables: input chunks)
    S = list(range(1, n, 2))
    rows = [a * i + j for i in S for j in range(a)]
    yin = Blocks(K, NBYTES, 0, Y[rows])
    xout = Blocks(K, NBYTES)
    c.decode(S, yin.ptrs(), xout.ptrs(), NBYTES)
    assert xout.guards_intact()
    assert np.array_equal(xout.get(), O.decode(n, k, O.SPARSE, True, S, Y[rows]))


def test_k32_encode_and_decode():
    n, k = 64, 32
    a, K = k - 1, k * (k - 1)
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    nbytes = 2048 + 5
    X = inputs.blocks(K, nbytes, seed=32)
    Y = O.encode(n, k, O.SPARSE, True, X)
    assert np.array_equal(_encode(c, X, nbytes), Y[K:])
    rng = np.random.default_rng(33)
    S = rng.permutation(rng.choice(n, k, replace=False)).tolist()
    rows = [a * i + j for i in S for j in range(a)]
    yin = Blocks(K, nbytes, 0, Y[rows])
    xout = Blocks(K, nbytes)
    c.decode(S, yin.ptrs(), xout.ptrs(), nbytes)
    assert np.array_equal(xout.get(), X)


def test_large_plan_refused_by_the_batch_kernel():
    """The batched kernel takes operations of one launch only."""
    c = P.Code(48, 24, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    K = c.data_blocks
    xin = Blocks(K, 4096)
    y = Blocks(c.n_outputs, 4096)
    b = P.Batch()
    with pytest.raises(P.PMRCError) as e:
        b.add_encode(c, xin.ptrs(), y.ptrs(), 4096)
    assert e.value.rc == P.PMRC_EUNSUPPORTED
    b.close()


def test_mbr_n32_nonsystematic_encode():
    """PM-MBR n=32 k=16 d=30: 360 data blocks into 960 coded ones."""
    n, k, d = 32, 16, 30
    c = P.Code(n, k, P.PMRC_MBR, P.PMRC_NONSYSTEMATIC, d=d)
    _, B = O.mbr_params(n, k, d)
    X = inputs.blocks(B, NBYTES, seed=34)
    assert np.array_equal(_encode(c, X, NBYTES), O.mbr_encode(n, k, d, X))


def test_gf16_k20_encode_and_decode():
    """GF(2^16), n=40 k=20: 380 symbols a block row, 760 byte planes each
    side of the encode."""
    n, k = 40, 20
    a, K = k - 1, k * (k - 1)
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC, field_bits=16)
    nbytes = 2 * 2048 + 6
    X = inputs.blocks(K, nbytes, seed=35)
    Y = O.gf16_encode(n, k, O.SPARSE, True, X)
    assert np.array_equal(_encode(c, X, nbytes), Y[K:])
    S = list(range(n - k, n))           # the parity nodes only
    rows = [a * i + j for i in S for j in range(a)]
    yin = Blocks(K, nbytes, 0, Y[rows])
    xout = Blocks(K, nbytes)
    c.decode(S, yin.ptrs(), xout.ptrs(), nbytes)
    assert np.array_equal(xout.get(), X)
