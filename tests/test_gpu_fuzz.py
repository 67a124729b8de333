"""Seeded random cases across the PM-MSR path: random (n, k), construction,
form, block size (ragged and aligned), pointer misalignment and kernel
choice; encode, two-step and fused repair of a random node, degraded read
and reconstruction from a random node set, each compared byte for byte
with the CPU oracle.  Every case derives its inputs from its index, so a
failure names a reproducible case."""
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

KERNELS = [P.PMRC_KERNEL_AUTO, P.PMRC_KERNEL_GENERIC, P.PMRC_KERNEL_BITSLICED]


def _case(i):
    rng = np.random.default_rng(1000 + i)
    while True:
        k = int(rng.integers(2, 13))
        n = int(rng.integers(2 * k - 1, min(2 * k + 5, 254) + 1))
        cons = int(rng.integers(0, 2))
        form = int(rng.integers(0, 2))
        try:
            c = P.Code(n, k, cons, form)
        except P.PMRCError as e:      # vanilla codes with repeated lambda
            assert e.rc == P.PMRC_EUNSUPPORTED
            continue
        break
    nbytes = int(rng.choice([int(rng.integers(1, 20000)), 32 * int(rng.integers(1, 600)),
                             16 * int(rng.integers(1, 1200))]))
    shift = int(rng.choice([0, 0, 16, int(rng.integers(1, 16))]))
    # run-time bitsliced schedules only for small codes (their compilation)
    choices = KERNELS if k <= 6 else KERNELS[:2]
    enc_k, dec_k = (int(rng.choice(choices)) for _ in range(2))
    return rng, c, n, k, cons, form, nbytes, shift, enc_k, dec_k


@pytest.mark.parametrize("case", range(100))
def test_fuzz_case(case):
    rng, c, n, k, cons, form, nbytes, shift, enc_k, dec_k = _case(case)
    a, K = k - 1, k * (k - 1)
    try:
        c.set_encode_kernel(enc_k)
    except P.PMRCError as e:          # no schedule fits this code
        assert e.rc == P.PMRC_EUNSUPPORTED
    c.set_decode_kernel(dec_k)
    X = inputs.blocks(K, nbytes, seed=case)
    Yfull = O.encode(n, k, cons, bool(form), X)
    # encode
    xin = Blocks(K, nbytes, shift, X)
    y = Blocks(c.n_outputs, nbytes, shift)
    c.encode(xin.ptrs(), y.ptrs(), nbytes)
    assert y.guards_intact()
    assert np.array_equal(y.get(), Yfull[K:] if form else Yfull), "encode"
    # repair of a random node, two-step and fused
    f = int(rng.integers(0, n))
    try:
        H = c.default_helpers(f)
    except P.PMRCError as e:
        assert e.rc == P.PMRC_ESINGULAR
        H = None
    if H is not None:
        d = len(H)
        hin = Blocks(d * a, nbytes, shift, np.concatenate([Yfull[a * h:a * h + a] for h in H]))
        recv = Blocks(d, nbytes, shift)
        node = Blocks(a, nbytes, shift)
        c.repair_helpers(f, H, hin.ptrs(), recv.ptrs(), nbytes)
        c.repair_newcomer(f, H, recv.ptrs(), node.ptrs(), nbytes)
        assert node.guards_intact() and recv.guards_intact()
        assert np.array_equal(node.get(), Yfull[a * f:a * f + a]), ("repair", f, H)
        if a <= 16:
            fused = Blocks(a, nbytes, shift)
            c.repair(f, H, hin.ptrs(), fused.ptrs(), nbytes)
            assert np.array_equal(fused.get(), Yfull[a * f:a * f + a]), ("fused repair", f)
        if form and f < k and nbytes > 8:
            off = int(rng.integers(0, nbytes // 2))
            ln = int(rng.integers(1, nbytes - off + 1))
            part = Blocks(a, ln)
            c.read_degraded(f, H, hin.ptrs(), part.ptrs(), off, ln)
            assert np.array_equal(part.get(), X[a * f:a * f + a, off:off + ln]), "degraded read"
    # reconstruction from a random node set
    S = rng.permutation(rng.choice(n, k, replace=False)).tolist()
    rows = [a * i + j for i in S for j in range(a)]
    yin = Blocks(K, nbytes, shift, Yfull[rows])
    xout = Blocks(K, nbytes, shift)
    try:
        c.decode(S, yin.ptrs(), xout.ptrs(), nbytes)
    except P.PMRCError as e:
        # forced bitsliced reconstructions need aligned blocks and small rows
        assert e.rc == P.PMRC_EUNSUPPORTED and dec_k == P.PMRC_KERNEL_BITSLICED
        c.set_decode_kernel(P.PMRC_KERNEL_GENERIC)
        c.decode(S, yin.ptrs(), xout.ptrs(), nbytes)
    assert xout.guards_intact()
    assert np.array_equal(xout.get(), X), ("decode", S)


def _other(i):
    """A random PM-MBR, Reed-Solomon or GF(2^16) PM-MSR case."""
    rng = np.random.default_rng(5000 + i)
    kind = ("mbr", "rs", "gf16")[i % 3]
    if kind == "mbr":
        k = int(rng.integers(2, 8))
        n = int(rng.integers(k + 1, min(2 * k + 5, 24) + 1))
        d = int(rng.integers(k, n))
        c = P.Code(n, k, P.PMRC_MBR, int(rng.integers(0, 2)), d=d)
    elif kind == "rs":
        k = int(rng.integers(1, 12))
        n = int(rng.integers(k + 1, k + 10))
        c = P.Code(n, k, P.PMRC_RS, int(rng.integers(0, 2)))
    else:
        k = int(rng.integers(2, 7))
        n = int(rng.integers(2 * k - 1, 2 * k + 4))
        c = P.Code(n, k, int(rng.integers(0, 2)), int(rng.integers(0, 2)), field_bits=16)
    nbytes = 2 * int(rng.integers(1, 8000))
    shift = int(rng.choice([0, 16, 2 * int(rng.integers(1, 8))]))
    return rng, kind, c, nbytes, shift


def _oracle_codeword(kind, c, X):
    n, k, d = c.n, c.k, c.d
    sysf = c.form == P.PMRC_SYSTEMATIC
    if kind == "mbr":
        return O.mbr_encode(n, k, d, X)
    if kind == "rs":
        return O.rs_encode(n, k, sysf, X)
    return O.gf16_encode(n, k, c.construction, sysf, X)


@pytest.mark.parametrize("case", range(36))
def test_fuzz_other_codes(case):
    rng, kind, c, nbytes, shift = _other(case)
    n, k, a, K = c.n, c.k, c.alpha, c.data_blocks
    X = inputs.blocks(K, nbytes, seed=5000 + case)
    Y = _oracle_codeword(kind, c, X)
    first = k * a if c.form == P.PMRC_SYSTEMATIC else 0
    xin = Blocks(K, nbytes, shift, X)
    y = Blocks(c.n_outputs, nbytes, shift)
    c.encode(xin.ptrs(), y.ptrs(), nbytes)
    assert y.guards_intact()
    assert np.array_equal(y.get(), Y[first:]), (kind, "encode")
    f = int(rng.integers(0, n))
    H = c.default_helpers(f)
    if kind == "rs":
        hin = Blocks(k, nbytes, shift, Y[H])
        node = Blocks(1, nbytes, shift)
        c.repair(f, H, hin.ptrs(), node.ptrs(), nbytes)
    else:
        hin = Blocks(len(H) * a, nbytes, shift, np.concatenate([Y[a * h:a * h + a] for h in H]))
        recv = Blocks(len(H), nbytes, shift)
        node = Blocks(a, nbytes, shift)
        c.repair_helpers(f, H, hin.ptrs(), recv.ptrs(), nbytes)
        c.repair_newcomer(f, H, recv.ptrs(), node.ptrs(), nbytes)
    assert node.guards_intact()
    assert np.array_equal(node.get(), Y[a * f:a * f + a]), (kind, "repair", f)
    S = rng.permutation(rng.choice(n, k, replace=False)).tolist()
    rows = [a * i + j for i in S for j in range(a)]
    yin = Blocks(len(rows), nbytes, shift, Y[rows])
    xout = Blocks(K, nbytes, shift)
    c.decode(S, yin.ptrs(), xout.ptrs(), nbytes)
    assert xout.guards_intact()
    assert np.array_equal(xout.get(), X), (kind, "decode", S)
