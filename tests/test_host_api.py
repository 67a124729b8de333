"""CPU-only checks of libpmrc: it builds and loads, exports every symbol its
header declares, and its host-side matrices (generator, systematic form,
helper coefficients, newcomer and decode matrices) equal the oracle's byte
for byte.  No GPU work is launched here."""
import itertools
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_1412_3022_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pmrc_\w+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = P.lib()
    names = header_functions()
    assert "pmrc_create" in names and "pmrc_decode" in names
    for n in names:
        assert hasattr(L, n), n


CODES = [(5, 3), (6, 3), (8, 4), (16, 8), (24, 12), (32, 16), (9, 5)]


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("cons", [0, 1])
@pytest.mark.parametrize("n,k", CODES)
def test_generator_matches_oracle(n, k, cons, form):
    if cons == 0 and (n, k) == (32, 16):
        with pytest.raises(P.PMRCError) as e:
            P.Code(n, k, cons, form)
        assert e.value.rc == P.PMRC_EUNSUPPORTED
        return
    c = P.Code(n, k, cons, form)
    assert np.array_equal(c.generator(), O.generator(n, k, cons, systematic=bool(form)))


@pytest.mark.parametrize("cons", [0, 1])
@pytest.mark.parametrize("n,k", [(6, 3), (8, 4), (16, 8)])
def test_repair_and_decode_matrices_match_oracle(n, k, cons):
    c = P.Code(n, k, cons, 1)
    d = 2 * k - 2
    rng = np.random.default_rng(n * 100 + k)
    for f in range(n):
        assert np.array_equal(c.helper_coefficients(f), O.helper_coefficients(n, k, cons, f))
        H = c.default_helpers(f)
        assert len(H) == d and f not in H and len(set(H)) == d
        assert np.array_equal(c.newcomer_matrix(f, H), O.newcomer_matrix(n, k, cons, f, H))
        Hs = list(rng.permutation(H))
        assert np.array_equal(c.newcomer_matrix(f, Hs), O.newcomer_matrix(n, k, cons, f, Hs))
    subsets = list(itertools.combinations(range(n), k))
    for i in rng.choice(len(subsets), min(30, len(subsets)), replace=False):
        S = list(subsets[i])
        assert np.array_equal(c.decode_matrix(S), O.decode_matrix(n, k, cons, True, S))


@pytest.mark.parametrize("k", [3, 4, 8, 12, 16])
def test_default_helpers_valid_for_every_node(k):
    n = 2 * k
    c = P.Code(n, k, 1, 1)
    for f in range(n):
        H = c.default_helpers(f)
        O.newcomer_matrix(n, k, 1, f, H)  # the oracle agrees it is invertible


def test_error_statuses():
    with pytest.raises(P.PMRCError) as e:
        P.pmrc_create(16, 8, 13, 1, 1)          # d != 2k-2
    assert e.value.rc == P.PMRC_EINVAL
    with pytest.raises(P.PMRCError) as e:
        P.pmrc_create(14, 8, 14, 1, 1)          # n < 2k-1
    assert e.value.rc == P.PMRC_EINVAL
    with pytest.raises(P.PMRCError) as e:
        P.pmrc_create(16, 8, 14, 3, 1)          # construction
    assert e.value.rc == P.PMRC_EINVAL
    c = P.Code(8, 4, 1, 1)
    with pytest.raises(P.PMRCError) as e:
        c.newcomer_matrix(0, [1, 1, 2, 3, 4, 5])  # repeated helper
    assert e.value.rc == P.PMRC_EINVAL
    with pytest.raises(P.PMRCError) as e:
        c.newcomer_matrix(0, [0, 1, 2, 3, 4, 5])  # failed node helps
    assert e.value.rc == P.PMRC_EINVAL
    with pytest.raises(P.PMRCError) as e:
        c.newcomer_matrix(0, [2, 3, 4, 5, 6, 7])  # leaves out 0 and 1 (both < alpha)
    assert e.value.rc == P.PMRC_ESINGULAR
    with pytest.raises(P.PMRCError) as e:
        c.decode_matrix([0, 1, 2, 2])
    assert e.value.rc == P.PMRC_EINVAL
    assert "repeated" in P.pmrc_last_error()
    # calls that validate before touching the GPU
    with pytest.raises(P.PMRCError) as e:
        c.repair_newcomer(0, [2, 3, 4, 5, 6, 7], [0] * 6, [0] * 3, 16)
    assert e.value.rc == P.PMRC_EINVAL  # NULL outputs are rejected first
    with pytest.raises(P.PMRCError) as e:
        c.decode([0, 1, 2, 9], [0] * 12, [0] * 12, 16)
    assert e.value.rc == P.PMRC_EINVAL


def test_plan_structure():
    """The planner turns PM generators into dense blocks (rows of one slot
    share the symbols of one column of the message matrix, Sec. 3.1) and keeps
    block-diagonal matrices (batched helper projections) apart."""
    import oracle as O2
    n, k, a = 16, 8, 7
    G2 = O2.generator(n, k, 1, True)[k * a:]
    st = P.pmrc_plan_stats(G2)
    assert st == {"blocks": 7, "R": 8, "entries": 784, "input_splits": 98, "nnz": 784}
    G = O2.generator(n, k, 0, False)
    st = P.pmrc_plan_stats(G)
    assert st["blocks"] == 7 and st["R"] == 16 and st["entries"] == st["nnz"] == 1568
    phi = O2.helper_coefficients(n, k, 1, 12)
    M = np.zeros((14, 14 * a), np.uint8)
    for h in range(14):
        M[h, h * a:(h + 1) * a] = phi
    st = P.pmrc_plan_stats(M)
    assert st["blocks"] == 14 and st["R"] == 1 and st["entries"] == st["nnz"] == 98
    # a decode matrix: merging may add zero products but never more than it saves
    c = P.Code(n, k, 1, 1)
    R = c.decode_matrix([0, 1, 4, 5, 7, 8, 11, 12])
    miss = [r for r in range(56) if r // a not in (0, 1, 4, 5, 7)]
    st = P.pmrc_plan_stats(R[miss])
    assert st["entries"] <= 1.5 * st["nnz"]


def test_plans_above_one_launch_are_cut_into_parts():
    """Matrices above 1024 block pointers, or with blocks whose split tables
    would overflow shared memory, run as parts: every non-zero coefficient
    is still planned exactly once, and a block-diagonal matrix (helper
    projections of a k = 32 code) needs no zero products or accumulation."""
    a = 31
    phi = np.arange(1, a + 1, dtype=np.uint8)
    M = np.zeros((62, 62 * a), np.uint8)
    for h in range(62):
        M[h, h * a:(h + 1) * a] = phi
    st = P.pmrc_plan_stats(M)
    assert st["nnz"] == st["entries"] == 62 * a and st["R"] == 1
    assert st["input_splits"] == 62 * a            # each helper block read once
    rng = np.random.default_rng(5)
    D = rng.integers(0, 256, (700, 600), dtype=np.uint8)  # dense rows of 600 inputs
    st = P.pmrc_plan_stats(D)
    assert st["nnz"] == int((D != 0).sum())
    assert st["R"] <= 16 and st["entries"] >= st["nnz"]
    # 600 columns > 512 per part: every block reads one of two 300-input chunks
    assert st["input_splits"] == 300 * st["blocks"]
    S = rng.integers(0, 256, (300, 900), dtype=np.uint8) * (rng.random((300, 900)) < 0.05)
    st = P.pmrc_plan_stats(S.astype(np.uint8))
    assert st["nnz"] == int((S != 0).sum())


@pytest.mark.parametrize("n,k", [(48, 24), (64, 32)])
def test_codes_beyond_one_launch_are_created(n, k):
    """k >= 24 at n = 2k needs more than 1024 block pointers per encode; the
    code is built (its operations run as several launches)."""
    for cons, form in [(P.PMRC_SPARSE, P.PMRC_SYSTEMATIC), (P.PMRC_VANILLA, P.PMRC_NONSYSTEMATIC)]:
        c = P.Code(n, k, cons, form)
        assert (c.alpha, c.data_blocks, c.coded_blocks) == (k - 1, k * (k - 1), n * (k - 1))
    if k == 24:
        G = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC).generator()
        assert np.array_equal(G, O.generator(n, k, 1, systematic=True))


def test_encode_kernel_choice():
    for n, k, cons, form in [(16, 8, 1, 1), (16, 8, 0, 0), (8, 4, 1, 1)]:
        c = P.Code(n, k, cons, form)
        c.set_encode_kernel(P.PMRC_KERNEL_BITSLICED)
        c.set_encode_kernel(P.PMRC_KERNEL_GENERIC)
    # no built-in schedule: a run-time one when the encode matrix fits it
    # (k = 12: 264 blocks, 22 blocks of 22 inputs), unless NVRTC is missing
    c = P.Code(24, 12, 1, 1)
    try:
        c.set_encode_kernel(P.PMRC_KERNEL_BITSLICED)
    except P.PMRCError as e:
        assert e.rc == P.PMRC_EUNSUPPORTED and "NVRTC" in str(e)
    c.set_encode_kernel(P.PMRC_KERNEL_AUTO)
    # too large for one bitsliced launch (1984 block pointers)
    c = P.Code(64, 32, 1, 1)
    with pytest.raises(P.PMRCError) as e:
        c.set_encode_kernel(P.PMRC_KERNEL_BITSLICED)
    assert e.value.rc == P.PMRC_EUNSUPPORTED
    c.set_encode_kernel(P.PMRC_KERNEL_GENERIC)


@pytest.mark.parametrize("S", [list(range(16)), list(range(16, 32)),
                               [0, 2, 3, 5, 7, 11, 13, 17, 19, 20, 21, 22, 23, 27, 29, 31],
                               [31, 1, 17, 4, 30, 6, 8, 25, 10, 12, 14, 15, 18, 20, 22, 24]])
def test_k16_systematic_decode_matrix_matches_full_inverse(S):
    """The library inverts only the block of missing data columns for the
    systematic form; the rows must equal the oracle's full inverse."""
    c = P.Code(32, 16, 1, 1)
    assert np.array_equal(c.decode_matrix(S), O.decode_matrix(32, 16, 1, True, S))


# ------------------------------------------------------------------ PM-MBR
MBR_CASES = [(6, 3, 4), (8, 4, 6), (8, 4, 7), (16, 8, 14), (16, 8, 15), (32, 16, 30)]


@pytest.mark.parametrize("n,k,d", MBR_CASES)
def test_mbr_matrices_match_oracle(n, k, d):
    c = P.Code(n, k, P.PMRC_MBR, P.PMRC_SYSTEMATIC, d=d)
    a, B = O.mbr_params(n, k, d)
    assert (c.alpha, c.data_blocks, c.coded_blocks) == (a, B, n * a)
    assert np.array_equal(P.pmrc_code_generator(c.handle), O.mbr_generator(n, k, d))
    rng = np.random.default_rng(n + d)
    for f in range(n):
        H = c.default_helpers(f)
        assert f not in H and len(set(H)) == d
        assert np.array_equal(P.pmrc_helper_coefficients(c.handle, f),
                              O.mbr_helper_coefficients(n, k, d, f))
        H2 = rng.permutation([h for h in range(n) if h != f])[:d].tolist()
        assert np.array_equal(P.pmrc_newcomer_matrix(c.handle, f, H2),
                              O.mbr_newcomer_matrix(n, k, d, f, H2))
    X = rng.integers(0, 256, (B, 3), dtype=np.uint8)
    Y = O.mbr_encode(n, k, d, X)
    for _ in range(6):   # the decode matrix may pick other rows than the oracle's
        S = rng.permutation(rng.choice(n, k, replace=False)).tolist()
        R = P.pmrc_decode_matrix(c.handle, S)
        assert R.shape == (B, k * a)
        assert np.array_equal(O.region_apply(R, Y[[a * i + j for i in S for j in range(a)]]), X)


def test_mbr_create_rejects_bad_points():
    for n, k, d in [(8, 4, 3), (8, 4, 8), (8, 0, 4)]:
        with pytest.raises(P.PMRCError) as e:
            P.Code(n, k, P.PMRC_MBR, P.PMRC_SYSTEMATIC, d=d)
        assert e.value.rc == P.PMRC_EINVAL
    c = P.Code(8, 4, P.PMRC_MBR, P.PMRC_SYSTEMATIC, d=6)
    assert c.specific_workspace_bytes(4096) == 0
    with pytest.raises(P.PMRCError) as e:   # PM-MSR data collector only
        c.decode_specific([0, 1, 2, 3], [0] * 24, [0] * 18, 4096, 1 << 20, 1 << 20)
    assert e.value.rc == P.PMRC_EUNSUPPORTED


def test_mbr_encode_plan_is_sparse():
    """Parity rows touch d or k data blocks (Sec. 4.2: naturally sparse)."""
    c = P.Code(16, 8, P.PMRC_MBR, P.PMRC_SYSTEMATIC, d=14)
    G = P.pmrc_code_generator(c.handle)
    par = G[8 * 14:]
    st = P.pmrc_plan_stats(par)
    assert st["nnz"] == int((par != 0).sum()) == 8 * (8 * 14 + 6 * 8)


# ------------------------------------------------------------ Reed-Solomon
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("n,k", [(6, 3), (9, 6), (16, 8), (32, 16)])
def test_rs_matrices_match_oracle(n, k, form):
    c = P.Code(n, k, P.PMRC_RS, form)
    assert (c.alpha, c.d, c.data_blocks, c.coded_blocks) == (1, k, k, n)
    assert np.array_equal(P.pmrc_code_generator(c.handle), O.rs_generator(n, k, bool(form)))
    X = np.random.default_rng(n).integers(0, 256, (k, 3), dtype=np.uint8)
    Y = O.rs_encode(n, k, bool(form), X)
    rng = np.random.default_rng(k)
    for f in range(n):
        H = rng.permutation([h for h in range(n) if h != f])[:k].tolist()
        assert list(P.pmrc_helper_coefficients(c.handle, f)) == [1]
        D = P.pmrc_newcomer_matrix(c.handle, f, H)
        assert np.array_equal(O.region_apply(D, Y[H])[0], O.rs_repair(n, k, bool(form), f, H, Y[H]))
    for _ in range(5):
        S = rng.permutation(rng.choice(n, k, replace=False)).tolist()
        R = P.pmrc_decode_matrix(c.handle, S)
        assert np.array_equal(O.region_apply(R, Y[S]), X)


def test_rs_rejects_bad_parameters():
    for n, k, d in [(8, 4, 6), (4, 4, 4), (300, 8, 8)]:
        with pytest.raises(P.PMRCError) as e:
            P.pmrc_create(n, k, d, P.PMRC_RS, 1)
        assert e.value.rc == P.PMRC_EINVAL


# ------------------------------------------------------------ GF(2^16)
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("cons", [0, 1])
@pytest.mark.parametrize("n,k", [(5, 3), (8, 4), (16, 8)])
def test_gf16_generator_matches_oracle(n, k, cons, form):
    c = P.Code(n, k, cons, form, field_bits=16)
    assert P.pmrc_code_field_bits(c.handle) == 16
    assert (c.alpha, c.data_blocks, c.coded_blocks) == (k - 1, k * (k - 1), n * (k - 1))
    assert np.array_equal(P.pmrc_code_generator16(c.handle),
                          O.gf16_generator(n, k, cons, bool(form)))


def test_gf16_vanilla_k16_valid_and_errors():
    c = P.Code(32, 16, P.PMRC_VANILLA, P.PMRC_SYSTEMATIC, field_bits=16)   # invalid in GF(2^8)
    assert np.array_equal(P.pmrc_code_generator16(c.handle),
                          O.gf16_generator(32, 16, O.VANILLA, True))
    with pytest.raises(P.PMRCError) as e:
        P.pmrc_create_field(8, 4, 6, P.PMRC_SPARSE, 1, 12)
    assert e.value.rc == P.PMRC_EINVAL
    with pytest.raises(P.PMRCError) as e:
        P.pmrc_create_field(16, 8, 14, P.PMRC_MBR, 1, 16)
    assert e.value.rc == P.PMRC_EINVAL
    c = P.Code(8, 4, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC, field_bits=16)
    with pytest.raises(P.PMRCError) as e:   # fused repair is GF(2^8) only
        c.repair(5, c.default_helpers(5), [1] * 18, [1] * 3, 64)
    assert e.value.rc == P.PMRC_EUNSUPPORTED
    with pytest.raises(P.PMRCError) as e:   # whole 2-byte symbols
        c.encode([1] * 12, [1] * 12, 63)
    assert e.value.rc == P.PMRC_EINVAL
    for f in range(8):
        H = c.default_helpers(f)
        O.gf16_newcomer_matrix(8, 4, O.SPARSE, f, H)   # the oracle agrees it is invertible


def test_degraded_read_argument_checks():
    """Refused before any device work: a non-systematic handle, a node that
    is not systematic."""
    H = list(range(1, 15))
    blocks, out = [0] * (14 * 7), [0] * 7
    c = P.Code(16, 8, P.PMRC_SPARSE, P.PMRC_NONSYSTEMATIC)
    with pytest.raises(P.PMRCError) as e:
        P.pmrc_read_degraded(c.handle, 2, H, blocks, out, 0, 16)
    assert e.value.rc == P.PMRC_EINVAL
    c = P.Code(16, 8, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    for node in (8, 15, -1):
        with pytest.raises(P.PMRCError) as e:
            P.pmrc_read_degraded(c.handle, node, H, blocks, out, 0, 16)
        assert e.value.rc == P.PMRC_EINVAL


def test_runtime_kernel_queries_on_a_fresh_handle():
    """Nothing compiled or compiling before any call (host only)."""
    c = P.Code(16, 8, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    assert c.runtime_kernels() == (0, 0)
    c.wait_kernels(0)
    c.wait_kernels()
    P.wait_kernels(0)
