"""CPU oracle for product-matrix MSR regenerating codes.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow statement of the
method (Le Scouarnec, "Fast Product-Matrix Regenerating Codes") that the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library in
``paper_1412_3022_gb300`` never does, and this package never imports the
library.

The arithmetic lives in ``pmrc_oracle.c`` (plain C, log/antilog GF(2^8) with
modulus 0x11D and generator 2, Gauss-Jordan inverses, byte-at-a-time region
work).  This module only compiles it with gcc and marshals numpy arrays.

Parity status per function (what pins it is in ``tests/test_oracle_pins.py``):
  gf_mul / gf_inv            pinned: field axioms by brute force and an
                             independent shift-and-reduce multiply
  phi_lambda / psi           pinned: the paper's printed n=5, k=3 matrices
                             (Sec. 3.3), Table 1, the k<=39 validity range
  generator                  pinned: equals Psi*M(X) computed as a matrix
                             product (Sec. 3.1), Table 1
  systematic_generator       pinned: identity on top (Sec. 3.2), Table 1
  region_apply / encode      pinned: brute-force definition on tiny inputs
  repair_*                   pinned: repair reproduces every node exactly
  decode                     pinned: every k-subset recovers the data
  dc_decode / decode_specific
                             pinned: every k-subset (n <= 8) and sampled
                             subsets at n = 16 recover the data exactly
  encode_precode             pinned: data as nodes 0..k-1 re-decodes to itself
                             and every k-subset of the result recovers the data
  gf16_* (GF(2^16) variant)  pinned: the tower multiply against an
                             independent GF(2^8) shift-and-reduce, w has
                             trace 1 (no root), g has order 65535, inverses;
                             linearization vs Psi M(X); repair from every
                             helper set and decode from every k-subset (n <= 8)
  rs_*                       pinned: V Z is polynomial evaluation (Horner,
                             independent multiply); systematic identity top;
                             every k-subset decodes and every node repairs
                             from every k helpers (small n), sampled at n=16
  mbr_*                      pinned: k Delta = k(2d-k+1)/2 and alpha = d
                             (Sec. 2); G X equals Psi M(X); systematic nodes
                             hold the symbols verbatim; any d rows of Psi and
                             any k rows of Phi independent; repair of every
                             node from every helper set and decode from every
                             k-subset are exact (small n)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmrc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

VANILLA = 0
SPARSE = 1

OK = 0
EINVAL = -1
ESINGULAR = -2


class OracleError(RuntimeError):
    def __init__(self, rc: int, what: str):
        super().__init__(f"oracle {what} failed with status {rc}")
        self.rc = rc


def build(force: bool = False) -> str:
    """Compile pmrc_oracle.c into liboracle.so next to it (gcc, no GPU)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u16p = ctypes.POINTER(ctypes.c_uint16)
            ip = ctypes.POINTER(ctypes.c_int)
            i, sz = ctypes.c_int, ctypes.c_size_t
            sig = {
                "or_gf_mul": (ctypes.c_uint8, [ctypes.c_uint8, ctypes.c_uint8]),
                "or_gf_inv": (ctypes.c_uint8, [ctypes.c_uint8]),
                "or_gf_pow_g": (ctypes.c_uint8, [i]),
                "or_gf_log": (i, [ctypes.c_uint8]),
                "or_invert": (i, [i, u8p, u8p]),
                "or_mat_mul": (None, [i, i, i, u8p, u8p, u8p]),
                "or_params": (i, [i, i, ip, ip]),
                "or_phi_lambda": (i, [i, i, i, u8p, u8p]),
                "or_psi": (i, [i, i, i, u8p]),
                "or_index_matrix": (i, [i, ip]),
                "or_generator": (i, [i, i, i, u8p]),
                "or_systematic_generator": (i, [i, i, i, u8p]),
                "or_code_generator": (i, [i, i, i, i, u8p]),
                "or_region_apply": (None, [i, i, u8p, u8p, sz, u8p, sz, sz]),
                "or_encode": (i, [i, i, i, i, u8p, u8p, sz]),
                "or_helper_coefficients": (i, [i, i, i, i, u8p]),
                "or_repair_helper": (i, [i, i, i, i, u8p, u8p, sz]),
                "or_newcomer_matrix": (i, [i, i, i, i, ip, u8p]),
                "or_repair_newcomer": (i, [i, i, i, i, ip, u8p, u8p, sz]),
                "or_decode_matrix": (i, [i, i, i, i, ip, u8p]),
                "or_decode": (i, [i, i, i, i, ip, u8p, u8p, sz]),
                "or_dc_decode": (i, [i, i, i, ip, u8p, u8p, sz]),
                "or_decode_specific": (i, [i, i, i, i, ip, u8p, u8p, sz]),
                "or_encode_precode": (i, [i, i, i, u8p, u8p, sz]),
                "or_mbr_params": (i, [i, i, i, ip, ip]),
                "or_mbr_psi": (i, [i, i, i, u8p]),
                "or_mbr_index_matrix": (i, [i, i, ip]),
                "or_mbr_generator": (i, [i, i, i, u8p]),
                "or_mbr_encode": (i, [i, i, i, u8p, u8p, sz]),
                "or_mbr_helper_coefficients": (i, [i, i, i, i, u8p]),
                "or_mbr_newcomer_matrix": (i, [i, i, i, i, ip, u8p]),
                "or_mbr_decode_matrix": (i, [i, i, i, ip, u8p]),
                "or_mbr_decode": (i, [i, i, i, ip, u8p, u8p, sz]),
                "or_rs_generator": (i, [i, i, i, u8p]),
                "or_rs_encode": (i, [i, i, i, u8p, u8p, sz]),
                "or_rs_decode": (i, [i, i, i, ip, u8p, u8p, sz]),
                "or_rs_repair": (i, [i, i, i, i, ip, u8p, u8p, sz]),
                "or16_omega": (ctypes.c_uint8, []),
                "or16_primitive": (ctypes.c_uint16, []),
                "or16_gf_mul": (ctypes.c_uint16, [ctypes.c_uint16, ctypes.c_uint16]),
                "or16_gf_inv": (ctypes.c_uint16, [ctypes.c_uint16]),
                "or16_gf_pow_g": (ctypes.c_uint16, [i]),
                "or16_phi_lambda": (i, [i, i, i, u16p, u16p]),
                "or16_psi": (i, [i, i, i, u16p]),
                "or16_code_generator": (i, [i, i, i, i, u16p]),
                "or16_region_apply": (None, [i, i, u16p, u8p, u8p, sz]),
                "or16_encode": (i, [i, i, i, i, u8p, u8p, sz]),
                "or16_newcomer_matrix": (i, [i, i, i, i, ip, u16p]),
                "or16_helper_coefficients": (i, [i, i, i, i, u16p]),
                "or16_decode_matrix": (i, [i, i, i, i, ip, u16p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def _u8(a: np.ndarray):
    assert a.dtype == np.uint8 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _ints(seq) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(seq, dtype=np.int32))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _check(rc: int, what: str):
    if rc != OK:
        raise OracleError(rc, what)


# ----------------------------------------------------------------- field
def gf_mul(a: int, b: int) -> int:
    return int(lib().or_gf_mul(a, b))


def gf_inv(a: int) -> int:
    return int(lib().or_gf_inv(a))


def gf_pow_g(e: int) -> int:
    return int(lib().or_gf_pow_g(e))


def gf_mul_table() -> np.ndarray:
    """256x256 table T[a, b] = a*b, filled by calling or_gf_mul."""
    L = lib()
    return np.array([[L.or_gf_mul(a, b) for b in range(256)] for a in range(256)],
                    dtype=np.uint8)


def invert(A: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.uint8)
    m = A.shape[0]
    out = np.zeros((m, m), np.uint8)
    _check(lib().or_invert(m, _u8(A), _u8(out)), "invert")
    return out


def mat_mul(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.uint8)
    C = np.zeros((A.shape[0], B.shape[1]), np.uint8)
    lib().or_mat_mul(A.shape[0], A.shape[1], B.shape[1], _u8(A), _u8(B), _u8(C))
    return C


# ----------------------------------------------------------------- code
def params(n: int, k: int):
    d, a = ctypes.c_int(), ctypes.c_int()
    _check(lib().or_params(n, k, ctypes.byref(d), ctypes.byref(a)), "params")
    return d.value, a.value


def phi_lambda(n: int, k: int, construction: int):
    d, a = params(n, k)
    phi = np.zeros((n, a), np.uint8)
    lam = np.zeros(n, np.uint8)
    _check(lib().or_phi_lambda(n, k, construction, _u8(phi), _u8(lam)), "phi_lambda")
    return phi, lam


def psi(n: int, k: int, construction: int) -> np.ndarray:
    d, a = params(n, k)
    P = np.zeros((n, d), np.uint8)
    _check(lib().or_psi(n, k, construction, _u8(P)), "psi")
    return P


def index_matrix(k: int) -> np.ndarray:
    a, d = k - 1, 2 * k - 2
    L = np.zeros((d, a), np.int32)
    _check(lib().or_index_matrix(k, _ip(L)), "index_matrix")
    return L


def generator(n: int, k: int, construction: int, systematic: bool = False) -> np.ndarray:
    d, a = params(n, k)
    G = np.zeros((n * a, k * a), np.uint8)
    _check(lib().or_code_generator(n, k, construction, int(systematic), _u8(G)),
           "generator")
    return G


def region_apply(M: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Y = M X over byte blocks: X is (cols, B) uint8, returns (rows, B)."""
    M = np.ascontiguousarray(M, dtype=np.uint8)
    X = np.ascontiguousarray(X, dtype=np.uint8)
    rows, cols = M.shape
    assert X.shape[0] == cols
    B = X.shape[1]
    Y = np.zeros((rows, B), np.uint8)
    if B:
        lib().or_region_apply(rows, cols, _u8(M), _u8(X), B, _u8(Y), B, B)
    return Y


def encode(n: int, k: int, construction: int, systematic: bool, data: np.ndarray) -> np.ndarray:
    """All n*alpha coded blocks (node-major) of the k*alpha data blocks."""
    d, a = params(n, k)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    assert data.shape[0] == k * a
    B = data.shape[1]
    out = np.zeros((n * a, B), np.uint8)
    _check(lib().or_encode(n, k, construction, int(systematic), _u8(data), _u8(out), B),
           "encode")
    return out


def helper_coefficients(n: int, k: int, construction: int, f: int) -> np.ndarray:
    d, a = params(n, k)
    c = np.zeros(a, np.uint8)
    _check(lib().or_helper_coefficients(n, k, construction, f, _u8(c)), "helper_coefficients")
    return c


def repair_helper(n: int, k: int, construction: int, f: int, blocks: np.ndarray) -> np.ndarray:
    d, a = params(n, k)
    blocks = np.ascontiguousarray(blocks, dtype=np.uint8)
    assert blocks.shape[0] == a
    B = blocks.shape[1]
    out = np.zeros(B, np.uint8)
    _check(lib().or_repair_helper(n, k, construction, f, _u8(blocks), _u8(out), B),
           "repair_helper")
    return out


def newcomer_matrix(n: int, k: int, construction: int, f: int, helpers) -> np.ndarray:
    d, a = params(n, k)
    h = _ints(helpers)
    assert h.size == d
    D = np.zeros((a, d), np.uint8)
    _check(lib().or_newcomer_matrix(n, k, construction, f, _ip(h), _u8(D)), "newcomer_matrix")
    return D


def repair_newcomer(n: int, k: int, construction: int, f: int, helpers, recv: np.ndarray) -> np.ndarray:
    d, a = params(n, k)
    h = _ints(helpers)
    recv = np.ascontiguousarray(recv, dtype=np.uint8)
    assert recv.shape[0] == d and h.size == d
    B = recv.shape[1]
    out = np.zeros((a, B), np.uint8)
    _check(lib().or_repair_newcomer(n, k, construction, f, _ip(h), _u8(recv), _u8(out), B),
           "repair_newcomer")
    return out


def decode_matrix(n: int, k: int, construction: int, systematic: bool, nodes) -> np.ndarray:
    d, a = params(n, k)
    s = _ints(nodes)
    assert s.size == k
    R = np.zeros((k * a, k * a), np.uint8)
    _check(lib().or_decode_matrix(n, k, construction, int(systematic), _ip(s), _u8(R)),
           "decode_matrix")
    return R


def decode(n: int, k: int, construction: int, systematic: bool, nodes, node_blocks: np.ndarray) -> np.ndarray:
    d, a = params(n, k)
    s = _ints(nodes)
    node_blocks = np.ascontiguousarray(node_blocks, dtype=np.uint8)
    assert node_blocks.shape[0] == k * a and s.size == k
    B = node_blocks.shape[1]
    out = np.zeros((k * a, B), np.uint8)
    _check(lib().or_decode(n, k, construction, int(systematic), _ip(s), _u8(node_blocks),
                           _u8(out), B), "decode")
    return out


def dc_decode(n: int, k: int, construction: int, nodes, node_blocks: np.ndarray) -> np.ndarray:
    """The data collector's message recovery (k*alpha message blocks)."""
    d, a = params(n, k)
    s = _ints(nodes)
    node_blocks = np.ascontiguousarray(node_blocks, dtype=np.uint8)
    assert node_blocks.shape[0] == k * a and s.size == k
    B = node_blocks.shape[1]
    out = np.zeros((k * a, B), np.uint8)
    _check(lib().or_dc_decode(n, k, construction, _ip(s), _u8(node_blocks), _u8(out), B),
           "dc_decode")
    return out


def decode_specific(n: int, k: int, construction: int, systematic: bool, nodes,
                    node_blocks: np.ndarray) -> np.ndarray:
    d, a = params(n, k)
    s = _ints(nodes)
    node_blocks = np.ascontiguousarray(node_blocks, dtype=np.uint8)
    assert node_blocks.shape[0] == k * a and s.size == k
    B = node_blocks.shape[1]
    out = np.zeros((k * a, B), np.uint8)
    _check(lib().or_decode_specific(n, k, construction, int(systematic), _ip(s),
                                    _u8(node_blocks), _u8(out), B), "decode_specific")
    return out


def encode_precode(n: int, k: int, construction: int, data: np.ndarray) -> np.ndarray:
    """Parity blocks ((n-k)*alpha) of the systematic code, by decoding then encoding."""
    d, a = params(n, k)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    assert data.shape[0] == k * a
    B = data.shape[1]
    out = np.zeros(((n - k) * a, B), np.uint8)
    _check(lib().or_encode_precode(n, k, construction, _u8(data), _u8(out), B), "encode_precode")
    return out


# ------------------------------------------------------------------ PM-MBR
def mbr_params(n: int, k: int, d: int):
    a = ctypes.c_int()
    B = ctypes.c_int()
    _check(lib().or_mbr_params(n, k, d, ctypes.byref(a), ctypes.byref(B)), "mbr_params")
    return a.value, B.value


def mbr_psi(n: int, k: int, d: int) -> np.ndarray:
    P = np.zeros((n, d), np.uint8)
    _check(lib().or_mbr_psi(n, k, d, _u8(P)), "mbr_psi")
    return P


def mbr_index_matrix(k: int, d: int) -> np.ndarray:
    L = np.zeros((d, d), np.int32)
    _check(lib().or_mbr_index_matrix(k, d, _ip(L)), "mbr_index_matrix")
    return L


def mbr_generator(n: int, k: int, d: int) -> np.ndarray:
    a, B = mbr_params(n, k, d)
    G = np.zeros((n * a, B), np.uint8)
    _check(lib().or_mbr_generator(n, k, d, _u8(G)), "mbr_generator")
    return G


def mbr_encode(n: int, k: int, d: int, data: np.ndarray) -> np.ndarray:
    a, B = mbr_params(n, k, d)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    assert data.shape[0] == B
    out = np.zeros((n * a, data.shape[1]), np.uint8)
    _check(lib().or_mbr_encode(n, k, d, _u8(data), _u8(out), data.shape[1]), "mbr_encode")
    return out


def mbr_helper_coefficients(n: int, k: int, d: int, f: int) -> np.ndarray:
    c = np.zeros(d, np.uint8)
    _check(lib().or_mbr_helper_coefficients(n, k, d, f, _u8(c)), "mbr_helper_coefficients")
    return c


def mbr_repair_helper(n: int, k: int, d: int, f: int, blocks: np.ndarray) -> np.ndarray:
    return region_apply(mbr_helper_coefficients(n, k, d, f)[None, :], blocks)[0]


def mbr_newcomer_matrix(n: int, k: int, d: int, f: int, helpers) -> np.ndarray:
    h = _ints(helpers)
    D = np.zeros((d, d), np.uint8)
    _check(lib().or_mbr_newcomer_matrix(n, k, d, f, _ip(h), _u8(D)), "mbr_newcomer_matrix")
    return D


def mbr_repair_newcomer(n: int, k: int, d: int, f: int, helpers, recv: np.ndarray) -> np.ndarray:
    return region_apply(mbr_newcomer_matrix(n, k, d, f, helpers), recv)


def mbr_decode_matrix(n: int, k: int, d: int, nodes) -> np.ndarray:
    a, B = mbr_params(n, k, d)
    s = _ints(nodes)
    R = np.zeros((B, k * a), np.uint8)
    _check(lib().or_mbr_decode_matrix(n, k, d, _ip(s), _u8(R)), "mbr_decode_matrix")
    return R


def mbr_decode(n: int, k: int, d: int, nodes, node_blocks: np.ndarray) -> np.ndarray:
    a, B = mbr_params(n, k, d)
    s = _ints(nodes)
    node_blocks = np.ascontiguousarray(node_blocks, dtype=np.uint8)
    assert node_blocks.shape[0] == k * a
    out = np.zeros((B, node_blocks.shape[1]), np.uint8)
    _check(lib().or_mbr_decode(n, k, d, _ip(s), _u8(node_blocks), _u8(out),
                               node_blocks.shape[1]), "mbr_decode")
    return out


# ------------------------------------------------------------ Reed-Solomon
def rs_generator(n: int, k: int, systematic: bool = True) -> np.ndarray:
    G = np.zeros((n, k), np.uint8)
    _check(lib().or_rs_generator(n, k, int(systematic), _u8(G)), "rs_generator")
    return G


def rs_encode(n: int, k: int, systematic: bool, data: np.ndarray) -> np.ndarray:
    data = np.ascontiguousarray(data, dtype=np.uint8)
    assert data.shape[0] == k
    out = np.zeros((n, data.shape[1]), np.uint8)
    _check(lib().or_rs_encode(n, k, int(systematic), _u8(data), _u8(out), data.shape[1]),
           "rs_encode")
    return out


def rs_decode(n: int, k: int, systematic: bool, nodes, node_blocks: np.ndarray) -> np.ndarray:
    s = _ints(nodes)
    node_blocks = np.ascontiguousarray(node_blocks, dtype=np.uint8)
    out = np.zeros((k, node_blocks.shape[1]), np.uint8)
    _check(lib().or_rs_decode(n, k, int(systematic), _ip(s), _u8(node_blocks), _u8(out),
                              node_blocks.shape[1]), "rs_decode")
    return out


def rs_repair(n: int, k: int, systematic: bool, f: int, helpers, helper_blocks: np.ndarray) -> np.ndarray:
    h = _ints(helpers)
    helper_blocks = np.ascontiguousarray(helper_blocks, dtype=np.uint8)
    out = np.zeros((1, helper_blocks.shape[1]), np.uint8)
    _check(lib().or_rs_repair(n, k, int(systematic), f, _ip(h), _u8(helper_blocks), _u8(out),
                              helper_blocks.shape[1]), "rs_repair")
    return out[0]


# ------------------------------------------------------------ GF(2^16)
def _u16(a: np.ndarray):
    assert a.dtype == np.uint16 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16))


def gf16_omega() -> int:
    return int(lib().or16_omega())


def gf16_primitive() -> int:
    return int(lib().or16_primitive())


def gf16_mul(a: int, b: int) -> int:
    return int(lib().or16_gf_mul(a, b))


def gf16_inv(a: int) -> int:
    return int(lib().or16_gf_inv(a))


def gf16_phi_lambda(n: int, k: int, construction: int):
    d, a = params(n, k)
    phi = np.zeros((n, a), np.uint16)
    lam = np.zeros(n, np.uint16)
    _check(lib().or16_phi_lambda(n, k, construction, _u16(phi), _u16(lam)), "gf16_phi_lambda")
    return phi, lam


def gf16_psi(n: int, k: int, construction: int) -> np.ndarray:
    d, a = params(n, k)
    P = np.zeros((n, d), np.uint16)
    _check(lib().or16_psi(n, k, construction, _u16(P)), "gf16_psi")
    return P


def gf16_generator(n: int, k: int, construction: int, systematic: bool) -> np.ndarray:
    d, a = params(n, k)
    G = np.zeros((n * a, k * a), np.uint16)
    _check(lib().or16_code_generator(n, k, construction, int(systematic), _u16(G)),
           "gf16_generator")
    return G


def gf16_region_apply(M: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Y = M X over planar GF(2^16) blocks (rows of X: B bytes, B even)."""
    M = np.ascontiguousarray(M, dtype=np.uint16)
    X = np.ascontiguousarray(X, dtype=np.uint8)
    rows, cols = M.shape
    assert X.shape[0] == cols and X.shape[1] % 2 == 0
    Y = np.zeros((rows, X.shape[1]), np.uint8)
    if X.shape[1]:
        lib().or16_region_apply(rows, cols, _u16(M), _u8(X), _u8(Y), X.shape[1])
    return Y


def gf16_encode(n: int, k: int, construction: int, systematic: bool, data: np.ndarray) -> np.ndarray:
    d, a = params(n, k)
    data = np.ascontiguousarray(data, dtype=np.uint8)
    out = np.zeros((n * a, data.shape[1]), np.uint8)
    _check(lib().or16_encode(n, k, construction, int(systematic), _u8(data), _u8(out),
                             data.shape[1]), "gf16_encode")
    return out


def gf16_helper_coefficients(n: int, k: int, construction: int, f: int) -> np.ndarray:
    d, a = params(n, k)
    c = np.zeros(a, np.uint16)
    _check(lib().or16_helper_coefficients(n, k, construction, f, _u16(c)), "gf16_helper_coefficients")
    return c


def gf16_newcomer_matrix(n: int, k: int, construction: int, f: int, helpers) -> np.ndarray:
    d, a = params(n, k)
    h = _ints(helpers)
    D = np.zeros((a, d), np.uint16)
    _check(lib().or16_newcomer_matrix(n, k, construction, f, _ip(h), _u16(D)), "gf16_newcomer_matrix")
    return D


def gf16_decode_matrix(n: int, k: int, construction: int, systematic: bool, nodes) -> np.ndarray:
    d, a = params(n, k)
    s = _ints(nodes)
    R = np.zeros((k * a, k * a), np.uint16)
    _check(lib().or16_decode_matrix(n, k, construction, int(systematic), _ip(s), _u16(R)),
           "gf16_decode_matrix")
    return R
