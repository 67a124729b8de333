"""Python binding of libpmrc: product-matrix MSR regenerating codes on GB300.

Argument marshalling only.  Every function of ``include/pmrc.h`` is exposed
under the same name; region pointers are device addresses (ints) or CUDA
tensors (their ``data_ptr()``), pointer arrays are Python sequences, and the
stream is a ``torch.cuda.Stream``, a raw handle or ``None`` (torch's current
stream).  A negative status raises :class:`PMRCError` with the library's
message.  All region work runs in the library's CUDA kernels; there is no
CPU path.  If ``libpmrc.so`` is missing it is built with nvcc on first use,
and the import fails loudly if that is impossible.

:class:`Code` wraps a handle for convenience (the same calls as methods).
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpmrc.so")

PMRC_OK = 0
PMRC_EINVAL = -1
PMRC_ESINGULAR = -2
PMRC_EUNSUPPORTED = -3
PMRC_ENOMEM = -4
PMRC_ECUDA = -5
PMRC_ETIMEOUT = -6
PMRC_EBUSY = -7

PMRC_KERNEL_AUTO = 0
PMRC_KERNEL_GENERIC = 1
PMRC_KERNEL_BITSLICED = 2

PMRC_OP_ENCODE = 0
PMRC_OP_REPAIR = 1
PMRC_OP_DECODE = 2
PMRC_REQ_DEVICE = 0x100   # OR'ed into op: in/out are device blocks, used in place

PMRC_VANILLA = 0
PMRC_SPARSE = 1
PMRC_MBR = 2
PMRC_RS = 3
PMRC_NONSYSTEMATIC = 0
PMRC_SYSTEMATIC = 1

_STATUS = {v: k for k, v in dict(globals()).items() if k.startswith("PMRC_E")}

_lock = threading.Lock()
_lib = None


class PMRCError(RuntimeError):
    def __init__(self, rc: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(rc, rc)} ({msg})")
        self.rc = rc


_i = ctypes.c_int
_sz = ctypes.c_size_t
_vp = ctypes.c_void_p
_pp = ctypes.POINTER(ctypes.c_void_p)
_ip = ctypes.POINTER(ctypes.c_int)
_u8p = ctypes.POINTER(ctypes.c_uint8)

class pmrc_request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("code", ctypes.c_void_p), ("block_bytes", ctypes.c_size_t),
                ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("failed", ctypes.c_int),
                ("helpers", ctypes.POINTER(ctypes.c_int)), ("nodes", ctypes.POINTER(ctypes.c_int))]


_SIGNATURES = {
    "pmrc_create": (_i, [_i, _i, _i, _i, _i, ctypes.POINTER(_vp)]),
    "pmrc_destroy": (None, [_vp]),
    "pmrc_encode": (_i, [_vp, _pp, _pp, _sz, _vp]),
    "pmrc_repair_helper": (_i, [_vp, _i, _i, _pp, _vp, _sz, _vp]),
    "pmrc_repair_helpers": (_i, [_vp, _i, _i, _ip, _pp, _pp, _sz, _vp]),
    "pmrc_repair_newcomer": (_i, [_vp, _i, _ip, _pp, _pp, _sz, _vp]),
    "pmrc_decode": (_i, [_vp, _ip, _pp, _pp, _sz, _vp]),
    "pmrc_specific_workspace_bytes": (_sz, [_vp, _sz]),
    "pmrc_decode_specific": (_i, [_vp, _ip, _pp, _pp, _sz, _vp, _sz, _vp]),
    "pmrc_encode_precode": (_i, [_vp, _pp, _pp, _sz, _vp, _sz, _vp]),
    "pmrc_default_helpers": (_i, [_vp, _i, _ip]),
    "pmrc_last_error": (ctypes.c_char_p, []),
    "pmrc_code_params": (_i, [_vp, _ip]),
    "pmrc_code_blocks": (_i, [_vp, _ip, _ip]),
    "pmrc_set_decode_kernel": (_i, [_vp, _i]),
    "pmrc_wait_kernels": (_i, [_vp, _i]),
    "pmrc_runtime_kernels": (_i, [_vp, _ip, _ip]),
    "pmrc_create_field": (_i, [_i, _i, _i, _i, _i, _i, ctypes.POINTER(_vp)]),
    "pmrc_code_field_bits": (_i, [_vp]),
    "pmrc_code_generator16": (_i, [_vp, ctypes.POINTER(ctypes.c_uint16)]),
    "pmrc_code_generator": (_i, [_vp, _u8p]),
    "pmrc_helper_coefficients": (_i, [_vp, _i, _u8p]),
    "pmrc_newcomer_matrix": (_i, [_vp, _i, _ip, _u8p]),
    "pmrc_decode_matrix": (_i, [_vp, _ip, _u8p]),
    "pmrc_plan_stats": (_i, [_i, _i, _u8p, ctypes.POINTER(ctypes.c_int64)]),
    "pmrc_set_encode_kernel": (_i, [_vp, _i]),
    "pmrc_repair": (_i, [_vp, _i, _ip, _pp, _pp, _sz, _vp]),
    "pmrc_repair_noalloc": (_i, [_vp, _i, _ip, _pp, _pp, _sz, _vp]),
    "pmrc_read_degraded": (_i, [_vp, _i, _ip, _pp, _pp, _sz, _sz, _vp]),
    "pmrc_batch_create": (_i, [ctypes.POINTER(_vp)]),
    "pmrc_batch_destroy": (None, [_vp]),
    "pmrc_batch_add_encode": (_i, [_vp, _vp, _pp, _pp, _sz]),
    "pmrc_batch_add_repair": (_i, [_vp, _vp, _i, _ip, _pp, _pp, _sz]),
    "pmrc_batch_add_decode": (_i, [_vp, _vp, _ip, _pp, _pp, _sz]),
    "pmrc_batch_build": (_i, [_vp, _i, _i]),
    "pmrc_batch_launch": (_i, [_vp, _vp]),
    "pmrc_batch_tune": (_i, [_vp, _vp, _ip]),
    "pmrc_batch_info": (_i, [_vp, ctypes.POINTER(ctypes.c_int64)]),
    "pmrc_server_create": (_i, [_sz, _i, ctypes.POINTER(_vp)]),
    "pmrc_server_destroy": (None, [_vp]),
    "pmrc_server_submit": (_i, [_vp, ctypes.POINTER(pmrc_request), ctypes.POINTER(ctypes.c_uint64)]),
    "pmrc_server_poll": (_i, [_vp, ctypes.c_uint64, _ip, ctypes.POINTER(ctypes.c_double)]),
    "pmrc_server_wait": (_i, [_vp, ctypes.c_uint64, _i, _ip, ctypes.POINTER(ctypes.c_double)]),
    "pmrc_server_cancel": (_i, [_vp, ctypes.c_uint64]),
    "pmrc_server_stats": (_i, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "pmrc_server_reset_stats": (_i, [_vp]),
}


def lib() -> ctypes.CDLL:
    """The loaded libpmrc.so (built in-tree with nvcc if missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def _check(rc: int, where: str):
    if rc < 0:
        raise PMRCError(rc, where, lib().pmrc_last_error().decode())
    return rc


def _addr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _ptrs(seq):
    if isinstance(seq, ctypes.Array):   # built once by ptr_array()
        return seq
    arr = (ctypes.c_void_p * len(seq))()
    for i, x in enumerate(seq):
        arr[i] = _addr(x) or None
    return arr


def _ints(seq):
    if isinstance(seq, ctypes.Array):   # built once by int_array()
        return seq
    arr = (ctypes.c_int * len(seq))()
    for i, x in enumerate(seq):
        arr[i] = int(x)
    return arr


def ptr_array(seq):
    """A pointer array (tensors, addresses or None) converted once, for
    callers that repeat a call on the same blocks: every call below accepts
    it in place of a sequence and skips the per-call conversion."""
    return _ptrs(list(seq))


def int_array(seq):
    """A node-id list converted once (see ptr_array)."""
    return _ints(list(seq))


def _stream(s) -> int:
    if s is None:
        try:
            import torch
            if torch.cuda.is_initialized():
                return int(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return 0
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


# ---------------------------------------------------------------- C ABI
def pmrc_create(n: int, k: int, d: int, construction: int, form: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().pmrc_create(n, k, d, construction, form, ctypes.byref(h)), "pmrc_create")
    return int(h.value)


def pmrc_destroy(code: int) -> None:
    if code:
        lib().pmrc_destroy(code)


def pmrc_encode(code, data, out, block_bytes, stream=None) -> None:
    _check(lib().pmrc_encode(code, _ptrs(data), _ptrs(out), block_bytes, _stream(stream)),
           "pmrc_encode")


def pmrc_repair_helper(code, failed, helper, helper_blocks, out, block_bytes, stream=None):
    _check(lib().pmrc_repair_helper(code, failed, helper, _ptrs(helper_blocks), _addr(out),
                                    block_bytes, _stream(stream)), "pmrc_repair_helper")


def pmrc_repair_helpers(code, failed, helpers, helper_blocks, out, block_bytes, stream=None):
    _check(lib().pmrc_repair_helpers(code, failed, len(out), _ints(helpers),
                                     _ptrs(helper_blocks), _ptrs(out), block_bytes,
                                     _stream(stream)), "pmrc_repair_helpers")


def pmrc_repair_newcomer(code, failed, helpers, received, out, block_bytes, stream=None):
    _check(lib().pmrc_repair_newcomer(code, failed, _ints(helpers), _ptrs(received), _ptrs(out),
                                      block_bytes, _stream(stream)), "pmrc_repair_newcomer")


def pmrc_repair(code, failed, helpers, helper_blocks, out, block_bytes, stream=None):
    _check(lib().pmrc_repair(code, failed, _ints(helpers), _ptrs(helper_blocks), _ptrs(out),
                             block_bytes, _stream(stream)), "pmrc_repair")


def pmrc_read_degraded(code, node, helpers, helper_blocks, out, offset, length, stream=None):
    _check(lib().pmrc_read_degraded(code, node, _ints(helpers), _ptrs(helper_blocks), _ptrs(out),
                                    offset, length, _stream(stream)), "pmrc_read_degraded")


def pmrc_repair_noalloc(code, failed, helpers, helper_blocks, out, block_bytes, stream=None):
    _check(lib().pmrc_repair_noalloc(code, failed, _ints(helpers), _ptrs(helper_blocks),
                                     _ptrs(out), block_bytes, _stream(stream)),
           "pmrc_repair_noalloc")


def pmrc_decode(code, nodes, node_blocks, data_out, block_bytes, stream=None):
    _check(lib().pmrc_decode(code, _ints(nodes), _ptrs(node_blocks), _ptrs(data_out),
                             block_bytes, _stream(stream)), "pmrc_decode")


def pmrc_specific_workspace_bytes(code, block_bytes) -> int:
    return int(lib().pmrc_specific_workspace_bytes(code, block_bytes))


def pmrc_decode_specific(code, nodes, node_blocks, data_out, block_bytes, workspace,
                         workspace_bytes, stream=None):
    _check(lib().pmrc_decode_specific(code, _ints(nodes), _ptrs(node_blocks), _ptrs(data_out),
                                      block_bytes, _addr(workspace), workspace_bytes,
                                      _stream(stream)), "pmrc_decode_specific")


def pmrc_encode_precode(code, data, parity, block_bytes, workspace, workspace_bytes,
                        stream=None):
    _check(lib().pmrc_encode_precode(code, _ptrs(data), _ptrs(parity), block_bytes,
                                     _addr(workspace), workspace_bytes, _stream(stream)),
           "pmrc_encode_precode")


def pmrc_set_decode_kernel(code, which: int) -> None:
    _check(lib().pmrc_set_decode_kernel(code, which), "pmrc_set_decode_kernel")


def pmrc_wait_kernels(code, timeout_ms: int = -1) -> None:
    _check(lib().pmrc_wait_kernels(code, timeout_ms), "pmrc_wait_kernels")


def pmrc_runtime_kernels(code) -> tuple:
    ready, pending = ctypes.c_int(), ctypes.c_int()
    _check(lib().pmrc_runtime_kernels(code, ctypes.byref(ready), ctypes.byref(pending)),
           "pmrc_runtime_kernels")
    return ready.value, pending.value


def wait_kernels(timeout_ms: int = -1) -> None:
    """pmrc_wait_kernels on every live Code of this process."""
    for c in list(_live_codes):
        if c.handle:
            pmrc_wait_kernels(c.handle, timeout_ms)


def pmrc_set_encode_kernel(code, which: int) -> None:
    _check(lib().pmrc_set_encode_kernel(code, which), "pmrc_set_encode_kernel")


def pmrc_default_helpers(code, failed) -> list:
    p = pmrc_code_params(code)
    out = (ctypes.c_int * p["d"])()
    _check(lib().pmrc_default_helpers(code, failed, out), "pmrc_default_helpers")
    return list(out)


def pmrc_last_error() -> str:
    return lib().pmrc_last_error().decode()


def pmrc_code_params(code) -> dict:
    out = (ctypes.c_int * 6)()
    _check(lib().pmrc_code_params(code, out), "pmrc_code_params")
    return dict(zip(("n", "k", "d", "alpha", "construction", "form"), list(out)))


def pmrc_create_field(n: int, k: int, d: int, construction: int, form: int,
                      field_bits: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().pmrc_create_field(n, k, d, construction, form, field_bits, ctypes.byref(h)),
           "pmrc_create_field")
    return int(h.value)


def pmrc_code_field_bits(code) -> int:
    return int(lib().pmrc_code_field_bits(code))


def pmrc_code_generator16(code):
    import numpy as np
    K, N = pmrc_code_blocks(code)
    buf = (ctypes.c_uint16 * (K * N))()
    _check(lib().pmrc_code_generator16(code, buf), "pmrc_code_generator16")
    return np.frombuffer(bytes(buf), dtype=np.uint16).reshape(N, K).copy()


def pmrc_code_blocks(code):
    """(K data blocks, n*alpha coded blocks)."""
    K, N = ctypes.c_int(), ctypes.c_int()
    _check(lib().pmrc_code_blocks(code, ctypes.byref(K), ctypes.byref(N)), "pmrc_code_blocks")
    return K.value, N.value


def _u8buf(size):
    return (ctypes.c_uint8 * size)()


def _mat(buf, rows, cols):
    import numpy as np
    return np.frombuffer(bytes(buf), dtype=np.uint8).reshape(rows, cols).copy()


def pmrc_code_generator(code):
    K, N = pmrc_code_blocks(code)
    buf = _u8buf(N * K)
    _check(lib().pmrc_code_generator(code, buf), "pmrc_code_generator")
    return _mat(buf, N, K)


def pmrc_helper_coefficients(code, failed):
    p = pmrc_code_params(code)
    buf = _u8buf(p["alpha"])
    _check(lib().pmrc_helper_coefficients(code, failed, buf), "pmrc_helper_coefficients")
    return _mat(buf, 1, p["alpha"])[0]


def pmrc_newcomer_matrix(code, failed, helpers):
    p = pmrc_code_params(code)
    buf = _u8buf(p["alpha"] * p["d"])
    _check(lib().pmrc_newcomer_matrix(code, failed, _ints(helpers), buf), "pmrc_newcomer_matrix")
    return _mat(buf, p["alpha"], p["d"])


def pmrc_decode_matrix(code, nodes):
    p = pmrc_code_params(code)
    K, _ = pmrc_code_blocks(code)
    KA = p["k"] * p["alpha"]
    buf = _u8buf(K * KA)
    _check(lib().pmrc_decode_matrix(code, _ints(nodes), buf), "pmrc_decode_matrix")
    return _mat(buf, K, KA)


def pmrc_plan_stats(m) -> dict:
    import numpy as np
    m = np.ascontiguousarray(m, dtype=np.uint8)
    out = (ctypes.c_int64 * 5)()
    _check(lib().pmrc_plan_stats(m.shape[0], m.shape[1],
                                 m.ctypes.data_as(_u8p), out), "pmrc_plan_stats")
    return dict(zip(("blocks", "R", "entries", "input_splits", "nnz"), list(out)))


# ---------------------------------------------------------------- batch
def pmrc_batch_create() -> int:
    h = ctypes.c_void_p()
    _check(lib().pmrc_batch_create(ctypes.byref(h)), "pmrc_batch_create")
    return int(h.value)


def pmrc_batch_destroy(batch) -> None:
    if batch:
        lib().pmrc_batch_destroy(batch)


def pmrc_batch_add_encode(batch, code, data, out, block_bytes) -> int:
    return _check(lib().pmrc_batch_add_encode(batch, code, _ptrs(data), _ptrs(out), block_bytes),
                  "pmrc_batch_add_encode")


def pmrc_batch_add_repair(batch, code, failed, helpers, helper_blocks, out, block_bytes) -> int:
    return _check(lib().pmrc_batch_add_repair(batch, code, failed, _ints(helpers),
                                              _ptrs(helper_blocks), _ptrs(out), block_bytes),
                  "pmrc_batch_add_repair")


def pmrc_batch_add_decode(batch, code, nodes, node_blocks, data_out, block_bytes) -> int:
    return _check(lib().pmrc_batch_add_decode(batch, code, _ints(nodes), _ptrs(node_blocks),
                                              _ptrs(data_out), block_bytes),
                  "pmrc_batch_add_decode")


def pmrc_batch_build(batch, work_bytes=0, ctas_per_sm=0) -> None:
    _check(lib().pmrc_batch_build(batch, work_bytes, ctas_per_sm), "pmrc_batch_build")


def pmrc_batch_launch(batch, stream=None) -> None:
    _check(lib().pmrc_batch_launch(batch, _stream(stream)), "pmrc_batch_launch")


def pmrc_batch_tune(batch, stream=None) -> tuple:
    out = (ctypes.c_int * 2)()
    _check(lib().pmrc_batch_tune(batch, _stream(stream), out), "pmrc_batch_tune")
    return out[0], out[1]


def pmrc_batch_info(batch) -> dict:
    out = (ctypes.c_int64 * 8)()
    _check(lib().pmrc_batch_info(batch, out), "pmrc_batch_info")
    return dict(zip(("stripes", "items", "ctas", "work_bytes", "ctas_per_sm", "user_bytes",
                     "bitsliced_launches", "smem_bytes"), list(out)))


class Batch:
    """Owns a pmrc_batch handle; keeps the codes it references alive."""

    def __init__(self):
        self.handle = pmrc_batch_create()
        self._codes = []

    def close(self):
        if self.handle:
            pmrc_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_encode(self, code, data, out, block_bytes):
        self._codes.append(code)
        return pmrc_batch_add_encode(self.handle, code.handle, data, out, block_bytes)

    def add_repair(self, code, failed, helpers, helper_blocks, out, block_bytes):
        self._codes.append(code)
        return pmrc_batch_add_repair(self.handle, code.handle, failed, helpers, helper_blocks,
                                     out, block_bytes)

    def add_decode(self, code, nodes, node_blocks, data_out, block_bytes):
        self._codes.append(code)
        return pmrc_batch_add_decode(self.handle, code.handle, nodes, node_blocks, data_out,
                                     block_bytes)

    def build(self, work_bytes=0, ctas_per_sm=0):
        pmrc_batch_build(self.handle, work_bytes, ctas_per_sm)

    def launch(self, stream=None):
        pmrc_batch_launch(self.handle, stream)

    def tune(self, stream=None):
        return pmrc_batch_tune(self.handle, stream)

    def info(self):
        return pmrc_batch_info(self.handle)


# ---------------------------------------------------------------- serving
def pmrc_server_create(budget_bytes: int, max_slots: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().pmrc_server_create(budget_bytes, max_slots, ctypes.byref(h)),
           "pmrc_server_create")
    return int(h.value)


def pmrc_server_destroy(server) -> None:
    if server:
        lib().pmrc_server_destroy(server)


def pmrc_server_submit(server, op, code, block_bytes, in_ptr, out_ptr, failed=-1,
                       helpers=None, nodes=None) -> int:
    hs = _ints(helpers) if helpers is not None else None
    ns = _ints(nodes) if nodes is not None else None
    req = pmrc_request(op, code, block_bytes, _addr(in_ptr), _addr(out_ptr), failed,
                       ctypes.cast(hs, ctypes.POINTER(ctypes.c_int)) if hs is not None else None,
                       ctypes.cast(ns, ctypes.POINTER(ctypes.c_int)) if ns is not None else None)
    rid = ctypes.c_uint64()
    _check(lib().pmrc_server_submit(server, ctypes.byref(req), ctypes.byref(rid)),
           "pmrc_server_submit")
    return rid.value


def pmrc_server_poll(server, rid):
    st, lat = ctypes.c_int(), ctypes.c_double()
    done = _check(lib().pmrc_server_poll(server, rid, ctypes.byref(st), ctypes.byref(lat)),
                  "pmrc_server_poll")
    return (st.value, lat.value) if done else None


def pmrc_server_wait(server, rid, timeout_ms=-1):
    st, lat = ctypes.c_int(), ctypes.c_double()
    _check(lib().pmrc_server_wait(server, rid, timeout_ms, ctypes.byref(st), ctypes.byref(lat)),
           "pmrc_server_wait")
    return st.value, lat.value


def pmrc_server_cancel(server, rid) -> None:
    _check(lib().pmrc_server_cancel(server, rid), "pmrc_server_cancel")


def pmrc_server_stats(server) -> dict:
    out = (ctypes.c_double * 10)()
    _check(lib().pmrc_server_stats(server, out), "pmrc_server_stats")
    keys = ("completed", "failed", "p50_ms", "p99_ms", "max_ms", "user_bytes", "user_GBps",
            "peak_bytes", "iterations", "budget_bytes")
    return dict(zip(keys, list(out)))


def pmrc_server_reset_stats(server) -> None:
    _check(lib().pmrc_server_reset_stats(server), "pmrc_server_reset_stats")


class Server:
    """Owns a pmrc_server; submit() takes host buffers (tensors or addresses)."""

    def __init__(self, budget_bytes: int, max_slots: int = 64):
        self.handle = pmrc_server_create(budget_bytes, max_slots)

    def close(self):
        if self.handle:
            pmrc_server_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, op, code, block_bytes, in_buf, out_buf, failed=-1, helpers=None,
               nodes=None):
        return pmrc_server_submit(self.handle, op, code.handle, block_bytes, in_buf, out_buf,
                                  failed, helpers, nodes)

    def poll(self, rid):
        return pmrc_server_poll(self.handle, rid)

    def wait(self, rid, timeout_ms=-1):
        return pmrc_server_wait(self.handle, rid, timeout_ms)

    def cancel(self, rid):
        pmrc_server_cancel(self.handle, rid)

    def stats(self):
        return pmrc_server_stats(self.handle)

    def reset_stats(self):
        pmrc_server_reset_stats(self.handle)


# ---------------------------------------------------------------- handle
_live_codes = weakref.WeakSet()


class Code:
    """Owns a pmrc_code handle; methods are the C calls on it."""

    def __init__(self, n: int, k: int, construction: int = PMRC_SPARSE,
                 form: int = PMRC_SYSTEMATIC, d: int = None, field_bits: int = 8):
        """PM-MSR (PMRC_VANILLA / PMRC_SPARSE): d = 2k-2, over GF(2^8) or
        (field_bits=16) GF(2^16).  PM-MBR (PMRC_MBR): any k <= d <= n-1
        (default 2k-2).  Reed-Solomon (PMRC_RS): d = k."""
        if d is None:
            d = k if construction == PMRC_RS else 2 * k - 2
        self.handle = pmrc_create_field(n, k, d, construction, form, field_bits)
        self.field_bits = field_bits
        p = pmrc_code_params(self.handle)
        self.n, self.k, self.d, self.alpha = p["n"], p["k"], p["d"], p["alpha"]
        self.construction, self.form = construction, form
        self.data_blocks, self.coded_blocks = pmrc_code_blocks(self.handle)
        _live_codes.add(self)

    def close(self):
        if self.handle:
            pmrc_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_outputs(self) -> int:
        a = self.alpha
        return (self.n - self.k) * a if self.form == PMRC_SYSTEMATIC else self.n * a

    def encode(self, data, out, block_bytes, stream=None):
        pmrc_encode(self.handle, data, out, block_bytes, stream)

    def repair_helper(self, failed, helper, blocks, out, block_bytes, stream=None):
        pmrc_repair_helper(self.handle, failed, helper, blocks, out, block_bytes, stream)

    def repair_helpers(self, failed, helpers, blocks, out, block_bytes, stream=None):
        pmrc_repair_helpers(self.handle, failed, helpers, blocks, out, block_bytes, stream)

    def repair_newcomer(self, failed, helpers, received, out, block_bytes, stream=None):
        pmrc_repair_newcomer(self.handle, failed, helpers, received, out, block_bytes, stream)

    def repair(self, failed, helpers, helper_blocks, out, block_bytes, stream=None):
        pmrc_repair(self.handle, failed, helpers, helper_blocks, out, block_bytes, stream)

    def read_degraded(self, node, helpers, helper_blocks, out, offset, length, stream=None):
        """Bytes [offset, offset + length) of a lost systematic node's blocks,
        rebuilt from its helpers' whole blocks."""
        pmrc_read_degraded(self.handle, node, helpers, helper_blocks, out, offset, length, stream)

    def decode(self, nodes, node_blocks, data_out, block_bytes, stream=None):
        pmrc_decode(self.handle, nodes, node_blocks, data_out, block_bytes, stream)

    def specific_workspace_bytes(self, block_bytes) -> int:
        return pmrc_specific_workspace_bytes(self.handle, block_bytes)

    def decode_specific(self, nodes, node_blocks, data_out, block_bytes, workspace,
                        workspace_bytes=None, stream=None):
        """Data-collector reconstruction; `workspace` is a device tensor or
        address of at least specific_workspace_bytes(block_bytes) bytes."""
        if workspace_bytes is None:
            workspace_bytes = int(workspace.numel() * workspace.element_size())
        pmrc_decode_specific(self.handle, nodes, node_blocks, data_out, block_bytes, workspace,
                             workspace_bytes, stream)

    def encode_precode(self, data, parity, block_bytes, workspace, workspace_bytes=None,
                       stream=None):
        """Systematic encode by decoding then encoding (same parity as encode)."""
        if workspace_bytes is None:
            workspace_bytes = int(workspace.numel() * workspace.element_size())
        pmrc_encode_precode(self.handle, data, parity, block_bytes, workspace, workspace_bytes,
                            stream)

    def wait_kernels(self, timeout_ms: int = -1):
        pmrc_wait_kernels(self.handle, timeout_ms)

    def runtime_kernels(self) -> tuple:
        """(compiled, still compiling) run-time kernels of this handle."""
        return pmrc_runtime_kernels(self.handle)

    def set_decode_kernel(self, which: int):
        pmrc_set_decode_kernel(self.handle, which)

    def set_encode_kernel(self, which: int):
        pmrc_set_encode_kernel(self.handle, which)

    def default_helpers(self, failed):
        return pmrc_default_helpers(self.handle, failed)

    def generator(self):
        return pmrc_code_generator(self.handle)

    def helper_coefficients(self, failed):
        return pmrc_helper_coefficients(self.handle, failed)

    def newcomer_matrix(self, failed, helpers):
        return pmrc_newcomer_matrix(self.handle, failed, helpers)

    def decode_matrix(self, nodes):
        return pmrc_decode_matrix(self.handle, nodes)
