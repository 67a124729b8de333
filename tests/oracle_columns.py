"""Runs the CPU oracle over column slices of its inputs on host threads and
stitches the results: every operation of the method is independent per byte
column (Y[r][t] = sum_c M[r][c] X[c][t], Sec. 2), and the oracle's ctypes
calls release the interpreter lock.  Test infrastructure, like the oracle."""
import concurrent.futures as cf
import os

import numpy as np

THREADS = max(1, min(32, len(os.sched_getaffinity(0))))


def oracle_columns(fn, arrays, slices=None):
    """fn(*[a[:, s] for a in arrays]) for column slices s, stitched along
    the columns.  The first slice runs on this thread (it initializes the
    oracle's field tables), the rest on a thread pool."""
    nbytes = arrays[0].shape[1]
    parts = slices or max(1, min(4 * THREADS, nbytes // 4096))
    edges = [nbytes * i // parts for i in range(parts + 1)]
    cols = [slice(edges[i], edges[i + 1]) for i in range(parts) if edges[i + 1] > edges[i]]

    def run(s):
        return fn(*[np.ascontiguousarray(a[:, s]) for a in arrays])

    first = run(cols[0])
    with cf.ThreadPoolExecutor(THREADS) as ex:
        rest = list(ex.map(run, cols[1:]))
    return np.concatenate([first] + rest, axis=1)
