"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds no arithmetic of the method: only random bytes, random node choices
and workload mixes.  Bytes are uniform on 0..255 (the paper encodes
synthetic data of unstated content, Sec. 4).  Every draw takes an explicit
seed so that a GPU run and the CPU oracle see identical inputs.
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def blocks(count: int, nbytes: int, seed: int) -> np.ndarray:
    """`count` blocks of `nbytes` uniform random bytes, shape (count, nbytes)."""
    return rng(seed).integers(0, 256, (count, nbytes), dtype=np.uint8)


def failed_node(n: int, seed: int) -> int:
    return int(rng(seed ^ 0x5EED).integers(0, n))


def node_subset(n: int, k: int, seed: int) -> list:
    return sorted(int(i) for i in rng(seed ^ 0xC0DE).choice(n, k, replace=False))


def device_blocks(count: int, nbytes: int, seed: int, device="cuda"):
    """Device tensor (count, nbytes) of random bytes drawn on the GPU with a
    seeded torch generator (for workloads too large to draw on the host)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.randint(0, 256, (count, nbytes), dtype=torch.uint8, device=device, generator=g)


def log_uniform_bytes(r: np.random.Generator, lo: int, hi: int, align: int = 16) -> int:
    v = math.exp(r.uniform(math.log(lo), math.log(hi)))
    return int(-(-int(v) // align) * align)


def batch_mix(nstripes: int, seed: int, ks=(4, 8, 16), lo=4096, hi=1 << 20,
              encode_frac: float = 0.5):
    """Batched workload: per stripe (op, k, block_bytes, failed node).
    k uniform on `ks` (n = 2k, d = 2k-2), block size log-uniform on
    [lo, hi] rounded up to 16 bytes, encode or repair with the given split."""
    r = rng(seed)
    out = []
    for _ in range(nstripes):
        k = int(r.choice(ks))
        nb = log_uniform_bytes(r, lo, hi)
        op = "encode" if r.uniform() < encode_frac else "repair"
        f = int(r.integers(0, 2 * k))
        out.append({"op": op, "k": k, "block_bytes": nb, "failed": f})
    return out


def serve_requests(count: int, seed: int, ks=(4, 8, 12, 16), lo=64 << 10, hi=64 << 20,
                   mix=(0.60, 0.25, 0.15), rate_per_s: float = 1000.0, patterns: int = 4):
    """Serving workload: Poisson arrivals (exponential gaps at `rate_per_s`),
    k uniform on `ks`, stripe size log-uniform on [lo, hi], operation mix
    (encode, repair, reconstruct).  Block size = ceil(stripe / (k*alpha))
    rounded up to 16 bytes; the last data block is zero-padded.  A
    reconstruction reads the k nodes of one of `patterns` seeded node sets
    per k (the nodes up while a few others are down serve many stripes)."""
    r = rng(seed)
    t = 0.0
    out = []
    pools = {k: [sorted(int(x) for x in r.choice(2 * k, k, replace=False))
                 for _ in range(patterns)] for k in ks}
    for i in range(count):
        t += r.exponential(1.0 / rate_per_s)
        k = int(r.choice(ks))
        a = k - 1
        stripe = log_uniform_bytes(r, lo, hi, align=1)
        nb = -(-stripe // (k * a))
        nb = -(-nb // 16) * 16
        u = r.uniform()
        op = "encode" if u < mix[0] else ("repair" if u < mix[0] + mix[1] else "decode")
        n = 2 * k
        out.append({"id": i, "t": t, "op": op, "k": k, "stripe_bytes": stripe,
                    "block_bytes": nb, "failed": int(r.integers(0, n)),
                    "nodes": pools[k][int(r.integers(0, patterns))],
                    "seed": int(r.integers(0, 2**31 - 1))})
    return out
