#!/usr/bin/env python
"""Benchmark of the PM-MSR hot path on GB300.

Workload: the n=16, k=8, d=14, alpha=7 product-matrix MSR code over GF(2^8)
(modulus 0x11D), one stripe of 56 data blocks of 1 MiB (56 MiB) of seeded
uniform random bytes.  One step runs every operation of the hot path once:

  gen_encode  vanilla (Vandermonde) generator form, 56 -> 112 blocks
  sys_encode  sparse systematic form, 56 data -> 56 parity blocks
  repair      a seeded failed node: d=14 helper projections (one batched
              launch) and the newcomer's apply, 14 -> 7 blocks
  decode      reconstruction from a seeded 8-node subset (systematic, lazy:
              data blocks of surviving data nodes stay in place)

Throughput is user data / time (the paper's Sec. 4 definition: k*alpha
blocks for encode and decode, alpha blocks for repair), GB = 1e9 B.  L2 is
flushed before every operation, outside the timed events (a 512 MiB write,
then a 512 MiB read sweep so the lines left in L2 are clean).
Each operation is timed with CUDA events on the launch stream.

--impl reference times the CPU oracle (plain C, one core) on a bounded
column sample of the same stripe instead.
"""
from __future__ import annotations

import argparse
import gc
import json

import numpy as np
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PM-MSR k=8 encode/repair GB/s & %HBM roofline; batched vs plain; p99 ms"
N_, K_, A_ = 16, 8, 7
D_ = 2 * K_ - 2
WORKLOAD = ("PM-MSR n=16 k=8 d=14 alpha=7 GF(2^8)/0x11D, 56 data blocks x 1 MiB "
            "(56 MiB stripe): vanilla generator encode + sparse systematic encode + "
            "repair of a seeded node (14 helper projections + newcomer) + "
            "reconstruction from a seeded 8-node subset")
FLUSH_BYTES = 512 << 20
SMS = 152   # GB300 streaming multiprocessors


# ------------------------------------------------------------ ALU models
ALU_MODEL_BITSLICED = ("bitsliced kernel, per 32-byte lane and block: 44 lane-ops per input "
                       "(24 transpose + 20 subset-table XORs), 24 per output row (transpose "
                       "back), 8 per non-zero coefficient (one 3-input XOR per output plane)")
ALU_MODEL_FACTORED = ("factored reconstruction, per 32-byte lane: launch 1 (z) 44 lane-ops per "
                      "input per block and 8 per non-zero coefficient, outputs stored as bit "
                      "planes; launch 2 (B^-1 z, taken as dense) 20 per plane-layout input per "
                      "block, 24 per output row, 8 per coefficient")
ALU_MODEL_PROJECTION = ("bitsliced projection kernel, per 32-byte lane: 24 lane-ops per helper "
                        "block read (transpose), per output plane of each constant product one "
                        "3-input XOR per two terms, 24 per helper (transpose back)")


def gf_mul_11d(x, y):
    """x * y in GF(2^8) modulo 0x11D (for the instruction model only)."""
    r = 0
    while y:
        if y & 1:
            r ^= x
        y >>= 1
        x = (x << 1) ^ (0x11D if x & 0x80 else 0)
    return r


def alu_ops_projection(phi, helpers):
    """ALU lane-ops per 32-byte column of the bitsliced helper-projection
    kernel: each block a helper's phi reads is transposed into planes once
    and multiplied by its constant as XORs of planes (output plane i of c*x
    takes the input planes jj with bit i of c*2^jj set); the first block's
    product starts the accumulator, later ones fold into it, two terms per
    3-input XOR; the projection is transposed back."""
    per_helper = 24
    first = True
    for c in phi:
        if not c:
            continue
        per_helper += 24
        for i in range(8):
            t = sum((gf_mul_11d(int(c), 1 << jj) >> i) & 1 for jj in range(8))
            per_helper += (t // 2) if first else -(-t // 2)
        first = False
    return per_helper * helpers


def factored_blocks(Z, own, max_inputs=64):
    """The library's first-launch blocks of a factored reconstruction: rows
    of Z grouped by their non-zero columns other than their own parity
    block, groups packed whole into blocks of at most 8 rows within
    max_inputs inputs (a group of more than 8 rows cut into blocks of its
    own); returns (rows, inputs) per block."""
    groups, order = {}, []
    for r in range(Z.shape[0]):
        key = tuple(int(q) for q in np.flatnonzero(Z[r]) if q != own[r])
        if key not in groups:
            order.append(key)
        groups.setdefault(key, []).append(r)

    def union(rs):
        return int((Z[rs] != 0).any(axis=0).sum())

    sets, cur = [], []
    for key in order:
        rs = groups[key]
        if len(rs) > 8:
            nb = -(-len(rs) // 8)
            sets += [rs[len(rs) * b // nb:len(rs) * (b + 1) // nb] for b in range(nb)]
            continue
        grown = cur + rs
        if cur and (len(grown) > 8 or union(grown) > max_inputs):
            sets.append(cur)
            cur = list(rs)
        else:
            cur = grown
    if cur:
        sets.append(cur)
    return [(len(rs), union(rs)) for rs in sets]


def alu_ops_factored(Z, own, m_out):
    """ALU lane-ops per 32-byte column of the factored reconstruction's two
    launches: z = Z y (blocks of factored_blocks, 44 per input, plane-layout
    outputs) and the m_out wanted rows of B^-1 z (taken as dense: blocks of
    at most 8 consecutive rows over all z, 20 per plane-layout input, 24 per
    output row), 8 per non-zero coefficient in both."""
    m = Z.shape[0]
    c1 = sum(44 * c for _, c in factored_blocks(Z, own)) + 8 * int((Z != 0).sum())
    nb = -(-m_out // 8)
    c2 = nb * 20 * m + 24 * m_out + 8 * m_out * m
    return c1 + c2


def alu_ops_bitsliced(M, kind):
    """ALU lane-ops per 32-byte column of the bitsliced kernels for the
    matrix M, with their block rule: rows of identical support in blocks of
    at most 8 ("support", the built-in encode kernels) or consecutive rows
    in balanced blocks of at most 8 over the union of their inputs
    ("chunked", the run-time reconstruction kernels)."""
    rows = M.shape[0]
    blocks = []
    if kind == "support":
        groups = {}
        for r in range(rows):
            groups.setdefault(tuple(np.flatnonzero(M[r]).tolist()), []).append(r)
        for sup, rs in groups.items():
            nb = -(-len(rs) // 8)
            for b in range(nb):
                blocks.append((len(rs) * (b + 1) // nb - len(rs) * b // nb, len(sup)))
    else:
        nb = -(-rows // 8)
        for b in range(nb):
            rs = list(range(rows * b // nb, rows * (b + 1) // nb))
            blocks.append((len(rs), int((M[rs] != 0).any(axis=0).sum())))
    return sum(44 * c + 24 * r for r, c in blocks) + 8 * int((M != 0).sum())


# ------------------------------------------------------------ multi-rank
# Stripes are independent, so N ranks run N replicas of the step on their own
# seeded stripes (weak scaling) with no collective on the data path; the only
# communication is the timing reduction below.
def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s stripe (distinct stripes per rank)."""
    return seed + 1000 * rank


def ranks_max(dist, x: float, device) -> float:
    """Largest x over all ranks (x itself when running alone)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbps(user_bytes_per_rank: int, world: int, max_ms: float) -> float:
    """Aggregate user-data throughput of all ranks over the slowest rank's time."""
    return user_bytes_per_rank * world / (max_ms * 1e-3) / 1e9


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--block-bytes", type=int, default=1 << 20)
    p.add_argument("--seed", type=int, default=2)
    p.add_argument("--ref-seconds", type=float, default=6.0,
                   help="--impl reference: CPU seconds per step, at most")
    p.add_argument("--cpu-seconds", type=float, default=12.0,
                   help="target CPU time of the oracle baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--batch-stripes", type=int, default=4096)
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-mbr", action="store_true")
    p.add_argument("--no-sweep", action="store_true",
                   help="skip the block-size sweep (64 KiB - 4 MiB) and the k sweep (4 - 32) "
                        "of encode, repair, decode")
    p.add_argument("--no-extra", action="store_true",
                   help="skip the rows outside the step (fused repair, specific algorithms, "
                        "PM-MBR, Reed-Solomon), e.g. for a launch list of the step alone")
    p.add_argument("--serve-requests", type=int, default=10000,
                   help="requests per offered-load level")
    p.add_argument("--cfg1-reps", type=int, default=2000,
                   help="timed calls per operation of the n=6 k=3 4 KiB latency section")
    p.add_argument("--no-cfg1", action="store_true")
    return p.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ peaks
class L2Flush:
    """Evicts the timed operation's data from L2 before each timed call: a
    512 MiB write (larger than the 126 MB L2), then a read sweep of another
    512 MiB buffer (one 4-byte load per 128-byte line, gathered into a small
    buffer) so that the lines left in L2 are clean and the next call does
    not pay for writing the flush's dirty lines back.  Both are single
    kernels queued ahead of the timed call (no idle gap before it)."""

    def __init__(self, torch, dev):
        self.w = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
        self.r = torch.ones(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
        self.g = torch.empty(FLUSH_BYTES // 128, dtype=torch.int32, device=dev)

    def __call__(self, v=7):
        self.w.fill_(v)
        self.g.copy_(self.r.view(-1, 32)[:, 0])

    def fill_(self, v):  # the call sites' former flush.fill_(v)
        self(v)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ ours
class Workload:
    def __init__(self, torch, P, inputs, B, seed, device):
        self.t = torch
        self.P = P
        self.seed = seed
        self.B = B
        a, K = A_, K_ * A_
        self.sysc = P.Code(N_, K_, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
        self.genc = P.Code(N_, K_, P.PMRC_VANILLA, P.PMRC_NONSYSTEMATIC)
        self.X = inputs.device_blocks(K, B, seed, device=device)
        self.gen_out = torch.empty((N_ * a, B), dtype=torch.uint8, device=device)
        # the stored codeword (data + parity) that repair and decode read
        self.Y = torch.empty((N_ * a, B), dtype=torch.uint8, device=device)
        self.Y[:K].copy_(self.X)
        self.f = inputs.failed_node(N_, seed)
        self.H = self.sysc.default_helpers(self.f)
        self.recv = torch.empty((D_, B), dtype=torch.uint8, device=device)
        self.node = torch.empty((a, B), dtype=torch.uint8, device=device)
        self.S = inputs.node_subset(N_, K_, seed)
        self.data_out = torch.empty((K, B), dtype=torch.uint8, device=device)
        self.x_ptrs = [self.X[i] for i in range(K)]
        self.gen_ptrs = [self.gen_out[i] for i in range(N_ * a)]
        self.par_ptrs = [self.Y[K + i] for i in range(K)]
        self.helper_in = [self.Y[a * h + j] for h in self.H for j in range(a)]
        self.recv_ptrs = [self.recv[i] for i in range(D_)]
        self.node_ptrs = [self.node[j] for j in range(a)]
        self.dec_in = [self.Y[a * i + j] for i in self.S for j in range(a)]
        self.dec_out = [self.data_out[r] for r in range(K)]
        for pos, i in enumerate(self.S):   # lazy decode: present data stays in place
            if i < K_:
                for j in range(a):
                    self.dec_out[a * i + j] = self.dec_in[a * pos + j]
        self.sysc.encode(self.x_ptrs, self.par_ptrs, B)  # codeword for repair/decode
        self._bytes()
        # pointer and node arrays converted once, so that no per-call host
        # conversion runs between a timing event and its kernel
        self.stream = int(torch.cuda.current_stream(device).cuda_stream)
        self.c_args = {name: P.ptr_array(getattr(self, name)) for name in
                       ("x_ptrs", "gen_ptrs", "par_ptrs", "helper_in", "recv_ptrs", "node_ptrs",
                        "dec_in", "dec_out")}
        self.c_H = P.int_array(self.H)
        self.c_S = P.int_array(self.S)

    def _bytes(self):
        """Algorithmic HBM bytes and user bytes per operation."""
        B, a, K = self.B, A_, K_ * A_
        coef = self.sysc.helper_coefficients(self.f)
        reads_per_helper = int((coef != 0).sum())
        R = self.sysc.decode_matrix(self.S)
        present = {a * i + j for i in self.S if i < K_ for j in range(a)}
        missing = [r for r in range(K) if r not in present]
        dec_inputs = int((R[missing] != 0).any(axis=0).sum()) if missing else 0
        self.alg = {
            "gen_encode": (K + N_ * a) * B,
            "sys_encode": (K + K) * B,
            "repair_helpers": (D_ * reads_per_helper + D_) * B,
            "repair_newcomer": (D_ + a) * B,
            "repair_fused": (D_ * reads_per_helper + a) * B,
            "decode": (dec_inputs + len(missing)) * B,
        }
        self.user = {"gen_encode": K * B, "sys_encode": K * B, "repair": a * B, "decode": K * B}
        self.decode_missing = len(missing)
        self.helper_reads = reads_per_helper
        # the kernel each operation runs, and its ALU lane-ops per launch
        # (alu_model); the reconstruction and the helper projections (blocks
        # of at least 256 KiB) and the newcomer (at least 1 MiB) run
        # run-time bitsliced kernels
        P = self.P
        G = self.genc.generator()
        Gs = self.sysc.generator()[K:]
        Dn = self.sysc.newcomer_matrix(self.f, self.H)
        Rm = R[missing] if missing else np.zeros((0, K), np.uint8)
        # the factored form of the reconstruction (z = received parity
        # blocks plus their present-data terms, then B^-1 z), which the
        # library takes when its instruction model, second launch included,
        # beats the one-launch schedule's (the same rule and constants)
        Gfull = self.sysc.generator()
        slots = [(a * i + j, a * pos + j) for pos, i in enumerate(self.S) if i >= K_ for j in range(a)]
        Z = np.zeros((len(slots), K), np.uint8)
        own = []
        for q, (row, slot) in enumerate(slots):
            Z[q, slot] = 1
            own.append(slot)
            for pos, i in enumerate(self.S):
                if i < K_:
                    for j in range(a):
                        Z[q, a * pos + j] = Gfull[row, a * i + j]
        one_launch = alu_ops_bitsliced(Rm, "chunked")
        factored = alu_ops_factored(Z, own, len(missing)) if missing else None
        self.decode_factored = factored is not None and \
            factored + 1227 * (1 << 20) / B < one_launch
        self.kernel = {"gen_encode": "bitsliced encode bs_n16_k8_c0_f0",
                       "sys_encode": "bitsliced encode bs_n16_k8_c1_f1",
                       "repair_helpers": "bitsliced helper projections bs_rt_project (compiled at run time)",
                       "repair_newcomer": "bitsliced newcomer bs_rt_newcomer (compiled at run time)",
                       "decode": ("factored bitsliced reconstruction bs_rt_dstage1 + bs_rt_dstage2 "
                                  "(compiled at run time, two launches)") if self.decode_factored else
                                 "bitsliced reconstruction bs_rt_decode (compiled at run time)"}
        self.alu_ops, self.alu_model = {}, {}
        for n, M, kind in (("gen_encode", G, "support"), ("sys_encode", Gs, "support"),
                           ("decode", Rm, "chunked"), ("repair_newcomer", Dn, "chunked")):
            self.alu_ops[n] = alu_ops_bitsliced(M, kind) * (B // 32)
            self.alu_model[n] = ALU_MODEL_BITSLICED
        if self.decode_factored:
            self.alu_ops["decode"] = factored * (B // 32)
            self.alu_model["decode"] = ALU_MODEL_FACTORED
        self.alu_ops["repair_helpers"] = alu_ops_projection(coef, D_) * (B // 32)
        self.alu_model["repair_helpers"] = ALU_MODEL_PROJECTION

    def ops(self, stream=None):
        s, B, a = self, self.B, self.c_args
        st = self.stream if stream is None else stream
        return [
            ("gen_encode", lambda: s.genc.encode(a["x_ptrs"], a["gen_ptrs"], B, st)),
            ("sys_encode", lambda: s.sysc.encode(a["x_ptrs"], a["par_ptrs"], B, st)),
            ("repair_helpers", lambda: s.sysc.repair_helpers(s.f, s.c_H, a["helper_in"],
                                                             a["recv_ptrs"], B, st)),
            ("repair_newcomer", lambda: s.sysc.repair_newcomer(s.f, s.c_H, a["recv_ptrs"],
                                                               a["node_ptrs"], B, st)),
            ("decode", lambda: s.sysc.decode(s.c_S, a["dec_in"], a["dec_out"], B, st)),
        ]


def run_ours(args, rank, world, local_rank):
    # an empty on-disk kernel cache of this run's own: the initialization
    # section measures cold compilations whatever earlier processes cached
    import atexit
    import shutil
    cache = tempfile.mkdtemp(prefix="pmrc-bench-kernels-")
    os.environ["PMRC_KERNEL_CACHE"] = cache
    atexit.register(shutil.rmtree, cache, True)
    import torch

    import paper_1412_3022_gb300 as P
    from paper_1412_3022_gb300 import inputs

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    B = args.block_bytes
    W = Workload(torch, P, inputs, B, rank_seed(args.seed, rank), dev)
    ops = W.ops()
    flush = L2Flush(torch, dev)
    stream = torch.cuda.current_stream()
    names = [n for n, _ in ops]
    ev = {n: [] for n in names}

    def step(record):
        for name, fn in ops:
            flush.fill_(7)
            if record:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            fn()
            if record:
                e1.record(stream)
                ev[name].append((e0, e1))

    for _ in range(args.warmup):
        step(False)
    # kernels compiled at run time in the background (the reconstruction's)
    # are ready and loaded before the timed steps
    P.wait_kernels()
    step(False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(True)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    ck = clocks.stop()
    op_ms = {n: sum(a.elapsed_time(b) for a, b in ev[n]) / args.steps for n in names}
    step_ms = ranks_max(dist, sum(op_ms.values()), dev)
    user_step = sum(W.user.values())
    value = whole_job_gbps(user_step, world, step_ms)
    hbm, peak_src = measured_peaks()

    per_op = {}
    for n in names:
        gbs = W.alg[n] / (op_ms[n] * 1e-3) / 1e9
        per_op[n] = {"ms": round(op_ms[n], 4), "alg_bytes": W.alg[n],
                     "hbm_GBps": round(gbs, 1), "frac_hbm": round(gbs / hbm, 4)}
    for n in ("gen_encode", "sys_encode", "decode"):
        per_op[n]["user_GBps"] = round(W.user[n] / (op_ms[n] * 1e-3) / 1e9, 2)
    rep_ms = op_ms["repair_helpers"] + op_ms["repair_newcomer"]
    per_op["repair"] = {"ms": round(rep_ms, 4),
                        "user_GBps": round(W.user["repair"] / (rep_ms * 1e-3) / 1e9, 2),
                        "frac_hbm": round((W.alg["repair_helpers"] + W.alg["repair_newcomer"])
                                          / (rep_ms * 1e-3) / 1e9 / hbm, 4),
                        "failed_node": W.f, "helper_reads": W.helper_reads}
    per_op["decode"]["nodes"] = W.S
    per_op["decode"]["missing_rows"] = W.decode_missing
    dom = max(names, key=lambda n: op_ms[n])
    ach = W.alg[dom] / (op_ms[dom] * 1e-3) / 1e9
    roofline = {"kernel": W.kernel[dom] + " (" + dom + ")", "bound": "hbm",
                "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(ach / hbm, 4), "peak_source": peak_src + " hbm_gbs (burst copy)",
                "traffic": None}
    # the same kernel against its integer-ALU ceiling (64 ALU lanes/clk/SM
    # on 152 SMs at the sampled clock); ALU lane-ops per launch measured by
    # ncu (sm__inst_executed_pipe_alu.sum x 32 on one launch of this
    # workload, profiles/kernel_counters.json), the instruction model beside
    # it; DRAM bytes per launch from the same captures
    mhz = (ck or {}).get("sm_mhz") or 2070.0
    peak_ops = 64.0 * SMS * mhz * 1e6 / 1e12
    counters = {}
    prof = os.path.join(ROOT, "profiles", "kernel_counters.json")
    if os.path.exists(prof):
        try:
            with open(prof) as f:
                counters = json.load(f).get("ops", {})
        except (OSError, ValueError):
            counters = {}

    def alu_lane_ops(n):
        c = counters.get(n, {})
        return (int(c["alu_warp_inst"]) * 32, "measured") if "alu_warp_inst" in c else (
            W.alu_ops[n], "model")

    lane_ops, src = alu_lane_ops(dom)
    ach_ops = lane_ops / (op_ms[dom] * 1e-3) / 1e12
    roofline["alu"] = {"unit": "T lane-ops/s", "achieved": round(ach_ops, 2),
                       "peak": round(peak_ops, 2), "frac": round(ach_ops / peak_ops, 4),
                       "lane_ops_per_launch": lane_ops, "lane_ops_source": src,
                       "model_lane_ops_per_launch": W.alu_ops[dom], "sm_mhz": mhz,
                       "model": W.alu_model[dom]}
    for n in names:
        per_op[n]["kernel"] = W.kernel[n]
        lo, src = alu_lane_ops(n)
        per_op[n]["alu_frac"] = round(lo / (op_ms[n] * 1e-3) / 1e12 / peak_ops, 4)
        per_op[n]["alu_source"] = src
        if "dram_bytes" in counters.get(n, {}):
            per_op[n]["traffic"] = int(counters[n]["dram_bytes"])
    if "dram_bytes" in counters.get(dom, {}):
        roofline["traffic"] = int(counters[dom]["dram_bytes"])

    # the end-to-end run comes before the extra rows: their handles, run-time
    # compilations and allocations stay out of its pipelined copy timing
    e2e = None if args.no_e2e else run_e2e(torch, W, args, dev, stream, dist, world, inputs)
    degraded = None
    if not args.no_extra:
        # the fused single-GPU repair (helper projections kept in scratch)
        fused_ms = time_op(torch, stream, flush, args, lambda: W.sysc.repair(
            W.f, W.c_H, W.c_args["helper_in"], W.c_args["node_ptrs"], B, W.stream))
        per_op["repair_fused"] = {"ms": round(fused_ms, 4),
                                  "user_GBps": round(W.user["repair"] / (fused_ms * 1e-3) / 1e9, 2),
                                  "alg_bytes": W.alg["repair_fused"],
                                  "frac_hbm": round(W.alg["repair_fused"] / (fused_ms * 1e-3) / 1e9
                                                    / hbm, 4)}
        # the paper's "specific" algorithms (Sec. 4) beside the linearized ones:
        # data-collector decode of the same node set, precode systematic encode
        ws_bytes = W.sysc.specific_workspace_bytes(B)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        spec = {
            "decode_specific": (lambda: W.sysc.decode_specific(
                W.c_S, W.c_args["dec_in"], W.c_args["dec_out"], B, ws.data_ptr(), ws_bytes, W.stream),
                "decode", W.user["decode"]),
            "encode_precode": (lambda: W.sysc.encode_precode(
                W.c_args["x_ptrs"], W.c_args["par_ptrs"], B, ws.data_ptr(), ws_bytes, W.stream),
                "sys_encode", W.user["sys_encode"]),
        }
        for name, (fn, linear, user) in spec.items():
            ms = time_op(torch, stream, flush, args, fn)
            per_op[name] = {"ms": round(ms, 4), "user_GBps": round(user / (ms * 1e-3) / 1e9, 2),
                            "linear_op": linear, "linear_over_specific": round(op_ms[linear] / ms, 3),
                            "launches": 5 if name == "encode_precode" else 4 + (W.decode_missing > 0)}
        del ws
        degraded = run_degraded(torch, P, inputs, W, args, flush, stream, dev, hbm)
        if not args.no_mbr:
            per_op.update(run_mbr(torch, P, inputs, args, flush, stream, dev, hbm))
            per_op.update(run_rs(torch, P, inputs, args, flush, stream, dev, hbm))
            per_op.update(run_gf16(torch, P, inputs, args, flush, stream, dev, hbm))
    sweep = None if (args.no_sweep or args.no_extra) else run_sweep(torch, P, inputs, args, flush,
                                                                    stream, dev, hbm)
    ksweep = None if (args.no_sweep or args.no_extra) else run_ksweep(torch, P, inputs, args, flush,
                                                                      stream, dev)
    init = None if args.no_extra else run_init(torch, P, inputs, args, dev)
    cfg1 = None if args.no_cfg1 else run_cfg1(torch, P, inputs, args, dev, stream)
    batched = None if args.no_batched else run_batched(torch, P, inputs, args, dev, stream)
    serving = None if args.no_serving else run_serving(torch, P, inputs, args)
    result = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 4),
        "wall_ms_per_step": round(wall * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded uniform random bytes, generated on device)",
        "config": {"workload": WORKLOAD, "block_bytes": B, "stripe_bytes": K_ * A_ * B,
                   "user_bytes_per_step": user_step, "l2": "flushed before every op, outside the timed events: "
                   "512 MiB write, then a 512 MiB read sweep (clean lines left in L2)",
                   "parallelism": f"replicas x{world} (independent stripes, no collective)"},
        "roofline": roofline,
        "per_op": per_op,
        "gpu_launches": 5 * args.steps,
        "clocks": ck,
        "paper_context_MBps": {"sys_encode_sparse_k8_16KB_1core": 790,
                               "sys_encode_vanilla_k8_1core": 210, "repair_sparse_1core": 480},
    }
    if e2e:
        result["e2e"] = e2e
    if sweep:
        result["block_sweep"] = sweep
    if ksweep:
        result["k_sweep"] = ksweep
    if init:
        result["init"] = init
    if cfg1:
        result["cfg1_latency"] = cfg1
    if degraded:
        result["degraded_read"] = degraded
    if batched:
        result["batched"] = batched
    if serving:
        result["serving"] = serving
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args, W, torch)
    if dist:
        dist.destroy_process_group()
    return result


def run_cfg1(torch, P, inputs, args, dev, stream):
    """The n=6, k=3, d=4 code of the small configuration: vanilla generator
    (non-systematic) encode of 6 data blocks of 4 KiB into 12, repair of node
    0 from helpers {1, 2, 3, 4} (projections + newcomer, and fused), and
    reconstruction from nodes {1, 2, 3}.  Latency-bound: each call is timed
    on its own over `args.cfg1_reps` repetitions, as device time between CUDA
    events around the call and as host time from the call to its completion
    (synchronized); p50 / p99 of both.  Results are checked on the device
    against the stored codeword and the data."""
    n, k, a, B = 6, 3, 2, 4096
    c = P.Code(n, k, P.PMRC_VANILLA, P.PMRC_NONSYSTEMATIC)
    X = inputs.device_blocks(k * a, B, args.seed + 11, device=dev)
    Y = torch.empty((n * a, B), dtype=torch.uint8, device=dev)
    f, H, S = 0, [1, 2, 3, 4], [1, 2, 3]
    recv = torch.empty((len(H), B), dtype=torch.uint8, device=dev)
    node = torch.empty((a, B), dtype=torch.uint8, device=dev)
    fused = torch.empty((a, B), dtype=torch.uint8, device=dev)
    Xd = torch.empty_like(X)
    st = int(stream.cuda_stream)
    x_p = P.ptr_array([X[i] for i in range(k * a)])
    y_p = P.ptr_array([Y[i] for i in range(n * a)])
    hb = P.ptr_array([Y[a * h + j] for h in H for j in range(a)])
    r_p = P.ptr_array([recv[i] for i in range(len(H))])
    n_p = P.ptr_array([node[j] for j in range(a)])
    f_p = P.ptr_array([fused[j] for j in range(a)])
    d_in = P.ptr_array([Y[a * i + j] for i in S for j in range(a)])
    d_out = P.ptr_array([Xd[r] for r in range(k * a)])
    cH, cS = P.int_array(H), P.int_array(S)
    ops = {
        "encode": lambda: c.encode(x_p, y_p, B, st),
        "repair": lambda: (c.repair_helpers(f, cH, hb, r_p, B, st),
                           c.repair_newcomer(f, cH, r_p, n_p, B, st)),
        "repair_fused": lambda: c.repair(f, cH, hb, f_p, B, st),
        "decode": lambda: c.decode(cS, d_in, d_out, B, st),
    }
    out = {"workload": "PM-MSR n=6 k=3 d=4 alpha=2, vanilla generator form, 4 KiB blocks: "
                       "encode 6 -> 12 blocks, repair of node 0 from {1,2,3,4}, "
                       "reconstruction from {1,2,3}",
           "reps": args.cfg1_reps}
    for name, fn in ops.items():
        for _ in range(20):
            fn()
        torch.cuda.synchronize()
        dev_ms, host_ms = [], []
        for _ in range(args.cfg1_reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            host_ms.append((time.perf_counter() - t0) * 1e3)
            dev_ms.append(e0.elapsed_time(e1))
        dev_ms.sort()
        host_ms.sort()
        q = lambda v, p: v[min(len(v) - 1, int(p * len(v)))]
        user = (k * a if name in ("encode", "decode") else a) * B
        out[name] = {"device_p50_ms": round(q(dev_ms, 0.5), 4), "device_p99_ms": round(q(dev_ms, 0.99), 4),
                     "host_p50_ms": round(q(host_ms, 0.5), 4), "host_p99_ms": round(q(host_ms, 0.99), 4),
                     "user_GBps_p50": round(user / (q(dev_ms, 0.5) * 1e-3) / 1e9, 3)}
    torch.cuda.synchronize()
    out["checked"] = bool(torch.equal(node, Y[a * f:a * f + a]) and torch.equal(fused, node)
                          and torch.equal(Xd, X))
    return out


def run_sweep(torch, P, inputs, args, flush, stream, dev, hbm):
    """The n=16 k=8 sparse systematic code at block sizes 64 KiB - 4 MiB:
    encode, repair of a seeded node (helpers + newcomer) and reconstruction
    from a seeded 8-node set, each on its own seeded stripe of that size."""
    out = {}
    for B in (64 << 10, 256 << 10, 1 << 20, 4 << 20):
        W = Workload(torch, P, inputs, B, args.seed + 500 + B % 977, dev)
        ops = dict(W.ops())
        row = {}
        for name, fn, user, alg in (
                ("sys_encode", ops["sys_encode"], W.user["sys_encode"], W.alg["sys_encode"]),
                ("repair", lambda: (ops["repair_helpers"](), ops["repair_newcomer"]()),
                 W.user["repair"], W.alg["repair_helpers"] + W.alg["repair_newcomer"]),
                ("decode", ops["decode"], W.user["decode"], W.alg["decode"])):
            ms = time_op(torch, stream, flush, args, fn)
            row[name] = {"ms": round(ms, 4), "user_GBps": round(user / (ms * 1e-3) / 1e9, 2),
                         "frac_hbm": round(alg / (ms * 1e-3) / 1e9 / hbm, 4)}
        row["decode"]["missing_rows"] = W.decode_missing
        out[f"{B >> 10} KiB"] = row
        del W
    torch.cuda.synchronize()
    return out


def run_degraded(torch, P, inputs, W, args, flush, stream, dev, hbm):
    """Degraded read of a lost systematic node of the stripe's code (a seeded
    node among the alpha first, whose helpers each contribute one block,
    Sec. 3.3): its alpha data blocks rebuilt by pmrc_read_degraded from the
    d helpers, against reading them through a reconstruction from k nodes
    (the other data nodes and one parity node, only the lost node's rows
    computed)."""
    B, a, K = W.B, A_, K_ * A_
    node = inputs.failed_node(A_, args.seed + 300)
    c, st = W.sysc, W.stream
    H = c.default_helpers(node)
    reads = int((c.helper_coefficients(node) != 0).sum())
    h_in = P.ptr_array([W.Y[a * h + j] for h in H for j in range(a)])
    out = torch.empty((a, B), dtype=torch.uint8, device=dev)
    out_arr = P.ptr_array([out[j] for j in range(a)])
    H_arr = P.int_array(H)
    S = [i for i in range(K_) if i != node] + [K_]
    dec_in = [W.Y[a * i + j] for i in S for j in range(a)]
    dec_out = [W.data_out[r] for r in range(K)]
    for pos, i in enumerate(S):             # surviving data stays in place
        if i < K_:
            for j in range(a):
                dec_out[a * i + j] = dec_in[a * pos + j]
    for j in range(a):
        dec_out[a * node + j] = out[j]
    S_arr, din, dout = P.int_array(S), P.ptr_array(dec_in), P.ptr_array(dec_out)
    R = c.decode_matrix(S)
    dec_reads = int((R[a * node:a * node + a] != 0).any(axis=0).sum())
    rows = {}
    for name, fn, alg in (
            ("via_repair", lambda: c.read_degraded(node, H_arr, h_in, out_arr, 0, B, st),
             (D_ * reads + a) * B),
            ("via_reconstruction", lambda: c.decode(S_arr, din, dout, B, st), (dec_reads + a) * B)):
        ms = time_op(torch, stream, flush, args, fn)
        rows[name] = {"ms": round(ms, 4), "user_GBps": round(a * B / (ms * 1e-3) / 1e9, 2),
                      "blocks_read": alg // B - a, "frac_hbm": round(alg / (ms * 1e-3) / 1e9 / hbm, 4)}
    rows["node"] = node
    del out
    return rows


def run_init(torch, P, inputs, args, dev):
    """Initialization, which the paper reports apart from throughput (Sec. 4):
    host wall time of building the n=16 k=8 codes (pmrc_create), and of the
    first reconstruction of a node set and the first repair of a failed node
    on a fresh handle beyond the same call repeated (host plans, their
    upload, and the reconstruction kernel compiled at run time), 1 MiB
    blocks."""
    B = args.block_bytes
    out = {}
    t0 = time.perf_counter()
    c = P.Code(N_, K_, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    out["create_sparse_systematic_ms"] = round((time.perf_counter() - t0) * 1e3, 3)
    t0 = time.perf_counter()
    P.Code(N_, K_, P.PMRC_VANILLA, P.PMRC_NONSYSTEMATIC)
    out["create_vanilla_ms"] = round((time.perf_counter() - t0) * 1e3, 3)
    a, K = A_, K_ * A_
    seed = args.seed + 700
    Y = torch.empty((N_ * a, B), dtype=torch.uint8, device=dev)
    Y[:K] = inputs.device_blocks(K, B, seed, device=dev)
    c.encode([Y[i] for i in range(K)], [Y[K + r] for r in range(K)], B)
    S = inputs.node_subset(N_, K_, seed)
    Xr = torch.empty((K, B), dtype=torch.uint8, device=dev)
    din = [Y[a * i + j] for i in S for j in range(a)]
    f = inputs.failed_node(N_, seed)
    H = c.default_helpers(f)
    hin = [Y[a * h + j] for h in H for j in range(a)]
    recv = torch.empty((D_, B), dtype=torch.uint8, device=dev)
    node = torch.empty((a, B), dtype=torch.uint8, device=dev)

    def wall(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) * 1e3

    dec = lambda: c.decode(S, din, [Xr[r] for r in range(K)], B)
    rep = lambda: (c.repair_helpers(f, H, hin, [recv[i] for i in range(D_)], B),
                   c.repair_newcomer(f, H, [recv[i] for i in range(D_)], [node[j] for j in range(a)], B))
    first = wall(dec)                    # host plan; compilation started
    t = time.perf_counter()
    c.wait_kernels()
    ready = first + (time.perf_counter() - t) * 1e3
    wall(dec)                            # loads the compiled kernel
    again = min(wall(dec) for _ in range(3))
    out["decode_pattern_first_call_ms"] = round(first, 2)
    out["decode_pattern_kernel_ready_ms"] = round(ready, 2)
    out["decode_pattern_init_ms"] = round(first - again, 2)
    # a new handle (as in a new process) has none of these kernels loaded:
    # its first reconstruction of the same node set finds the compiled
    # kernel in the on-disk cache instead of running NVRTC again
    c2 = P.Code(N_, K_, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    first2 = wall(lambda: c2.decode(S, din, [Xr[r] for r in range(K)], B))
    t = time.perf_counter()
    c2.wait_kernels()
    out["decode_pattern_kernel_ready_from_disk_cache_ms"] = round(
        first2 + (time.perf_counter() - t) * 1e3, 2)
    del c2
    first = wall(rep)                    # plans; the newcomer's kernel compiling
    t = time.perf_counter()
    c.wait_kernels()                     # (no compilation outlives this section)
    ready = first + (time.perf_counter() - t) * 1e3
    wall(rep)
    again = min(wall(rep) for _ in range(3))
    out["repair_pattern_init_ms"] = round(first - again, 2)
    out["repair_pattern_kernel_ready_ms"] = round(ready, 2)
    out["note"] = ("host wall clock; a pattern's first call builds its plans and starts "
                   "compiling its bitsliced kernel (NVRTC: the reconstruction's, the newcomer's, "
                   "the helper projections') in the background, running the split-table kernel "
                   "meanwhile; kernel_ready is when the compilation ended; the bench runs with an "
                   "empty on-disk kernel cache of its own, so the first compilations are cold")
    del Y, Xr, recv, node, c
    torch.cuda.synchronize()
    return out


def run_ksweep(torch, P, inputs, args, flush, stream, dev):
    """Throughput against k, the axis of the paper's encode and repair
    figures (Sec. 4, k up to 32 at 16 KB blocks): the n = 2k sparse
    systematic code for k in {4, 8, 12, 16, 24, 32} at 16 KiB and 1 MiB
    blocks -- systematic encode, repair of a seeded node (helper projections
    + newcomer) and lazy reconstruction from a seeded k-node set.  From
    k = 24 the operations exceed one launch's 1024 block pointers and run as
    several launches."""
    out = {}
    st = int(torch.cuda.current_stream(dev).cuda_stream)
    for B in (16 << 10, 1 << 20):
        rows = {}
        for k in (4, 8, 12, 16, 24, 32):
            n, a, d, K = 2 * k, k - 1, 2 * k - 2, k * (k - 1)
            seed = args.seed + 900 + k
            c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
            Y = torch.empty((n * a, B), dtype=torch.uint8, device=dev)
            Y[:K] = inputs.device_blocks(K, B, seed, device=dev)
            x_arr = P.ptr_array([Y[i] for i in range(K)])
            par_arr = P.ptr_array([Y[K + r] for r in range(n * a - K)])
            c.encode(x_arr, par_arr, B, st)
            f = inputs.failed_node(n, seed)
            H_arr = P.int_array(c.default_helpers(f))
            h_in = P.ptr_array([Y[a * h + j] for h in H_arr for j in range(a)])
            recv = torch.empty((d, B), dtype=torch.uint8, device=dev)
            node = torch.empty((a, B), dtype=torch.uint8, device=dev)
            recv_arr = P.ptr_array([recv[i] for i in range(d)])
            node_arr = P.ptr_array([node[j] for j in range(a)])
            S = inputs.node_subset(n, k, seed)
            Xr = torch.empty((K, B), dtype=torch.uint8, device=dev)
            dec_in = [Y[a * i + j] for i in S for j in range(a)]
            dec_out = [Xr[r] for r in range(K)]
            for pos, i in enumerate(S):       # data blocks of surviving data nodes stay put
                if i < k:
                    for j in range(a):
                        dec_out[a * i + j] = dec_in[a * pos + j]
            S_arr, din, dout = P.int_array(S), P.ptr_array(dec_in), P.ptr_array(dec_out)
            ops = {
                "sys_encode": (lambda: c.encode(x_arr, par_arr, B, st), K * B),
                "repair": (lambda: (c.repair_helpers(f, H_arr, h_in, recv_arr, B, st),
                                    c.repair_newcomer(f, H_arr, recv_arr, node_arr, B, st)), a * B),
                "decode": (lambda: c.decode(S_arr, din, dout, B, st), K * B),
            }
            row = {}
            for name, (fn, user) in ops.items():
                ms = time_op(torch, stream, flush, args, fn)
                row[name] = {"ms": round(ms, 4), "user_GBps": round(user / (ms * 1e-3) / 1e9, 2)}
            row["decode"]["missing_rows"] = a * sum(1 for i in range(k) if i not in S)
            rows[f"k={k}"] = row
            del Y, recv, node, Xr, c
        out[f"{B >> 10} KiB"] = rows
    torch.cuda.synchronize()
    return out


def run_mbr(torch, P, inputs, args, flush, stream, dev, hbm):
    """PM-MBR rows (n=16, k=8, d=14: alpha=14, K=84 data blocks of the
    stripe's block size): systematic encode (112 parity blocks), fused repair
    of a seeded node, lazy reconstruction from a seeded 8-node set."""
    n, k, d, B = 16, 8, 14, args.block_bytes
    c = P.Code(n, k, P.PMRC_MBR, P.PMRC_SYSTEMATIC, d=d)
    a, K = c.alpha, c.data_blocks
    st = int(torch.cuda.current_stream(dev).cuda_stream)
    X = inputs.device_blocks(K, B, args.seed + 77, device=dev)
    Y = torch.empty((n * a, B), dtype=torch.uint8, device=dev)
    cn = P.Code(n, k, P.PMRC_MBR, P.PMRC_NONSYSTEMATIC, d=d)
    cn.encode(P.ptr_array([X[i] for i in range(K)]), P.ptr_array([Y[r] for r in range(n * a)]), B)
    f = inputs.failed_node(n, args.seed + 77)
    H = c.default_helpers(f)
    S = inputs.node_subset(n, k, args.seed + 77)
    coef = P.pmrc_helper_coefficients(c.handle, f)
    reads = int((coef != 0).sum())
    node = torch.empty((a, B), dtype=torch.uint8, device=dev)
    Xr = torch.empty((K, B), dtype=torch.uint8, device=dev)
    dec_in = [Y[a * i + j] for i in S for j in range(a)]
    dec_out = [Xr[r] for r in range(K)]
    G = P.pmrc_code_generator(c.handle)
    for pos, i in enumerate(S):          # data blocks held verbatim stay in place
        for j in range(a):
            col = np.flatnonzero(G[a * i + j])
            if len(col) == 1 and G[a * i + j, col[0]] == 1:
                dec_out[int(col[0])] = dec_in[a * pos + j]
    missing = sum(1 for r in range(K) if dec_out[r] is not None and
                  dec_out[r].data_ptr() == Xr[r].data_ptr())
    R = P.pmrc_decode_matrix(c.handle, S)
    dec_reads = int((R[[r for r in range(K) if dec_out[r].data_ptr() == Xr[r].data_ptr()]]
                     != 0).any(axis=0).sum()) if missing else 0
    x_arr = P.ptr_array([X[i] for i in range(K)])
    par_arr = P.ptr_array([Y[k * a + r] for r in range(n * a - k * a)])
    H_arr = P.int_array(H)
    h_in = P.ptr_array([Y[a * h + j] for h in H for j in range(a)])
    node_arr = P.ptr_array([node[j] for j in range(a)])
    S_arr = P.int_array(S)
    din, dout = P.ptr_array(dec_in), P.ptr_array(dec_out)
    ops = {
        "mbr_encode": (lambda: c.encode(x_arr, par_arr, B, st), K * B, (K + n * a - k * a) * B),
        "mbr_repair": (lambda: c.repair(f, H_arr, h_in, node_arr, B, st), a * B,
                       (d * reads + a) * B),
        "mbr_decode": (lambda: c.decode(S_arr, din, dout, B, st), K * B,
                       (dec_reads + missing) * B),
    }
    out = {}
    for name, (fn, user, alg) in ops.items():
        ms = time_op(torch, stream, flush, args, fn)
        out[name] = {"ms": round(ms, 4), "user_GBps": round(user / (ms * 1e-3) / 1e9, 2),
                     "alg_bytes": alg, "frac_hbm": round(alg / (ms * 1e-3) / 1e9 / hbm, 4)}
    out["mbr_repair"].update({"failed_node": f, "helper_reads": reads})
    out["mbr_decode"].update({"nodes": S, "missing_rows": missing})
    torch.cuda.synchronize()
    return out


def run_rs(torch, P, inputs, args, flush, stream, dev, hbm):
    """Reed-Solomon baseline rows (the paper's comparison code, Sec. 4):
    RS(16, 8) systematic over the same 56 MiB stripe (8 data blocks of
    7 x the block size): encode, repair of a seeded node from 8 helpers,
    lazy decode from a seeded 8-node set."""
    n, k, B = 16, 8, 7 * args.block_bytes
    c = P.Code(n, k, P.PMRC_RS, P.PMRC_SYSTEMATIC)
    st = int(torch.cuda.current_stream(dev).cuda_stream)
    Y = torch.empty((n, B), dtype=torch.uint8, device=dev)
    Y[:k].copy_(inputs.device_blocks(k, B, args.seed + 88, device=dev))
    c.encode(P.ptr_array([Y[i] for i in range(k)]), P.ptr_array([Y[k + i] for i in range(n - k)]), B)
    f = inputs.failed_node(n, args.seed + 88)
    H = c.default_helpers(f)
    S = inputs.node_subset(n, k, args.seed + 88)
    node = torch.empty((1, B), dtype=torch.uint8, device=dev)
    Xr = torch.empty((k, B), dtype=torch.uint8, device=dev)
    dec_in = [Y[i] for i in S]
    dec_out = [Xr[r] for r in range(k)]
    for pos, i in enumerate(S):       # present data blocks stay in place
        if i < k:
            dec_out[i] = dec_in[pos]
    missing = [r for r in range(k) if r not in S]
    x_arr, par_arr = P.ptr_array([Y[i] for i in range(k)]), P.ptr_array([Y[k + i] for i in range(n - k)])
    H_arr, h_in, n_out = P.int_array(H), P.ptr_array([Y[h] for h in H]), P.ptr_array([node[0]])
    S_arr, din, dout = P.int_array(S), P.ptr_array(dec_in), P.ptr_array(dec_out)
    ops = {
        "rs_encode": (lambda: c.encode(x_arr, par_arr, B, st), k * B, (k + n - k) * B),
        "rs_repair": (lambda: c.repair(f, H_arr, h_in, n_out, B, st), B, (k + 1) * B),
        "rs_decode": (lambda: c.decode(S_arr, din, dout, B, st), k * B,
                      ((k if missing else 0) + len(missing)) * B),
    }
    out = {}
    for name, (fn, user, alg) in ops.items():
        ms = time_op(torch, stream, flush, args, fn)
        out[name] = {"ms": round(ms, 4), "user_GBps": round(user / (ms * 1e-3) / 1e9, 2),
                     "alg_bytes": alg, "frac_hbm": round(alg / (ms * 1e-3) / 1e9 / hbm, 4),
                     "block_bytes": B}
    out["rs_repair"]["failed_node"] = f
    out["rs_decode"].update({"nodes": S, "missing_rows": len(missing)})
    torch.cuda.synchronize()
    return out


def run_gf16(torch, P, inputs, args, flush, stream, dev, hbm):
    """GF(2^16) rows: the n=16 k=8 sparse systematic code over GF(2^16) on
    the same 56 MiB stripe (blocks of two byte planes): encode, two-step
    repair of a seeded node, lazy decode from a seeded 8-node set."""
    n, k, B = 16, 8, args.block_bytes
    a, K = k - 1, k * (k - 1)
    c = P.Code(n, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC, field_bits=16)
    st = int(torch.cuda.current_stream(dev).cuda_stream)
    Y = torch.empty((n * a, B), dtype=torch.uint8, device=dev)
    Y[:K].copy_(inputs.device_blocks(K, B, args.seed + 99, device=dev))
    x_arr = P.ptr_array([Y[i] for i in range(K)])
    par_arr = P.ptr_array([Y[K + i] for i in range(K)])
    c.encode(x_arr, par_arr, B)
    f = inputs.failed_node(n, args.seed + 99)
    H = c.default_helpers(f)
    S = inputs.node_subset(n, k, args.seed + 99)
    recv = torch.empty((2 * k - 2, B), dtype=torch.uint8, device=dev)
    node = torch.empty((a, B), dtype=torch.uint8, device=dev)
    Xr = torch.empty((K, B), dtype=torch.uint8, device=dev)
    dec_in = [Y[a * i + j] for i in S for j in range(a)]
    dec_out = [Xr[r] for r in range(K)]
    for pos, i in enumerate(S):
        if i < k:
            for j in range(a):
                dec_out[a * i + j] = dec_in[a * pos + j]
    missing = sum(1 for i in range(k) if i not in S) * a
    H_arr, S_arr = P.int_array(H), P.int_array(S)
    h_in = P.ptr_array([Y[a * h + j] for h in H for j in range(a)])
    r_arr, n_arr = P.ptr_array([recv[i] for i in range(2 * k - 2)]), P.ptr_array([node[j] for j in range(a)])
    din, dout = P.ptr_array(dec_in), P.ptr_array(dec_out)

    def repair():
        c.repair_helpers(f, H_arr, h_in, r_arr, B, st)
        c.repair_newcomer(f, H_arr, r_arr, n_arr, B, st)
    ops = {
        "gf16_sys_encode": (lambda: c.encode(x_arr, par_arr, B, st), K * B, 2 * K * B),
        "gf16_repair": (repair, a * B, ((2 * k - 2) * a + 2 * (2 * k - 2) + a) * B),
        "gf16_decode": (lambda: c.decode(S_arr, din, dout, B, st), K * B, (K + missing) * B),
    }
    out = {}
    for name, (fn, user, alg) in ops.items():
        ms = time_op(torch, stream, flush, args, fn)
        out[name] = {"ms": round(ms, 4), "user_GBps": round(user / (ms * 1e-3) / 1e9, 2),
                     "alg_bytes": alg, "frac_hbm": round(alg / (ms * 1e-3) / 1e9 / hbm, 4)}
    out["gf16_repair"]["failed_node"] = f
    out["gf16_decode"].update({"nodes": S, "missing_rows": missing})
    torch.cuda.synchronize()
    return out


def time_op(torch, stream, flush, args, fn):
    """Average device time of fn over args.steps runs, L2 flushed before each;
    after the warm-up, any kernel compiled at run time in the background is
    waited for and loaded, so the timed runs use it."""
    import paper_1412_3022_gb300 as P
    for _ in range(args.warmup):
        flush.fill_(3)
        fn()
    P.wait_kernels()
    fn()
    tot = 0.0
    for _ in range(args.steps):
        flush.fill_(5)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / args.steps


def run_batched(torch, P, inputs, args, dev, stream):
    """Batched workload: stripes with k uniform on {4, 8, 16} (n = 2k, sparse
    systematic), block sizes log-uniform on [4 KiB, 1 MiB] rounded up to 16 B,
    half encode and half repair (fused, default helpers of a seeded failed
    node).  One persistent launch from a CUDA graph, tuned by the library's
    autotuner, against the same stripes issued as plain per-stripe calls."""
    import numpy as np
    mix = inputs.batch_mix(args.batch_stripes, seed=args.seed + 4)
    codes = {k: P.Code(2 * k, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC) for k in (4, 8, 16)}
    # one arena for every block of the workload
    need = 0
    for m in mix:
        k, a, nb = m["k"], m["k"] - 1, m["block_bytes"]
        need += (2 * k * a if m["op"] == "encode" else 2 * k * a + a) * nb
    free, _ = torch.cuda.mem_get_info()
    scale_note = None
    if need > 0.8 * free:
        keep = max(16, int(len(mix) * 0.8 * free / need))
        scale_note = f"device memory: {keep} of {len(mix)} stripes"
        mix = mix[:keep]
        need = sum((2 * m["k"] * (m["k"] - 1) + (0 if m["op"] == "encode" else m["k"] - 1))
                   * m["block_bytes"] for m in mix)
    arena = torch.empty(need, dtype=torch.uint8, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(args.seed + 5)
    chunk = 1 << 30
    for o in range(0, need, chunk):  # seeded random fill, in 1 GiB pieces
        arena[o:o + chunk].random_(0, 256, generator=g)
    base = arena.data_ptr()
    ops, off = [], 0
    for m in mix:
        k, a, nb = m["k"], m["k"] - 1, m["block_bytes"]
        c = codes[k]
        if m["op"] == "encode":
            ins = [base + off + i * nb for i in range(k * a)]
            outs = [base + off + (k * a + i) * nb for i in range(k * a)]
            span = (off + k * a * nb, k * a * nb)
            off += 2 * k * a * nb
            ops.append(("encode", c, ins, outs, nb, dict(m, span=span, alg=2 * k * a * nb)))
        else:
            Y = [base + off + i * nb for i in range(2 * k * a)]
            outs = [base + off + (2 * k * a + j) * nb for j in range(a)]
            span = (off + 2 * k * a * nb, a * nb)
            off += (2 * k * a + a) * nb
            c.encode(Y[:k * a], Y[k * a:], nb)  # stored codeword
            f = m["failed"]
            H = c.default_helpers(f)
            reads = int((c.helper_coefficients(f) != 0).sum())
            ops.append(("repair", c, [Y[a * h + j] for h in H for j in range(a)], outs, nb,
                        dict(m, H=H, span=span, alg=(len(H) * reads + a) * nb)))
    torch.cuda.synchronize()
    user = sum((m["k"] * (m["k"] - 1) if op == "encode" else m["k"] - 1) * m["block_bytes"]
               for op, _, _, _, _, m in ops)
    b = P.Batch()
    for op, c, ins, outs, nb, m in ops:
        if op == "encode":
            b.add_encode(c, ins, outs, nb)
        else:
            b.add_repair(c, m["failed"], m["H"], ins, outs, nb)
    t0 = time.perf_counter()
    best = b.tune(stream)
    tune_s = time.perf_counter() - t0
    info = b.info()

    def run_batch():
        b.launch(stream)

    def run_plain():
        for op, c, ins, outs, nb, m in ops:
            if op == "encode":
                c.encode(ins, outs, nb, stream)
            else:
                c.repair(m["failed"], m["H"], ins, outs, nb, stream)

    reps = 3
    res = {}
    for name, fn in (("batched", run_batch), ("plain", run_plain)):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = (e0.elapsed_time(e1) / reps, (time.perf_counter() - t0) * 1e3 / reps)
    # every stripe of the batched launch equals the same stripe run through
    # the plain call (compared on the device, one stripe at a time)
    b.launch(stream)
    torch.cuda.synchronize()
    mismatches = 0
    scratch = torch.empty(max(m["span"][1] for _, _, _, _, _, m in ops), dtype=torch.uint8,
                          device=dev)
    for op, c, ins, outs, nb, m in ops:
        o, ln = m["span"]
        view = arena[o:o + ln]
        scratch[:ln].copy_(view)
        if op == "encode":
            c.encode(ins, outs, nb, stream)
        else:
            c.repair(m["failed"], m["H"], ins, outs, nb, stream)
        mismatches += int(not torch.equal(scratch[:ln], view))
    del scratch
    alg = sum(m["alg"] for _, _, _, _, _, m in ops)
    hbm, peak_src = measured_peaks()
    out = {
        "workload": f"{len(ops)} stripes, k uniform on {{4,8,16}} (n=2k, sparse systematic), "
                    "block sizes log-uniform 4 KiB-1 MiB, 50% encode / 50% fused repair",
        "checked": mismatches == 0, "stripes_differing_from_plain_calls": mismatches,
        "alg_GB": round(alg / 1e9, 3),
        "batched_frac_hbm": round(alg / (res["batched"][0] * 1e-3) / 1e9 / hbm, 4),
        "plain_frac_hbm": round(alg / (res["plain"][0] * 1e-3) / 1e9 / hbm, 4),
        "user_GB": round(user / 1e9, 3),
        "batched_GBps": round(user / (res["batched"][0] * 1e-3) / 1e9, 1),
        "batched_ms": round(res["batched"][0], 3),
        "plain_GBps": round(user / (res["plain"][0] * 1e-3) / 1e9, 1),
        "plain_ms": round(res["plain"][0], 3),
        "plain_wall_ms": round(res["plain"][1], 3),
        "speedup": round(res["plain"][0] / res["batched"][0], 3),
        "launches": {"batched": 1 + info["bitsliced_launches"], "plain": len(ops)},
        "tuned": {"work_bytes": best[0], "ctas_per_sm": best[1], "tune_s": round(tune_s, 2),
                  "items": info["items"], "ctas": info["ctas"],
                  "bitsliced_launches": info["bitsliced_launches"]},
        "l2": "not flushed (working set far larger than L2)",
    }
    if scale_note:
        out["note"] = scale_note
    del arena
    del np
    return out


def run_serving(torch, P, inputs, args):
    """Serving workload: Poisson arrivals of encode / repair / reconstruct
    requests (60/25/15), k uniform on {4, 8, 12, 16} (n = 2k, sparse
    systematic), stripes log-uniform on [64 KiB, 64 MiB] split into k*alpha
    blocks (the last one zero-padded), host buffers pinned.  First the
    saturated rate (all requests arriving at once), then offered loads of
    25/50/75/90% of it; latency runs from a request's scheduled arrival to
    its completion seen by the host (a late submission counts), with the
    client's garbage collector paused in the timed loops.  `link` measures
    the pinned host link (256 MiB copies, each direction alone and both at
    once) and the mix's ceiling: the user GB/s at which its host-to-device
    and device-to-host bytes fill the link with both directions running.
    Three arms on the same requests and arrival times:

      served          the continuous-batching server, host buffers (inputs
                      copied in, results copied out, per request);
      device_resident the same server with every request's blocks already in
                      device memory (PMRC_REQ_DEVICE: no copies), at
                      saturation: the GPU side of continuous batching;
      plain           one request at a time through the single-stripe calls
                      in arrival order (copy in, call, copy out, wait), on one
                      stream: the per-stripe launches without batching."""
    import numpy as np
    dev = torch.device("cuda", torch.cuda.current_device())
    n = args.serve_requests
    reqs_all = inputs.serve_requests(n * 5, seed=args.seed + 6)
    codes = {k: P.Code(2 * k, k, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC) for k in (4, 8, 12, 16)}

    def sizes(q):
        k = q["k"]
        a, d = k - 1, 2 * k - 2
        B = q["block_bytes"]
        if q["op"] == "encode":
            return k * a * B, k * a * B, k * a * B
        if q["op"] == "repair":
            return d * a * B, a * B, a * B
        return k * a * B, k * a * B, k * a * B

    max_in = max(sizes(q)[0] for q in reqs_all)
    max_out = max(sizes(q)[1] for q in reqs_all)
    g = torch.Generator()
    g.manual_seed(args.seed + 7)
    hin = torch.randint(0, 256, (max_in,), dtype=torch.uint8, generator=g).pin_memory()
    hout = torch.empty(max_out, dtype=torch.uint8).pin_memory()
    din = torch.empty(max_in, dtype=torch.uint8, device=dev)
    din.copy_(hin)
    dout = torch.empty(max_out, dtype=torch.uint8, device=dev)
    helpers = {}
    for k, c in codes.items():
        for f in range(2 * k):
            helpers[(k, f)] = c.default_helpers(f)
    budget = 16 << 30
    srv = P.Server(budget_bytes=budget, max_slots=64)
    opcode = {"encode": P.PMRC_OP_ENCODE, "repair": P.PMRC_OP_REPAIR,
              "decode": P.PMRC_OP_DECODE}

    def submit(q, device):
        k = q["k"]
        op = opcode[q["op"]] | (P.PMRC_REQ_DEVICE if device else 0)
        return srv.submit(op, codes[k], q["block_bytes"], din if device else hin,
                          dout if device else hout, failed=q["failed"],
                          helpers=helpers[(k, q["failed"])], nodes=q["nodes"])

    def arrivals(batch, rate):
        rng = np.random.default_rng(args.seed + 8)
        t, out = 0.0, []
        for _ in batch:
            if rate:
                t += rng.exponential(1.0 / rate)
            out.append(t)
        return out

    def summary(batch, lats, wall):
        user = sum(sizes(q)[2] for q in batch)
        lat = np.array(lats)
        ub = np.array([sizes(q)[2] for q in batch])
        by_size = {}
        for name, lo, hi in (("<1MiB", 0, 1 << 20), ("1-8MiB", 1 << 20, 8 << 20),
                             (">8MiB", 8 << 20, 1 << 62)):
            m = (ub >= lo) & (ub < hi)
            if m.any():
                by_size[name] = {"requests": int(m.sum()),
                                 "p50_ms": round(float(np.percentile(lat[m], 50)), 3),
                                 "p99_ms": round(float(np.percentile(lat[m], 99)), 3)}
        return {"requests": len(batch), "p50_ms": round(float(np.percentile(lat, 50)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "max_ms": round(float(lat.max()), 3), "GBps": round(user / wall / 1e9, 2),
                "by_size": by_size}

    def run(batch, rate, device=False):
        srv.reset_stats()
        ids, late = [], []
        when = arrivals(batch, rate)
        gc.collect()
        gc.disable()   # no collector pause inside the client's submission loop
        t0 = time.perf_counter()
        for q, tq in zip(batch, when):
            dt = t0 + tq - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            late.append((time.perf_counter() - t0 - tq) * 1e3)
            ids.append(submit(q, device))
        lats, lost = [], 0
        for rid, lt in zip(ids, late):
            try:   # from the arrival time: the client's lateness plus the server's latency
                lats.append(lt + srv.wait(rid, timeout_ms=120000)[1])
            except P.PMRCError:
                lost += 1
        wall = time.perf_counter() - t0
        gc.enable()
        st = srv.stats()
        if lost or st["failed"]:
            raise RuntimeError(f"serving: {lost} requests timed out, {int(st['failed'])} failed")
        out = summary(batch, lats, wall)
        out.update({"iterations": int(st["iterations"]), "peak_GB": round(st["peak_bytes"] / 1e9, 2)})
        return out

    stream = torch.cuda.Stream(device=dev)
    st_handle = int(stream.cuda_stream)

    def plain_call(q):
        k, B = q["k"], q["block_bytes"]
        a = k - 1
        c = codes[k]
        nin, nout = sizes(q)[0] // B, sizes(q)[1] // B
        ib, ob = din.data_ptr(), dout.data_ptr()
        ins = P.ptr_array([ib + i * B for i in range(nin)])
        outs = P.ptr_array([ob + j * B for j in range(nout)])
        with torch.cuda.stream(stream):
            din[:nin * B].copy_(hin[:nin * B], non_blocking=True)
        if q["op"] == "encode":
            c.encode(ins, outs, B, st_handle)
        elif q["op"] == "repair":
            c.repair(q["failed"], helpers[(k, q["failed"])], ins, outs, B, st_handle)
        else:
            c.decode(q["nodes"], ins, outs, B, st_handle)
        with torch.cuda.stream(stream):
            hout[:nout * B].copy_(dout[:nout * B], non_blocking=True)
        stream.synchronize()
        del a

    def run_plain(batch, rate):
        when = arrivals(batch, rate)
        lats = []
        gc.collect()
        gc.disable()
        t0 = time.perf_counter()
        for q, tq in zip(batch, when):
            dt = t0 + tq - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            plain_call(q)
            lats.append((time.perf_counter() - t0 - tq) * 1e3)
        wall = time.perf_counter() - t0
        gc.enable()
        return summary(batch, lats, wall)

    def link():
        """Pinned 256 MiB copies: each direction alone and both at once on
        two streams (GB/s per direction)."""
        size = 256 << 20
        h1 = torch.empty(size, dtype=torch.uint8).pin_memory()
        h2 = torch.empty(size, dtype=torch.uint8).pin_memory()
        d1 = torch.empty(size, dtype=torch.uint8, device=dev)
        d2 = torch.empty(size, dtype=torch.uint8, device=dev)
        sa, sb = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        best = {"h2d": 0.0, "d2h": 0.0, "both_h2d": 0.0, "both_d2h": 0.0}
        for _ in range(4):
            for key, fn in (("h2d", lambda: d1.copy_(h1, non_blocking=True)),
                            ("d2h", lambda: h2.copy_(d2, non_blocking=True))):
                ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                with torch.cuda.stream(sa):
                    ea.record(sa)
                    fn()
                    eb.record(sa)
                torch.cuda.synchronize()
                best[key] = max(best[key], size / (ea.elapsed_time(eb) * 1e-3) / 1e9)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            torch.cuda.synchronize()
            with torch.cuda.stream(sa):
                ev[0].record(sa)
                d1.copy_(h1, non_blocking=True)
                ev[1].record(sa)
            with torch.cuda.stream(sb):
                ev[2].record(sb)
                h2.copy_(d2, non_blocking=True)
                ev[3].record(sb)
            torch.cuda.synchronize()
            best["both_h2d"] = max(best["both_h2d"], size / (ev[0].elapsed_time(ev[1]) * 1e-3) / 1e9)
            best["both_d2h"] = max(best["both_d2h"], size / (ev[2].elapsed_time(ev[3]) * 1e-3) / 1e9)
        del h1, h2, d1, d2
        return {k: round(v, 1) for k, v in best.items()}

    warm = reqs_all[:min(64, n)]
    run(warm, 0)             # plans, pools, kernels
    run(warm, 0, device=True)
    for q in warm:
        plain_call(q)
    P.wait_kernels()
    sat = run(reqs_all[:n], 0)
    mean_user = sum(sizes(q)[2] for q in reqs_all[:n]) / n
    tot = np.array([sizes(q) for q in reqs_all[:n]], dtype=float).sum(0)
    lk = link()
    h_per, d_per = tot[0] / tot[2], tot[1] / tot[2]
    lk.update({"h2d_bytes_per_user_byte": round(h_per, 3), "d2h_bytes_per_user_byte": round(d_per, 3),
               "ceiling_GBps": round(min(lk["both_h2d"] / h_per, lk["both_d2h"] / d_per), 1)})
    out = {"workload": "Poisson arrivals; encode/repair/reconstruct 60/25/15; k in {4,8,12,16} "
                       "(n=2k, sparse systematic); stripes log-uniform 64 KiB-64 MiB; pinned "
                       "host buffers; HBM budget 16 GiB, 64 slots",
           "requests_per_level": n,
           "saturated": sat, "loads": {}, "link": lk,
           "device_resident": {"saturated": run(reqs_all[:n], 0, device=True)},
           "plain": {"loads": {}}}
    levels = []
    for i, load in enumerate((0.25, 0.5, 0.75, 0.9)):
        rate = load * sat["GBps"] * 1e9 / mean_user
        levels.append((f"{int(load * 100)}%", reqs_all[(i + 1) * n:(i + 2) * n], rate,
                       round(load * sat["GBps"], 2)))
    # every served run comes first: the plain calls compile run-time kernels
    # in the background (default policy), which must not overlap a served run
    for name, batch, rate, offered in levels:
        r = run(batch, rate)
        r["offered_GBps"] = offered
        out["loads"][name] = r
    out["plain"]["saturated"] = run_plain(reqs_all[:n], 0)
    for name, batch, rate, offered in levels:
        rp = run_plain(batch, rate)
        rp["offered_GBps"] = offered
        out["plain"]["loads"][name] = rp
    out["served_over_plain_saturated"] = round(sat["GBps"] / out["plain"]["saturated"]["GBps"], 3)
    out["served_over_link_ceiling"] = round(sat["GBps"] / lk["ceiling_GBps"], 3)
    out["device_resident_over_host_saturated"] = round(
        out["device_resident"]["saturated"]["GBps"] / sat["GBps"], 3)
    srv.close()
    del np
    return out


def run_e2e(torch, W, args, dev, stream, dist=None, world=1, inputs=None):
    """Same step through the public API with host buffers: pinned H2D of the
    stripe, every operation, D2H of every block the step produced.  Steps
    are pipelined the way a streaming caller runs them: two device buffer
    sets on three streams (copy in, compute, copy out), so the copies of one
    step overlap the compute and copies of its neighbours; every step still
    moves its own inputs in and all its results out."""
    B, K, a = W.B, K_ * A_, A_
    hx = torch.empty((K, B), dtype=torch.uint8).pin_memory()
    hx.copy_(W.X.cpu())
    out_rows = W.gen_out.shape[0] + K + a + W.decode_missing
    hout = torch.empty((out_rows, B), dtype=torch.uint8).pin_memory()
    present = {a * i + j for i in W.S if i < K_ for j in range(a)}
    missing = [r for r in range(K) if r not in present]
    runs = []                                 # consecutive missing rows: one copy each
    for r in missing:
        if runs and runs[-1][1] == r:
            runs[-1][1] = r + 1
        else:
            runs.append([r, r + 1])
    sets = [W, Workload(torch, W.P, inputs, B, W.seed, dev)]   # same stripe, own buffers
    s_in, s_comp, s_out = (torch.cuda.Stream(device=dev) for _ in range(3))
    opsets = [S.ops(int(s_comp.cuda_stream)) for S in sets]
    ev_in = [torch.cuda.Event() for _ in sets]
    ev_comp = [torch.cuda.Event() for _ in sets]
    ev_out = [torch.cuda.Event() for _ in sets]
    for e in ev_out:
        e.record(s_out)

    def step(i):
        b = i % 2
        S = sets[b]
        s_in.wait_event(ev_out[b])           # buffers of step i-2 are free
        with torch.cuda.stream(s_in):
            S.X.copy_(hx, non_blocking=True)
        ev_in[b].record(s_in)
        s_comp.wait_event(ev_in[b])
        for _, fn in opsets[b]:
            fn()
        ev_comp[b].record(s_comp)
        s_out.wait_event(ev_comp[b])
        with torch.cuda.stream(s_out):
            o = 0
            hout[o:o + N_ * a].copy_(S.gen_out, non_blocking=True)
            o += N_ * a
            hout[o:o + K].copy_(S.Y[K:], non_blocking=True)
            o += K
            hout[o:o + a].copy_(S.node, non_blocking=True)
            o += a
            for r0, r1 in runs:
                hout[o:o + r1 - r0].copy_(S.data_out[r0:r1], non_blocking=True)
                o += r1 - r0
        ev_out[b].record(s_out)

    for i in range(max(2, args.warmup)):
        step(i)
    import gc

    import paper_1412_3022_gb300 as P
    P.wait_kernels()
    for i in range(2):              # both buffer sets load their kernels
        step(i)
    gc.collect()                    # no handle is freed inside the timed steps
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for i in range(args.steps):
        step(i)
    e1.record(s_out)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ranks_max(dist, e0.elapsed_time(e1) / args.steps, dev)
    user = sum(W.user.values())
    h2d, d2h = K * B, out_rows * B
    link = link_bandwidth(torch, dev)
    # the host link moves each step's inputs in and results out; with the
    # two directions fully overlapped the step cannot beat the slower one
    floor_ms = max(h2d / link["h2d_gbs"], d2h / link["d2h_gbs"]) / 1e6
    link["bound_gbs"] = round(whole_job_gbps(user, world, floor_ms), 2)
    link["frac"] = round(floor_ms / ms, 3)
    return {"value": round(whole_job_gbps(user, world, ms), 2), "unit": "GB/s",
            "ms_per_step": round(ms, 4), "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h,
            "pipeline": "2 buffer sets, 3 streams (H2D / compute / D2H)",
            "link": link}


def link_bandwidth(torch, dev, nbytes=256 << 20, reps=5):
    """Pinned host <-> device copy bandwidth of this machine's host link, each
    direction on its own (GB/s, median of `reps` timed copies of `nbytes`):
    the ceiling of the end-to-end number."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream(device=dev)
    out = {}
    for name, fn in (("h2d_gbs", lambda: d.copy_(h, non_blocking=True)),
                     ("d2h_gbs", lambda: h.copy_(d, non_blocking=True))):
        times = []
        with torch.cuda.stream(s):
            fn()
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(s)
                fn()
                e1.record(s)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        out[name] = round(nbytes / (sorted(times)[len(times) // 2] * 1e6), 1)
    s.synchronize()
    return out


# ------------------------------------------------------------------ oracle
def oracle_step(O, X, Y, f, H, S):
    """One pass of the four operations through the CPU oracle on column-sliced
    blocks X (data) and Y (stored codeword)."""
    a = A_
    O.encode(N_, K_, O.VANILLA, False, X)
    O.encode(N_, K_, O.SPARSE, True, X)
    sent = __import__("numpy").stack(
        [O.repair_helper(N_, K_, O.SPARSE, f, Y[a * h:a * h + a]) for h in H])
    O.repair_newcomer(N_, K_, O.SPARSE, f, H, sent)
    rows = [a * i + j for i in S for j in range(a)]
    O.decode(N_, K_, O.SPARSE, True, S, Y[rows])


def oracle_sample(cols, seed):
    import numpy as np

    import oracle as O
    from paper_1412_3022_gb300 import inputs
    X = inputs.blocks(K_ * A_, cols, seed)
    Y = O.encode(N_, K_, O.SPARSE, True, X)
    f = inputs.failed_node(N_, seed)
    S = inputs.node_subset(N_, K_, seed)
    # default helpers: the d lowest-index survivors if invertible, else the next set
    import itertools
    surv = [i for i in range(N_) if i != f]
    for H in itertools.combinations(surv, D_):
        try:
            O.newcomer_matrix(N_, K_, O.SPARSE, f, list(H))
            break
        except O.OracleError:
            continue
    del np
    return O, X, Y, f, list(H), S


def calibrate_cols(seconds, seed):
    cols = 4096
    O, X, Y, f, H, S = oracle_sample(cols, seed)
    t0 = time.perf_counter()
    oracle_step(O, X, Y, f, H, S)
    dt = time.perf_counter() - t0
    want = int(cols * seconds / max(dt, 1e-3))
    return max(4096, min(want // 4096 * 4096, 1 << 20))


def host_cores():
    """Threads this process may run on, and the host CPU's model name."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
            for ln in r.stdout.splitlines():
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return max(1, int(cores or 1)), model or "unknown"


def oracle_parallel_step(O, parts, pool):
    """One step of the oracle over column slices of the stripe, one slice per
    thread (the oracle's calls release the interpreter lock); returns the
    wall time."""
    t0 = time.perf_counter()
    list(pool.map(lambda pt: oracle_step(O, *pt), parts))
    return time.perf_counter() - t0


def oracle_parts(cols, threads, seed):
    """`threads` independent column slices of `cols` bytes each (the same
    code, failed node, helpers and node subset), for the all-cores oracle."""
    O, X, Y, f, H, S = oracle_sample(cols * threads, seed)
    parts = []
    for t in range(threads):
        cs = slice(t * cols, (t + 1) * cols)
        parts.append((np.ascontiguousarray(X[:, cs]), np.ascontiguousarray(Y[:, cs]), f, H, S))
    return O, parts


def cpu_baseline(args, W, torch):
    """The oracle on the host cores: one thread, and every core this process
    may use (a thread per column slice), on a bounded sample of the stripe."""
    import concurrent.futures as cf
    seed = args.seed
    cores, model = host_cores()
    cols = calibrate_cols(args.cpu_seconds / 2, seed)
    O, X, Y, f, H, S = oracle_sample(cols, seed)
    t0 = time.perf_counter()
    oracle_step(O, X, Y, f, H, S)
    dt1 = time.perf_counter() - t0
    user1 = (2 * K_ * A_ + A_ + K_ * A_) * cols
    one = {"value": round(user1 / dt1 / 1e9, 5), "seconds": round(dt1, 2), "cols": cols}
    O, parts = oracle_parts(cols, cores, seed)
    with cf.ThreadPoolExecutor(cores) as pool:
        dtn = oracle_parallel_step(O, parts, pool)
    usern = user1 * cores
    return {"value": round(usern / dtn / 1e9, 5), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "cpu_model": model, "seconds": round(dtn, 2),
            "sample": f"one step (all four operations) on {cores} column slices of {cols} bytes of "
                      f"the n=16 k=8 stripe (56 blocks each), plain C oracle, one thread per slice",
            "one_thread": one,
            "parallel_efficiency": round((usern / dtn) / (user1 / dt1) / cores, 3)}


def run_reference(args, rank):
    """The oracle as it stands on every host core this process may use, a
    bounded sample of the stripe per step."""
    if rank != 0:
        return None
    import concurrent.futures as cf
    cores, model = host_cores()
    # size each step so that warmup+steps stay within a few minutes
    budget = 150.0 / max(1, args.steps + args.warmup)
    cols = calibrate_cols(min(budget, args.ref_seconds), args.seed)
    O, parts = oracle_parts(cols, cores, args.seed)
    with cf.ThreadPoolExecutor(cores) as pool:
        for _ in range(args.warmup):
            oracle_parallel_step(O, parts, pool)
        times = [oracle_parallel_step(O, parts, pool) for _ in range(args.steps)]
    dt = sum(times) / len(times)
    user = (2 * K_ * A_ + A_ + K_ * A_) * cols * cores
    value = round(user / dt / 1e9, 5)
    sample = (f"each step: all four operations on {cores} column slices of {cols} bytes of the "
              f"n=16 k=8 stripe, plain C oracle, one thread per slice")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD + f" (oracle on {cores} x {cols}-byte column slices)",
                       "block_bytes": cols},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "cpu_model": model, "sample": sample},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank)
    else:
        out = run_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
