"""Parity at the stated sizes of the benchmarked workloads: every output byte
of the CUDA path, called through the C ABI, against the CPU oracle.

* n=16, k=8, 56 data blocks of 1 MiB: generator and sparse systematic
  encodes (and the other two construction/form pairs) on every column;
* n=16, k=8 repair of a seeded failed node (two-step and fused) and
  reconstruction from a seeded 8-node subset, 64 KiB to 4 MiB blocks, on
  every column;
* the batched mix at its real distribution (k uniform on {4, 8, 16}, blocks
  log-uniform on [4 KiB, 1 MiB], half encodes and half repairs), every
  stripe of a 256-stripe batch run in one persistent launch;
* the serving loop with stripes from 64 KiB up to 64 MiB.

Integer work, so the bar is bit-exact equality.  Every operation is
independent per byte column (Y[r][t] = sum_c M[r][c] X[c][t], Sec. 2), so
the oracle runs on column slices on host threads (its ctypes calls release
the interpreter lock) and the slices are stitched back together.  Inputs of
the repairs in the batch are seeded random helper blocks: the repair is a
linear map of the blocks it reads, and the oracle applies the same map
(helper projections, then the newcomer matrix) to the same bytes."""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle as O
import paper_1412_3022_gb300 as P
from oracle_columns import THREADS, oracle_columns
from paper_1412_3022_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def oracle_encode_rows(n, k, cons, form, X):
    Y = O.encode(n, k, cons, bool(form), X)
    return Y[k * (k - 1):] if form else Y


# ---------------------------------------------------------- n=16 k=8, 1 MiB
@pytest.mark.parametrize("cons,form", [(1, 1), (0, 0), (0, 1), (1, 0)])
def test_k8_1mib_encode_every_column(cons, form):
    """The 56 MiB stripe: every byte of every output block."""
    n, k, a = 16, 8, 7
    nbytes = 1 << 20
    c = P.Code(n, k, cons, form)
    X = inputs.device_blocks(k * a, nbytes, seed=2024 + 10 * cons + form)
    Y = torch.full((c.n_outputs, nbytes), 0xA5, dtype=torch.uint8, device="cuda")
    c.encode([X[i] for i in range(k * a)], [Y[i] for i in range(c.n_outputs)], nbytes)
    torch.cuda.synchronize()
    want = oracle_columns(lambda x: oracle_encode_rows(n, k, cons, form, x), [X.cpu().numpy()])
    assert np.array_equal(Y.cpu().numpy(), want)


# ------------------------------------------- n=16 k=8 repair / reconstruction
@pytest.mark.parametrize("nbytes", [64 << 10, 256 << 10, 1 << 20, 4 << 20])
def test_k8_repair_and_decode_every_column(nbytes):
    """Sparse systematic code: the failed node and the node subset are drawn
    from the block size as seed; the codeword comes from the oracle."""
    n, k, a = 16, 8, 7
    c = P.Code(n, k, 1, 1)
    X = inputs.blocks(k * a, nbytes, seed=nbytes + 1)
    Yh = oracle_columns(lambda x: O.encode(n, k, 1, True, x), [X])
    Y = torch.from_numpy(Yh).cuda()
    f = inputs.failed_node(n, seed=nbytes)
    H = c.default_helpers(f)
    hb = [Y[a * h + j] for h in H for j in range(a)]
    recv = torch.empty((len(H), nbytes), dtype=torch.uint8, device="cuda")
    c.repair_helpers(f, H, hb, [recv[i] for i in range(len(H))], nbytes)
    node = torch.full((a, nbytes), 0xA5, dtype=torch.uint8, device="cuda")
    c.repair_newcomer(f, H, [recv[i] for i in range(len(H))], [node[j] for j in range(a)], nbytes)
    fused = torch.full((a, nbytes), 0xA5, dtype=torch.uint8, device="cuda")
    c.repair(f, H, hb, [fused[j] for j in range(a)], nbytes)
    S = inputs.node_subset(n, k, seed=nbytes)
    rows = [a * i + j for i in S for j in range(a)]
    Xd = torch.full((k * a, nbytes), 0xA5, dtype=torch.uint8, device="cuda")
    c.decode(S, [Y[r] for r in rows], [Xd[r] for r in range(k * a)], nbytes)
    torch.cuda.synchronize()

    helper_in = np.concatenate([Yh[a * h:a * h + a] for h in H])

    def sent_fn(x):
        return np.stack([O.repair_helper(n, k, 1, f, x[a * i:a * i + a]) for i in range(len(H))])

    sent = oracle_columns(sent_fn, [helper_in])
    assert np.array_equal(recv.cpu().numpy(), sent)
    want_node = oracle_columns(lambda p: O.repair_newcomer(n, k, 1, f, H, p), [sent])
    assert np.array_equal(want_node, Yh[a * f:a * f + a])  # the oracle's own repair is exact
    assert np.array_equal(node.cpu().numpy(), want_node)
    assert np.array_equal(fused.cpu().numpy(), want_node)
    want_x = oracle_columns(lambda y: O.decode(n, k, 1, True, S, y), [Yh[rows]])
    assert np.array_equal(want_x, X)
    assert np.array_equal(Xd.cpu().numpy(), want_x)


# ------------------------------------------------------------ batched mix
def test_batched_mix_every_stripe_at_the_stated_distribution():
    """256 stripes drawn like the 4096-stripe benchmark mix, one persistent
    launch; each stripe's outputs equal the oracle's on every column and the
    same stripe run through the plain calls."""
    mix = inputs.batch_mix(256, seed=4)
    codes = {}
    stripes = []
    for s, m in enumerate(mix):
        k, nb = m["k"], m["block_bytes"]
        n, a, d = 2 * k, k - 1, 2 * k - 2
        c = codes.setdefault(k, P.Code(n, k, 1, 1))
        seed = 40_000 + s
        if m["op"] == "encode":
            X = inputs.blocks(k * a, nb, seed=seed)
            st = {"op": "encode", "k": k, "nb": nb, "seed": seed, "c": c,
                  "in": torch.from_numpy(X).cuda(),
                  "out": torch.full(((n - k) * a, nb), 0xA5, dtype=torch.uint8, device="cuda")}
        else:
            f = m["failed"]
            H = c.default_helpers(f)
            B = inputs.blocks(d * a, nb, seed=seed)   # helper i's alpha blocks, i in list order
            st = {"op": "repair", "k": k, "nb": nb, "seed": seed, "c": c, "f": f, "H": H,
                  "in": torch.from_numpy(B).cuda(),
                  "out": torch.full((a, nb), 0xA5, dtype=torch.uint8, device="cuda")}
        stripes.append(st)

    def ins(st):
        return [st["in"][i] for i in range(st["in"].shape[0])]

    def outs(st, t=None):
        t = st["out"] if t is None else t
        return [t[i] for i in range(t.shape[0])]

    b = P.Batch()
    for st in stripes:
        if st["op"] == "encode":
            b.add_encode(st["c"], ins(st), outs(st), st["nb"])
        else:
            b.add_repair(st["c"], st["f"], st["H"], ins(st), outs(st), st["nb"])
    b.build()
    assert b.info()["bitsliced_launches"] > 0   # the large encodes run as bitsliced launches
    b.launch()
    alone = []
    for st in stripes:
        t = torch.full_like(st["out"], 0x5A)
        if st["op"] == "encode":
            st["c"].encode(ins(st), outs(st, t), st["nb"])
        else:
            st["c"].repair(st["f"], st["H"], ins(st), outs(st, t), st["nb"])
        alone.append(t)
    torch.cuda.synchronize()
    for st, t in zip(stripes, alone):
        assert torch.equal(st["out"], t), (st["op"], st["k"], st["nb"])

    def expect(st):
        k, nb = st["k"], st["nb"]
        n, a, d = 2 * k, k - 1, 2 * k - 2
        if st["op"] == "encode":
            X = inputs.blocks(k * a, nb, seed=st["seed"])
            return O.encode(n, k, 1, True, X)[k * a:]
        B = inputs.blocks(d * a, nb, seed=st["seed"])
        sent = np.stack([O.repair_helper(n, k, 1, st["f"], B[a * i:a * i + a]) for i in range(d)])
        return O.repair_newcomer(n, k, 1, st["f"], st["H"], sent)

    order = sorted(range(len(stripes)), key=lambda i: -stripes[i]["nb"] * stripes[i]["k"] ** 2)
    expect(stripes[order[-1]])  # field tables initialized on this thread
    with cf.ThreadPoolExecutor(THREADS) as ex:
        wants = dict(zip(order, ex.map(lambda i: expect(stripes[i]), order)))
    ops = {"encode": 0, "repair": 0}
    for i, st in enumerate(stripes):
        assert np.array_equal(st["out"].cpu().numpy(), wants[i]), (i, st["op"], st["k"], st["nb"])
        ops[st["op"]] += 1
    assert min(ops.values()) > 64 and {st["k"] for st in stripes} == {4, 8, 16}
    assert max(st["nb"] for st in stripes) > 512 << 10 and min(st["nb"] for st in stripes) < 8 << 10


# ------------------------------------------------------------ serving, large stripes
def test_serving_stripes_up_to_64mib():
    """Encode, repair and reconstruction requests whose stripes span the
    serving workload's range (64 KiB to 64 MiB), served together; every
    result equals the oracle's."""
    plan = [(4, "encode", 64 << 10), (16, "encode", 64 << 20), (8, "repair", 16 << 20),
            (12, "decode", 24 << 20), (16, "repair", 40 << 20), (8, "encode", 3 << 20),
            (12, "encode", 48 << 20), (4, "decode", 300 << 10), (16, "decode", 20 << 20)]
    codes = {}
    reqs = []
    for i, (k, op, stripe) in enumerate(plan):
        n, a = 2 * k, k - 1
        c = codes.setdefault(k, P.Code(n, k, 1, 1))
        B = -(-stripe // (k * a))
        B = -(-B // 16) * 16
        X = inputs.blocks(k * a, B, seed=500 + i)
        q = {"op": op, "k": k, "c": c, "B": B}
        if op == "encode":
            q["in"] = X
            q["want"] = oracle_columns(lambda x: O.encode(n, k, 1, True, x)[k * a:], [X])
        else:
            Y = oracle_columns(lambda x: O.encode(n, k, 1, True, x), [X])
            if op == "repair":
                f = inputs.failed_node(n, seed=i)
                H = c.default_helpers(f)
                q.update(f=f, H=H)
                q["in"] = np.concatenate([Y[a * h:a * h + a] for h in H])
                q["want"] = Y[a * f:a * f + a]
            else:
                S = inputs.node_subset(n, k, seed=i)
                q["S"] = S
                q["in"] = Y[[a * s + j for s in S for j in range(a)]]
                q["want"] = X
        q["in"] = torch.from_numpy(np.ascontiguousarray(q["in"])).pin_memory()
        q["out"] = torch.full(q["want"].shape, 0xA5, dtype=torch.uint8).pin_memory()
        reqs.append(q)
    srv = P.Server(budget_bytes=2 << 30, max_slots=16)
    opc = {"encode": P.PMRC_OP_ENCODE, "repair": P.PMRC_OP_REPAIR, "decode": P.PMRC_OP_DECODE}
    ids = [srv.submit(opc[q["op"]], q["c"], q["B"], q["in"], q["out"], failed=q.get("f", -1),
                      helpers=q.get("H"), nodes=q.get("S")) for q in reqs]
    for rid in ids:
        st, lat = srv.wait(rid, timeout_ms=120000)
        assert st == P.PMRC_OK and lat >= 0
    stats = srv.stats()
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["peak_bytes"] <= stats["budget_bytes"]
    for q in reqs:
        assert np.array_equal(q["out"].numpy(), q["want"]), (q["op"], q["k"], q["B"])
    srv.close()
