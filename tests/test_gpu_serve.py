"""Serving loop (continuous batching): each request's result is the same
alone (the single-stripe calls) and in the mix (submitted in bursts while
other requests are copying or computing), and equals the CPU oracle's.
Admission respects the HBM budget; bad requests are refused at submit;
queued requests can be withdrawn; waits are bounded."""
import threading
import time

import numpy as np
import pytest

import oracle as O
import paper_1412_3022_gb300 as P
from paper_1412_3022_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def pinned(arr):
    t = torch.from_numpy(np.ascontiguousarray(arr)).pin_memory()
    return t


class Workload:
    def __init__(self, count, seed, ks=(4, 8, 12, 16), max_stripe=300_000):
        r = np.random.default_rng(seed)
        self.codes = {k: P.Code(2 * k, k, 1, 1) for k in ks}
        self.reqs = []
        for i in range(count):
            k = int(r.choice(ks))
            n, a, d = 2 * k, k - 1, 2 * k - 2
            c = self.codes[k]
            stripe = int(r.integers(1000, max_stripe))
            B = -(-stripe // (k * a))
            B = -(-B // 16) * 16 if i % 3 else B          # some ragged block sizes
            X = inputs.blocks(k * a, B, seed=seed * 1000 + i)
            op = ("encode", "repair", "decode")[i % 3]
            q = {"op": op, "k": k, "code": c, "B": B}
            if op == "encode":
                q["in"] = pinned(X)
                q["want"] = O.encode(n, k, 1, True, X)[k * a:]
            else:
                Y = O.encode(n, k, 1, True, X)
                if op == "repair":
                    f = int(r.integers(0, n))
                    H = c.default_helpers(f)
                    q.update(f=f, H=H)
                    q["in"] = pinned(np.concatenate([Y[a * h:a * h + a] for h in H]))
                    q["want"] = Y[a * f:a * f + a]
                else:
                    S = sorted(int(x) for x in r.choice(n, k, replace=False))
                    q["S"] = S
                    q["in"] = pinned(Y[[a * s + j for s in S for j in range(a)]])
                    q["want"] = X
            q["out"] = torch.full(q["want"].shape, 0xA5, dtype=torch.uint8).pin_memory()
            self.reqs.append(q)

    @staticmethod
    def submit(server, q):
        op = {"encode": P.PMRC_OP_ENCODE, "repair": P.PMRC_OP_REPAIR,
              "decode": P.PMRC_OP_DECODE}[q["op"]]
        return server.submit(op, q["code"], q["B"], q["in"], q["out"], failed=q.get("f", -1),
                             helpers=q.get("H"), nodes=q.get("S"))

    @staticmethod
    def alone(q):
        """The same operation through the single-stripe calls."""
        c, B = q["code"], q["B"]
        x = q["in"].cuda()
        a = c.alpha
        y = torch.empty(q["want"].shape, dtype=torch.uint8, device="cuda")
        xs = [x[i] for i in range(x.shape[0])]
        ys = [y[i] for i in range(y.shape[0])]
        if q["op"] == "encode":
            c.encode(xs, ys, B)
        elif q["op"] == "repair":
            c.repair(q["f"], q["H"], xs, ys, B)
        else:
            c.decode(q["S"], xs, ys, B)
        torch.cuda.synchronize()
        return y.cpu().numpy()


def test_serving_results_same_alone_and_in_the_mix():
    w = Workload(48, seed=21)
    srv = P.Server(budget_bytes=64 << 20, max_slots=16)
    ids = []

    def client():  # bursts of submissions while earlier requests run
        for i, q in enumerate(w.reqs):
            ids.append(Workload.submit(srv, q))
            if i % 6 == 5:
                time.sleep(0.002)

    t = threading.Thread(target=client)
    t.start()
    t.join()
    for rid in ids:
        st, lat = srv.wait(rid, timeout_ms=30000)
        assert st == P.PMRC_OK and lat >= 0
    stats = srv.stats()
    assert stats["completed"] == 48 and stats["failed"] == 0
    assert stats["peak_bytes"] <= stats["budget_bytes"]
    assert stats["iterations"] < 48      # requests shared launches
    for q in w.reqs:
        got = q["out"].numpy()
        assert np.array_equal(got, q["want"]), (q["op"], q["k"], q["B"])
        assert np.array_equal(got, Workload.alone(q)), (q["op"], q["k"], q["B"])
    srv.close()


def test_serving_admission_respects_budget():
    w = Workload(12, seed=22, ks=(8,), max_stripe=2_000_000)
    need = max(q["in"].numel() + q["out"].numel() + 512 for q in w.reqs)
    srv = P.Server(budget_bytes=need, max_slots=8)   # room for about one request at a time
    ids = [Workload.submit(srv, q) for q in w.reqs]
    for rid in ids:
        assert srv.wait(rid, timeout_ms=30000)[0] == P.PMRC_OK
    st = srv.stats()
    assert st["completed"] == 12 and st["peak_bytes"] <= need
    for q in w.reqs:
        assert np.array_equal(q["out"].numpy(), q["want"])
    srv.close()


def test_serving_refuses_bad_requests_and_cancels_queued():
    c = P.Code(16, 8, 1, 1)
    B = 1 << 20
    big_in = torch.zeros((56, B), dtype=torch.uint8).pin_memory()
    big_out = torch.zeros((56, B), dtype=torch.uint8).pin_memory()
    srv = P.Server(budget_bytes=2 * 56 * B + 4096, max_slots=4)
    with pytest.raises(P.PMRCError) as e:          # cannot fit even alone
        srv.submit(P.PMRC_OP_ENCODE, c, 2 * B, big_in, big_out)
    assert e.value.rc == P.PMRC_ENOMEM
    with pytest.raises(P.PMRCError) as e:          # singular helper set at n = 2k
        srv.submit(P.PMRC_OP_REPAIR, c, 1024, big_in, big_out, failed=0,
                   helpers=list(range(2, 16)))
    assert e.value.rc == P.PMRC_ESINGULAR
    with pytest.raises(P.PMRCError) as e:
        srv.submit(P.PMRC_OP_DECODE, c, 1024, big_in, big_out, nodes=[0, 1, 2, 3, 4, 5, 6, 6])
    assert e.value.rc == P.PMRC_EINVAL
    # the first request takes the whole budget, so the second stays queued
    a = srv.submit(P.PMRC_OP_ENCODE, c, B, big_in, big_out)
    b = srv.submit(P.PMRC_OP_ENCODE, c, B, big_in, big_out)
    with pytest.raises(P.PMRCError) as e:
        srv.wait(a, timeout_ms=0)
    assert e.value.rc == P.PMRC_ETIMEOUT
    srv.cancel(b)
    assert srv.wait(a, timeout_ms=30000)[0] == P.PMRC_OK
    st, _ = srv.wait(b, timeout_ms=0)
    assert st == P.PMRC_EBUSY                       # cancelled before admission
    srv.close()


def test_serving_many_small_requests_all_complete():
    """Hundreds of tiny requests finish within microseconds of each other,
    so output copies often complete while their iteration is still being
    retired; every request must still be retired exactly once."""
    c = P.Code(8, 4, 1, 1)
    B = 256
    X = inputs.blocks(12, B, seed=5)
    want = O.encode(8, 4, 1, True, X)[12:]
    xin = pinned(X)
    outs = [torch.zeros((12, B), dtype=torch.uint8).pin_memory() for _ in range(300)]
    srv = P.Server(budget_bytes=8 << 20, max_slots=32)
    ids = [srv.submit(P.PMRC_OP_ENCODE, c, B, xin, o) for o in outs]
    for rid in ids:
        assert srv.wait(rid, timeout_ms=20000)[0] == P.PMRC_OK
    assert srv.stats()["completed"] == 300
    for o in outs:
        assert np.array_equal(o.numpy(), want)
    srv.close()


def test_serving_device_resident_requests_in_place():
    """Requests whose blocks already live in device memory (PMRC_REQ_DEVICE):
    no arena space and no copies; results equal the oracle's and the host
    requests' in the same mix."""
    w = Workload(24, seed=23, max_stripe=400_000)
    for q in w.reqs:                 # device-resident blocks need 16-byte sizes
        if q["B"] % 16:
            q["skip"] = True
    srv = P.Server(budget_bytes=64 << 20, max_slots=16)
    ids, dev = [], []
    for q in w.reqs:
        if q.get("skip"):
            continue
        din = q["in"].cuda()
        dout = torch.full(q["want"].shape, 0xA5, dtype=torch.uint8, device="cuda")
        op = {"encode": P.PMRC_OP_ENCODE, "repair": P.PMRC_OP_REPAIR,
              "decode": P.PMRC_OP_DECODE}[q["op"]]
        ids.append(srv.submit(op | P.PMRC_REQ_DEVICE, q["code"], q["B"], din, dout,
                              failed=q.get("f", -1), helpers=q.get("H"), nodes=q.get("S")))
        dev.append((q, din, dout))
        ids.append(Workload.submit(srv, q))           # the same request from host buffers
    for rid in ids:
        st, lat = srv.wait(rid, timeout_ms=30000)
        assert st == P.PMRC_OK and lat >= 0
    assert srv.stats()["peak_bytes"] <= srv.stats()["budget_bytes"]
    torch.cuda.synchronize()
    for q, din, dout in dev:
        assert np.array_equal(dout.cpu().numpy(), q["want"]), (q["op"], q["k"], q["B"])
        assert np.array_equal(q["out"].numpy(), q["want"]), (q["op"], q["k"], q["B"])
    with pytest.raises(P.PMRCError) as e:            # misaligned device blocks are refused
        q, din, dout = dev[0]
        srv.submit(P.PMRC_OP_ENCODE | P.PMRC_REQ_DEVICE, q["code"], q["B"], din.data_ptr() + 1,
                   dout)
    assert e.value.rc == P.PMRC_EINVAL
    srv.close()
