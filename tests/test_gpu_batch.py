"""Batched execution (one persistent launch from a CUDA graph): every
stripe's result equals its result alone (the single-stripe calls) and the
CPU oracle's, for a mix of codes, block sizes and operations."""
import numpy as np
import pytest

import oracle as O
import paper_1412_3022_gb300 as P
from paper_1412_3022_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def dev(arr):
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


class Mix:
    """A seeded mix of stripes with host copies of their inputs and the
    oracle's expected outputs."""

    def __init__(self, nstripes, seed, max_bytes=20000, ks=(4, 8, 16)):
        r = np.random.default_rng(seed)
        self.codes = {}
        self.stripes = []
        for s in range(nstripes):
            k = int(r.choice(ks))
            n, a = 2 * k, k - 1
            op = ["encode", "repair", "decode", "gen_encode"][s % 4] if k <= 8 else \
                ["encode", "repair", "decode"][s % 3]
            cons, form = (0, 0) if op == "gen_encode" else (1, 1)
            key = (n, k, cons, form)
            if key not in self.codes:
                self.codes[key] = P.Code(n, k, cons, form)
            c = self.codes[key]
            nb = int(r.integers(1, max_bytes))
            if s % 5 == 0:
                nb = (nb // 16) * 16 or 16
            X = inputs.blocks(k * a, nb, seed=seed * 1000 + s)
            st = {"op": op, "code": c, "n": n, "k": k, "a": a, "nb": nb, "cons": cons,
                  "form": form}
            if op in ("encode", "gen_encode"):
                st["in"] = dev(X)
                Y = O.encode(n, k, cons, bool(form), X)
                st["want"] = Y[k * a:] if form else Y
                st["out"] = torch.empty((len(st["want"]), nb), dtype=torch.uint8, device="cuda")
            elif op == "repair":
                Y = O.encode(n, k, 1, True, X)
                f = int(r.integers(0, n))
                st["f"], st["H"] = f, c.default_helpers(f)
                st["in"] = dev(Y)
                st["want"] = Y[a * f:a * f + a]
                st["out"] = torch.empty((a, nb), dtype=torch.uint8, device="cuda")
            else:
                Y = O.encode(n, k, 1, True, X)
                S = sorted(int(i) for i in r.choice(n, k, replace=False))
                rows = [a * i + j for i in S for j in range(a)]
                st["S"] = S
                st["in"] = dev(Y[rows])
                st["want"] = X
                st["out"] = torch.empty((k * a, nb), dtype=torch.uint8, device="cuda")
            self.stripes.append(st)

    def in_ptrs(self, st):
        t = st["in"]
        if st["op"] == "repair":
            a = st["a"]
            return [t[a * h + j] for h in st["H"] for j in range(a)]
        return [t[i] for i in range(t.shape[0])]

    def out_ptrs(self, st):
        return [st["out"][i] for i in range(st["out"].shape[0])]

    def add_to(self, batch):
        for st in self.stripes:
            c, nb = st["code"], st["nb"]
            if st["op"] in ("encode", "gen_encode"):
                batch.add_encode(c, self.in_ptrs(st), self.out_ptrs(st), nb)
            elif st["op"] == "repair":
                batch.add_repair(c, st["f"], st["H"], self.in_ptrs(st), self.out_ptrs(st), nb)
            else:
                batch.add_decode(c, st["S"], self.in_ptrs(st), self.out_ptrs(st), nb)

    def run_alone(self):
        for st in self.stripes:
            c, nb = st["code"], st["nb"]
            if st["op"] in ("encode", "gen_encode"):
                c.encode(self.in_ptrs(st), self.out_ptrs(st), nb)
            elif st["op"] == "repair":
                c.repair(st["f"], st["H"], self.in_ptrs(st), self.out_ptrs(st), nb)
            else:
                c.decode(st["S"], self.in_ptrs(st), self.out_ptrs(st), nb)

    def clear(self):
        for st in self.stripes:
            st["out"].fill_(0xA5)

    def check(self):
        torch.cuda.synchronize()
        for i, st in enumerate(self.stripes):
            got = st["out"].cpu().numpy()
            assert np.array_equal(got, st["want"]), (i, st["op"], st["k"], st["nb"])


def test_batch_matches_alone_and_oracle():
    mix = Mix(48, seed=1)
    mix.run_alone()
    mix.check()
    alone = [st["out"].clone() for st in mix.stripes]
    b = P.Batch()
    mix.add_to(b)
    b.build()
    info = b.info()
    assert info["stripes"] == 48 and info["items"] >= 48
    for _ in range(2):  # replays reuse the same graph
        mix.clear()
        b.launch()
        mix.check()
    for st, ref in zip(mix.stripes, alone):
        assert torch.equal(st["out"], ref)


@pytest.mark.parametrize("work_bytes,ctas", [(4096, 1), (16384, 2), (1 << 20, 1)])
def test_batch_item_sizes(work_bytes, ctas):
    mix = Mix(24, seed=work_bytes, max_bytes=70000)
    b = P.Batch()
    mix.add_to(b)
    b.build(work_bytes, ctas)
    mix.clear()
    b.launch()
    mix.check()


def test_batch_tune_keeps_results():
    mix = Mix(16, seed=7, max_bytes=40000)
    b = P.Batch()
    mix.add_to(b)
    best = b.tune()
    assert best[0] in (16 << 10, 64 << 10, 256 << 10) and best[1] in (1, 2)
    mix.clear()
    b.launch()
    mix.check()


def test_batch_rejects_adds_after_build_and_bad_args():
    mix = Mix(2, seed=3, max_bytes=100)
    b = P.Batch()
    mix.add_to(b)
    b.build()
    st = mix.stripes[0]
    with pytest.raises(P.PMRCError) as e:
        b.add_encode(st["code"], mix.in_ptrs(st), mix.out_ptrs(st), st["nb"])
    assert e.value.rc == P.PMRC_EBUSY
    b2 = P.Batch()
    with pytest.raises(P.PMRCError) as e:
        b2.build()
    assert e.value.rc == P.PMRC_EINVAL
    c = P.Code(8, 4, 1, 1)
    with pytest.raises(P.PMRCError) as e:
        b2.add_decode(c, [0, 1, 1, 2], [0] * 12, [0] * 12, 64)
    assert e.value.rc == P.PMRC_EINVAL


def test_batch_large_encodes_take_bitsliced_launches_with_ragged_tails():
    """Encodes of at least 4 MiB of data on codes with a built-in bitsliced
    kernel run as their own launches in the batch's graph (their last
    bytes, beyond a multiple of 32, with the persistent kernel); every
    stripe equals the oracle and the plain call, whatever mix of launches."""
    cases = [(8, 80000 + 16), (8, 80000 + 32), (4, 360000 + 16), (16, 20000 + 16), (12, 40000),
             (8, 4000)]                        # the last one stays in the persistent kernel
    stripes = []
    b = P.Batch()
    for s, (k, nb) in enumerate(cases):
        n, a = 2 * k, k - 1
        c = P.Code(n, k, 1, 1)
        X = inputs.blocks(k * a, nb, seed=900 + s)
        st = {"c": c, "k": k, "nb": nb, "X": X, "in": dev(X),
              "out": torch.full(((n - k) * a, nb), 0xA5, dtype=torch.uint8, device="cuda")}
        b.add_encode(c, [st["in"][i] for i in range(k * a)],
                     [st["out"][i] for i in range(st["out"].shape[0])], nb)
        stripes.append(st)
    b.build()
    info = b.info()
    assert info["stripes"] == len(cases) and info["bitsliced_launches"] == 5
    for _ in range(2):
        for st in stripes:
            st["out"].fill_(0xA5)
        b.launch()
        torch.cuda.synchronize()
        for st in stripes:
            k = st["k"]
            want = O.encode(2 * k, k, 1, True, st["X"])[k * (k - 1):]
            assert np.array_equal(st["out"].cpu().numpy(), want), (k, st["nb"])


def test_heavy_stripes_with_short_blocks_are_cut_into_one_tile_items():
    """A batch holding only a k=16 repair over 84 KiB + 5 byte blocks and a
    k=16 reconstruction over 61 KiB + 3 byte blocks: no item may cost more
    than a fixed share of the list, so both are cut into items of one or
    two tiles (1 KiB tiles for the repair, 4 KiB for the reconstruction's
    blocks of rows) instead of 13 items of up to 64 KiB; the results,
    ragged tails included, equal the oracle and the plain calls."""
    n, k = 32, 16
    a = k - 1
    c = P.Code(n, k, 1, 1)
    nr, nd = (84 << 10) + 5, (61 << 10) + 3
    Xr = inputs.blocks(k * a, nr, seed=77)
    Yr = O.encode(n, k, 1, True, Xr)
    f = 21
    H = c.default_helpers(f)
    rin = dev(np.concatenate([Yr[a * h:a * h + a] for h in H]))
    rout = torch.full((a, nr), 0xA5, dtype=torch.uint8, device="cuda")
    Xd = inputs.blocks(k * a, nd, seed=78)
    Yd = O.encode(n, k, 1, True, Xd)
    S = [1, 4, 5, 9, 11, 16, 17, 18, 20, 22, 23, 25, 27, 29, 30, 31]
    din = dev(Yd[[a * i + j for i in S for j in range(a)]])
    dout = torch.full((k * a, nd), 0xA5, dtype=torch.uint8, device="cuda")
    b = P.Batch()
    b.add_repair(c, f, H, [rin[i] for i in range(len(H) * a)], [rout[j] for j in range(a)], nr)
    b.add_decode(c, S, [din[i] for i in range(k * a)], [dout[r] for r in range(k * a)], nd)
    b.build(64 << 10, 2)
    info = b.info()
    repair_tiles = -(-nr // 1024)
    assert info["items"] >= repair_tiles + 16   # 64 KiB items: 2 for the repair, 11 row blocks
    b.launch()
    alone_r = torch.full_like(rout, 0x5A)
    alone_d = torch.full_like(dout, 0x5A)
    c.repair(f, H, [rin[i] for i in range(len(H) * a)], [alone_r[j] for j in range(a)], nr)
    c.decode(S, [din[i] for i in range(k * a)], [alone_d[r] for r in range(k * a)], nd)
    torch.cuda.synchronize()
    assert np.array_equal(rout.cpu().numpy(), Yr[a * f:a * f + a])
    assert np.array_equal(dout.cpu().numpy(), Xd)
    assert torch.equal(rout, alone_r) and torch.equal(dout, alone_d)
