"""Host-side units of the library built and run on the CPU: the split of a
bitsliced launch's (block, tile) work items into per-CTA ranges, checked on
20 000 random shapes (endpoints, order, and every CTA within one tile's cost
of an equal share); the bitsliced XOR schedules the emitter writes,
evaluated statement by statement on the CPU against the GF(2^8) matrix
product; and the on-disk cache of run-time compiled cubins (NVRTC runs on
the CPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1412_3022_gb300", "csrc")


def test_bitsliced_cta_ranges():
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not found")
    out_dir = os.path.join(ROOT, "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "test_cta_ranges")
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-I" + CSRC, "-o", exe,
                        os.path.join(ROOT, "tests", "host", "cta_ranges.cpp"),
                        os.path.join(CSRC, "bs_emit.cpp")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr


def _gf_mul(a, b):
    """GF(2^8) product by shift and reduce (modulus 0x11D)."""
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        if a & 0x100:
            a ^= 0x11D
        b >>= 1
    return r


def _evaluate_schedule(text, cols, X):
    """Runs the emitted XOR schedule on byte columns X (cols x T) the way
    the kernel does: per block (per half of its inputs when the block is
    split over a warp pair), per input, bit planes -> subset tables Q, R ->
    the case's accumulate statements; the halves' sums XORed; then planes
    back to bytes."""
    import re
    import numpy as np
    T = X.shape[1]
    planes = [((X >> j) & 1).astype(np.uint8) for j in range(8)]     # [j][col][t]
    inputs = {name: [int(v) for v in lst.split(",")] for name, lst in
              re.findall(r"(k_b\d+(?:_h[01])?)_in\[\d+\] = \{([^}]*)\};", text)}
    acc_of = {}
    for name, body in re.findall(r"void (k_b\d+(?:_h[01])?)\(.*?\{(.*?)\n\}\n", text, re.S):
        b = int(re.match(r"k_b(\d+)", name).group(1))
        acc = acc_of.setdefault(b, np.zeros((8, 8, T), np.uint8))
        for i, case in re.findall(r"case (\d+):(.*?)break;", body, re.S):
            col = inputs[name][int(i)]
            p = [planes[j][col] for j in range(8)]
            Q = [np.bitwise_xor.reduce([p[j] for j in range(4) if s >> j & 1] or [np.zeros(T, np.uint8)])
                 for s in range(16)]
            R = [np.bitwise_xor.reduce([p[4 + j] for j in range(4) if s >> j & 1] or [np.zeros(T, np.uint8)])
                 for s in range(16)]
            for q, bit, terms in re.findall(
                    r"acc\[(\d+)\]\[(\d+)\] = bs_x[23]\(acc\[\1\]\[\2\], ([^;]*)\);", case):
                for nm, idx in re.findall(r"([QR])\[(\d+)\]", terms):
                    acc[int(q), int(bit)] ^= (Q if nm == "Q" else R)[int(idx)]
    out = {}
    for b, acc in acc_of.items():
        kernel_case = re.search(r"case %d: \{\s*(?:if \(half == 0\) )?k_b%d(?:_h0)?\(x, acc\);(.*?)\} break;"
                                % (b, b), text, re.S)
        for slot, q in re.findall(r"bs_store(?:_planes)?\(x, (\d+), acc\[(\d+)\]\)", kernel_case.group(1)):
            row = int(slot) - cols
            out[row] = sum((acc[int(q), bit].astype(np.uint16) << bit) for bit in range(8)).astype(np.uint8)
    return out


@pytest.mark.parametrize("rows,cols,by_support,seed,pairs",
                         [(13, 9, 0, 1, 0), (21, 56, 0, 2, 0), (8, 3, 1, 3, 0), (30, 17, 1, 4, 0),
                          (1, 1, 0, 5, 0), (7, 64, 0, 6, 0), (21, 56, 0, 7, 1), (7, 14, 0, 8, 1),
                          (13, 9, 0, 9, 1), (1, 1, 0, 10, 1), (3, 2, 0, 11, 1)])
def test_bitsliced_schedule_computes_the_matrix(rows, cols, by_support, seed, pairs):
    """The emitter's XOR schedule (blocks, input lists, subset-table terms,
    output slots), evaluated on the CPU, equals the GF(2^8) matrix product
    computed with an independent multiply."""
    import numpy as np
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not found")
    exe = os.path.join(ROOT, "_build", "test_emit_dump")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-I" + CSRC, "-o", exe,
                        os.path.join(ROOT, "tests", "host", "emit_dump.cpp"),
                        os.path.join(CSRC, "bs_emit.cpp")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe, str(rows), str(cols), str(by_support), str(seed), str(pairs)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    head, code = r.stdout.split("CODE\n", 1)
    lines = head.strip().splitlines()
    M = np.array([[int(v) for v in ln.split()] for ln in lines[1:]], np.uint8)
    assert M.shape == (rows, cols)
    X = np.random.default_rng(seed).integers(0, 256, (cols, 64), dtype=np.uint8)
    got = _evaluate_schedule(code, cols, X)
    assert sorted(got) == list(range(rows))           # every row written once
    for row in range(rows):
        want = np.zeros(64, np.uint8)
        for c in range(cols):
            if M[row, c]:
                want ^= np.array([_gf_mul(int(M[row, c]), int(x)) for x in X[c]], np.uint8)
        assert np.array_equal(got[row], want), row


@pytest.mark.parametrize("m,shared,r,groups,seed,max_inputs",
                         [(21, 35, 21, 7, 1, 64), (7, 49, 7, 7, 2, 64), (14, 42, 10, 7, 3, 64),
                          (64, 20, 64, 8, 4, 64), (3, 5, 2, 1, 5, 64), (24, 10, 24, 3, 6, 64),
                          (20, 30, 20, 2, 7, 64), (30, 90, 30, 15, 8, 40)])
def test_factored_schedules_compose_to_w_times_z(m, shared, r, groups, seed, max_inputs):
    """The two launch schedules of a factored product x = W (Z y), the
    reconstruction of a systematic code (z: the received parity blocks plus
    their present-data terms; W = B^-1), evaluated on the CPU one after the
    other -- stage 1's plane-layout outputs are stage 2's plane-layout
    inputs -- equal W (Z X) computed with an independent multiply; stage 1
    keeps the rows of one shared support together (groups of at most 8 rows
    whole in one block, larger groups in blocks of their own) and packs
    several groups into a block only within the input budget."""
    import numpy as np
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not found")
    exe = os.path.join(ROOT, "_build", "test_emit_factored_dump")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    res = subprocess.run([cxx, "-std=c++17", "-O2", "-I" + CSRC, "-o", exe,
                          os.path.join(ROOT, "tests", "host", "emit_factored_dump.cpp"),
                          os.path.join(CSRC, "bs_emit.cpp")], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    res = subprocess.run([exe, str(m), str(shared), str(r), str(groups), str(seed), str(max_inputs)],
                         capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stderr
    head, rest = res.stdout.split("STAGE1\n", 1)
    stage1, stage2 = rest.split("STAGE2\n", 1)
    lines = head.strip().splitlines()
    cols = shared + m
    Z = np.array([[int(v) for v in ln.split()] for ln in lines[1:1 + m]], np.uint8)
    W = np.array([[int(v) for v in ln.split()] for ln in lines[2 + m:2 + m + r]], np.uint8)
    assert Z.shape == (m, cols) and W.shape == (r, m)
    tokens = lines[2 + m + r].split()[1:]
    blocks = [[int(v) for v in b.split("/")[0].split(",")] for b in tokens]
    ninputs = [int(b.split("/")[1]) for b in tokens]
    assert sorted(sum(blocks, [])) == list(range(m)) and max(len(b) for b in blocks) <= 8
    size = {g: sum(1 for i in range(m) if i % groups == g) for g in range(groups)}
    for g in range(groups):
        holding = [b for b in blocks if any(i % groups == g for i in b)]
        if size[g] <= 8:
            assert len(holding) == 1, (g, blocks)
    for b, ni in zip(blocks, ninputs):
        if len({i % groups for i in b}) > 1:
            assert ni <= max_inputs, (b, ni)
    X = np.random.default_rng(seed).integers(0, 256, (cols, 64), dtype=np.uint8)
    z = _evaluate_schedule(stage1, cols, X)
    assert sorted(z) == list(range(m))
    zb = np.stack([z[i] for i in range(m)])
    got = _evaluate_schedule(stage2, m, zb)
    assert sorted(got) == list(range(r))

    def apply(M, Y):
        out = np.zeros((M.shape[0], Y.shape[1]), np.uint8)
        for i in range(M.shape[0]):
            for c in range(M.shape[1]):
                if M[i, c]:
                    out[i] ^= np.array([_gf_mul(int(M[i, c]), int(v)) for v in Y[c]], np.uint8)
        return out

    want = apply(W, apply(Z, X))
    for i in range(r):
        assert np.array_equal(got[i], want[i]), i


@pytest.mark.parametrize("m,shared,groups,seed,max_inputs", [(21, 35, 7, 1, 64), (30, 90, 15, 8, 40),
                                                            (24, 10, 3, 6, 64), (64, 20, 8, 4, 64)])
def test_bench_models_the_library_blocks_of_the_factored_reconstruction(m, shared, groups, seed,
                                                                         max_inputs):
    """The benchmark's instruction model of the factored reconstruction
    (bench.factored_blocks) cuts the first launch's rows into the same
    blocks, with the same input counts, as the library's rule
    (bs_blocks_grouped), on the emitter's own dump."""
    import sys
    import numpy as np
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not found")
    sys.path.insert(0, ROOT)
    import bench
    exe = os.path.join(ROOT, "_build", "test_emit_factored_dump")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    res = subprocess.run([cxx, "-std=c++17", "-O2", "-I" + CSRC, "-o", exe,
                          os.path.join(ROOT, "tests", "host", "emit_factored_dump.cpp"),
                          os.path.join(CSRC, "bs_emit.cpp")], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    res = subprocess.run([exe, str(m), str(shared), str(m), str(groups), str(seed), str(max_inputs)],
                         capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stderr
    lines = res.stdout.split("STAGE1\n", 1)[0].strip().splitlines()
    Z = np.array([[int(v) for v in ln.split()] for ln in lines[1:1 + m]], np.uint8)
    tokens = lines[2 + 2 * m].split()[1:]
    lib = [(len(b.split("/")[0].split(",")), int(b.split("/")[1])) for b in tokens]
    own = [shared + i for i in range(m)]
    assert bench.factored_blocks(Z, own, max_inputs) == lib


def _run_statements(env, lines):
    """Executes emitted assignments (x = y; x = 0u; x = bs_x2(a, b);
    x = bs_x3(a, b, c);) on integer bit vectors."""
    import re
    for ln in lines:
        m = re.match(r"\s*([\w\[\]]+) = (.*);$", ln)
        if not m or "(" in m.group(1):
            continue
        lhs, rhs = m.groups()
        if rhs == "0u":
            env[lhs] = 0
        elif rhs.startswith("bs_x"):
            v = 0
            for name in rhs[rhs.index("(") + 1:-1].split(", "):
                v ^= env[name]
            env[lhs] = v
        elif re.fullmatch(r"[\w\[\]]+", rhs):
            env[lhs] = env[rhs]


def _planes(block):
    """Bit planes of a byte block as integers (bit t = bit j of byte t)."""
    return [sum(((int(x) >> j) & 1) << t for t, x in enumerate(block)) for j in range(8)]


def _bytes(planes, T):
    import numpy as np
    return np.array([sum(((planes[i] >> t) & 1) << i for i in range(8)) for t in range(T)], np.uint8)


def _helper_sections(body):
    """Splits a helper-loop body into the per-input sections (each starts at
    bs_load) and the statements after the last one (the epilogue)."""
    secs, cur, pre = [], None, []
    for ln in body.splitlines():
        if "bs_load(rd, w)" in ln:
            cur = []
            secs.append(cur)
        elif cur is not None:
            cur.append(ln)
        else:
            pre.append(ln)
    return secs


@pytest.mark.parametrize("alpha,d,seed,zeros,single", [(7, 14, 1, 1, None), (7, 14, 2, 0, None),
                                                        (3, 4, 3, 1, None), (8, 16, 4, 1, None),
                                                        (7, 14, 5, 0, 3), (1, 8, 6, 0, None),
                                                        (2, 5, 7, 1, None)])
def test_repair_schedules_compute_projection_and_newcomer(alpha, d, seed, zeros, single):
    """The run-time repair schedules, evaluated on the CPU: the projection
    kernel's helper loop gives sum_j phi[j] Y_hj, and the fused kernel's two
    helper groups, tables and per-helper newcomer terms give D applied to the
    projections (independent GF(2^8) multiply)."""
    import re
    import numpy as np
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not found")
    exe = os.path.join(ROOT, "_build", "test_emit_repair_dump")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-I" + CSRC, "-o", exe,
                        os.path.join(ROOT, "tests", "host", "emit_repair_dump.cpp"),
                        os.path.join(CSRC, "bs_emit.cpp")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    args = [exe, str(alpha), str(d), str(seed), str(zeros)] + ([str(single)] if single is not None else [])
    out = subprocess.run(args, capture_output=True, text=True, timeout=60).stdout
    head, rest = out.split("PROJ\n", 1)
    proj, fused = rest.split("FUSED\n", 1)
    lines = head.strip().splitlines()
    phi = [int(v) for v in lines[0].split()[1:]]
    D = np.array([[int(v) for v in ln.split()] for ln in lines[2:2 + alpha]], np.uint8)
    nz = [j for j in range(alpha) if phi[j]]
    T = 48
    Y = np.random.default_rng(seed).integers(0, 256, (d, alpha, T), dtype=np.uint8)

    def gfvec(c, v):
        return np.array([_gf_mul(int(c), int(x)) for x in v], np.uint8)

    want_p = []
    for h in range(d):
        acc = np.zeros(T, np.uint8)
        for j in nz:
            acc ^= gfvec(phi[j], Y[h, j])
        want_p.append(acc)

    def projection_of(body, h):
        env = {}
        for jj, sec in enumerate(_helper_sections(body)):
            for i, pl in enumerate(_planes(Y[h, nz[jj]])):
                env["w[%d]" % i] = pl
            _run_statements(env, sec)
        return env

    # projection kernel: one loop body, run per helper
    body = proj[proj.index("for (uint32_t h = h0; h < h1; h++) {"):]
    assert len(_helper_sections(body)) == len(nz)
    for h in range(d):
        env = projection_of(body, h)
        assert np.array_equal(_bytes([env["p[%d]" % i] for i in range(8)], T), want_p[h]), h
    # fused kernel: both helper groups, tables of the projection, D terms
    acc = {}
    for g in (0, 1):
        fn = fused[fused.index("void kf_g%d(" % g):]
        fn = fn[:fn.index("\n}\n")]
        h0, h1 = map(int, re.search(r"for \(uint32_t h = (\d+); h < (\d+); h\+\+\)", fn).groups())
        loop = fn[fn.index("h++) {"):]
        head_part, cases = loop.split("bs_tables(p, Q, R);", 1)
        for h in range(h0, h1):
            env = projection_of(head_part, h)
            p = [env["p[%d]" % i] for i in range(8)]
            for s in range(16):
                env["Q[%d]" % s] = 0
                env["R[%d]" % s] = 0
                for i in range(4):
                    if s >> i & 1:
                        env["Q[%d]" % s] ^= p[i]
                        env["R[%d]" % s] ^= p[4 + i]
            for key, v in acc.items():
                env[key] = v
            for r_ in range(alpha):
                for i in range(8):
                    env.setdefault("acc[%d][%d]" % (r_, i), 0)
            m = re.search(r"case %d:(.*?)break;" % h, cases, re.S)
            _run_statements(env, m.group(1).splitlines() if m else [])
            acc = {k: v for k, v in env.items() if k.startswith("acc[")}
    for r_ in range(alpha):
        want = np.zeros(T, np.uint8)
        for q in range(d):
            want ^= gfvec(D[r_, q], want_p[q])
        got = _bytes([acc.get("acc[%d][%d]" % (r_, i), 0) for i in range(8)], T)
        assert np.array_equal(got, want), r_


def test_kernel_cache_on_disk():
    """jit_compile with PMRC_KERNEL_CACHE: the first compilation writes one
    cubin file (an ELF image, no temporary left), later ones read it back
    unchanged; a damaged file is ignored and replaced."""
    cxx = shutil.which("g++")
    cuda = "/usr/local/cuda"
    if not cxx or not os.path.exists(os.path.join(cuda, "include", "nvrtc.h")):
        pytest.skip("g++ or the CUDA headers not found")
    build = os.path.join(ROOT, "_build")
    exe = os.path.join(build, "test_jit_cache")
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-I" + CSRC, "-I" + os.path.join(cuda, "include"),
                        "-o", exe, os.path.join(ROOT, "tests", "host", "jit_cache.cpp"),
                        os.path.join(CSRC, "jit.cpp"), "-L" + os.path.join(cuda, "lib64"),
                        "-lcudart", "-ldl", "-lpthread"], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("cannot build against the CUDA runtime here: " + r.stderr[-200:])
    cache = os.path.join(build, "test_kernel_cache")
    shutil.rmtree(cache, ignore_errors=True)
    os.makedirs(cache)
    env = dict(os.environ, PMRC_KERNEL_CACHE=cache,
               LD_LIBRARY_PATH=os.path.join(cuda, "lib64") + ":" + os.environ.get("LD_LIBRARY_PATH", ""))

    def run():
        p = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
        assert p.returncode == 0, p.stdout + p.stderr
        return p.stdout.strip()

    first = run()
    if first == "nonvrtc":
        pytest.skip("NVRTC is not available")
    assert first.startswith("ok")
    files = sorted(os.listdir(cache))
    assert len(files) == 1 and files[0].startswith("pmrc-") and files[0].endswith(".cubin"), files
    path = os.path.join(cache, files[0])
    with open(path, "rb") as f:
        image = f.read()
    assert image[:4] == b"\x7fELF"
    assert run() == first and sorted(os.listdir(cache)) == files
    with open(path, "wb") as f:                      # damaged: not a cubin
        f.write(b"garbage")
    assert run() == first
    with open(path, "rb") as f:
        assert f.read() == image                     # replaced by a fresh compilation
    shutil.rmtree(cache)


def test_kernel_cache_default_directory_and_off():
    """Without PMRC_KERNEL_CACHE the cubins go to $XDG_CACHE_HOME/pmrc
    (created); PMRC_KERNEL_CACHE=off writes nothing."""
    cxx = shutil.which("g++")
    cuda = "/usr/local/cuda"
    if not cxx or not os.path.exists(os.path.join(cuda, "include", "nvrtc.h")):
        pytest.skip("g++ or the CUDA headers not found")
    build = os.path.join(ROOT, "_build")
    exe = os.path.join(build, "test_jit_cache")
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-I" + CSRC, "-I" + os.path.join(cuda, "include"),
                        "-o", exe, os.path.join(ROOT, "tests", "host", "jit_cache.cpp"),
                        os.path.join(CSRC, "jit.cpp"), "-L" + os.path.join(cuda, "lib64"),
                        "-lcudart", "-ldl", "-lpthread"], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("cannot build against the CUDA runtime here: " + r.stderr[-200:])
    base = os.path.join(build, "test_kernel_cache_xdg")
    shutil.rmtree(base, ignore_errors=True)
    os.makedirs(base)
    env = {k: v for k, v in os.environ.items() if k != "PMRC_KERNEL_CACHE"}
    env.update(XDG_CACHE_HOME=base,
               LD_LIBRARY_PATH=os.path.join(cuda, "lib64") + ":" + os.environ.get("LD_LIBRARY_PATH", ""))
    p = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert p.returncode == 0, p.stdout + p.stderr
    if p.stdout.strip() == "nonvrtc":
        pytest.skip("NVRTC is not available")
    files = os.listdir(os.path.join(base, "pmrc"))
    assert len(files) == 1 and files[0].endswith(".cubin")
    assert oct(os.stat(os.path.join(base, "pmrc")).st_mode & 0o777) == oct(0o700)
    shutil.rmtree(base)
    os.makedirs(base)
    env["PMRC_KERNEL_CACHE"] = "off"
    p = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert p.returncode == 0 and p.stdout.startswith("ok"), p.stdout + p.stderr
    assert os.listdir(base) == []
    shutil.rmtree(base)
