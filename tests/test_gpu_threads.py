"""One code handle used from several host threads at once (each on its own
CUDA stream): the plan caches and the cache of kernels compiled at run time
are shared, so concurrent first uses of the same and of different failure
patterns must each get a correct plan.  Results are compared byte for byte
with the CPU oracle."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as O
import paper_1412_3022_gb300 as P
from paper_1412_3022_gb300 import inputs
from test_gpu_parity import Blocks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

N, K_, A = 16, 8, 7


def _setup(nbytes, seed):
    X = inputs.blocks(K_ * A, nbytes, seed=seed)
    Y = O.encode(N, K_, O.SPARSE, True, X)
    rng = np.random.default_rng(seed)
    subsets = [rng.permutation(rng.choice(N, K_, replace=False)).tolist() for _ in range(5)]
    return X, Y, subsets


def _run_threads(c, X, Y, subsets, nbytes, nthreads, iters):
    fails = [2, 9, 13]
    jobs = []
    for t in range(nthreads):   # buffers made on the main thread
        per = []
        for it in range(iters):
            S = subsets[(t + it) % len(subsets)]
            rows = [A * i + j for i in S for j in range(A)]
            f = fails[(t + it) % len(fails)]
            H = c.default_helpers(f)
            per.append(dict(
                S=S, yin=Blocks(K_ * A, nbytes, 0, Y[rows]), xout=Blocks(K_ * A, nbytes), f=f, H=H,
                hin=Blocks(len(H) * A, nbytes, 0, np.concatenate([Y[A * h:A * h + A] for h in H])),
                recv=Blocks(len(H), nbytes), node=Blocks(A, nbytes)))
        jobs.append(per)
    torch.cuda.synchronize()

    def worker(per):
        s = torch.cuda.Stream()
        for j in per:
            c.decode(j["S"], j["yin"].ptrs(), j["xout"].ptrs(), nbytes, s)
            c.repair_helpers(j["f"], j["H"], j["hin"].ptrs(), j["recv"].ptrs(), nbytes, s)
            c.repair_newcomer(j["f"], j["H"], j["recv"].ptrs(), j["node"].ptrs(), nbytes, s)
        s.synchronize()

    with ThreadPoolExecutor(nthreads) as ex:
        for fut in [ex.submit(worker, per) for per in jobs]:
            fut.result()
    torch.cuda.synchronize()
    for per in jobs:
        for j in per:
            assert np.array_equal(j["xout"].get(), X), j["S"]
            assert np.array_equal(j["node"].get(), Y[A * j["f"]:A * j["f"] + A]), j["f"]


def test_one_handle_many_threads_split_table():
    nbytes = 16 * 1024 + 5
    X, Y, subsets = _setup(nbytes, 95)
    c = P.Code(N, K_, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    _run_threads(c, X, Y, subsets, nbytes, nthreads=8, iters=6)


def test_one_handle_many_threads_runtime_kernels():
    """Reconstructions and newcomer applies through kernels compiled at run
    time: threads that first meet the same node set wait for one compile."""
    nbytes = 8 * 1024 + 32
    X, Y, subsets = _setup(nbytes, 96)
    c = P.Code(N, K_, P.PMRC_SPARSE, P.PMRC_SYSTEMATIC)
    c.set_decode_kernel(P.PMRC_KERNEL_BITSLICED)
    _run_threads(c, X, Y, subsets[:2], nbytes, nthreads=4, iters=2)
