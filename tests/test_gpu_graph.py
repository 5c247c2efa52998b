"""GPU parity of CUDA-graph replays (the batched launch form of Sec. III-B,
captured once and replayed): the uniform forward and inverse transforms as
the benchmark captures them, the single-launch mixed-degree plan, and a
MulLinRS batch. Each graph is replayed on new contents of the same device
buffers, and every replay is checked against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2109_14704_gb300 import he
from paper_2109_14704_gb300.synth import Rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tests.gpu_util import host  # noqa: E402


def empty(*shape):
    # zero-filled: the warm-up call before each capture runs on these buffers
    return torch.zeros(shape, dtype=torch.int64, device="cuda")


def _load(t, a):
    t.copy_(torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)))


def _capture(fn):
    """Capture fn(stream) into a graph on a side stream (as the benchmark
    does), after one eager warm-up call."""
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn(side)
        with torch.cuda.graph(g, stream=side):
            fn(side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    return g


@pytest.mark.parametrize("N,limbs,count", [(32768, 8, 6), (4096, 2, 3), (65536, 3, 2)])
def test_uniform_graph_replay(N, limbs, count):
    qs = he.primes_generate(60, 2 * N, limbs // 2 + limbs % 2) + he.primes_generate(50, 2 * N, limbs // 2)
    tables = he.NttTables(N, qs)
    d = empty(count, limbs, N)
    g_fwd = _capture(lambda s: he.ntt_fwd(d, N, limbs, count, tables, stream=s))
    g_inv = _capture(lambda s: he.ntt_inv(d, N, limbs, count, tables, stream=s))
    r = Rng(800 + N)
    for rep in range(2):
        x = np.stack([r.uniform_limbs(qs, N) for _ in range(count)])
        _load(d, x)
        g_fwd.replay()
        got = host(d)
        for p in range(count):
            assert np.array_equal(got[p], oracle.ntt_fwd(x[p], qs)), (rep, p)
        # the inverse graph on an independent NTT-domain input
        y = np.stack([r.uniform_limbs(qs, N) for _ in range(count)])
        _load(d, y)
        g_inv.replay()
        got = host(d)
        for p in range(count):
            assert np.array_equal(got[p], oracle.ntt_inv(y[p], qs)), (rep, p)


def test_mixed_degree_plan_graph_replay():
    pool = he.primes_generate(60, 1 << 16, 6) + he.primes_generate(55, 1 << 16, 5) + \
        he.primes_generate(50, 1 << 16, 5)
    degrees = (4096, 8192, 16384, 32768)
    tables = {N: he.NttTables(N, pool) for N in degrees}
    r = Rng(810)
    Ns = [4096, 32768, 8192, 16384, 4096, 8192, 16384, 32768, 4096, 16384, 8192]
    Ls = [1, 3, 16, 5, 7, 2, 1, 1, 16, 3, 9]
    Fs = [0, 2, 0, 11, 4, 14, 15, 5, 0, 1, 7]
    ds = [empty(L, N) for N, L in zip(Ns, Ls)]
    plan = he.NttPlan([(ds[i], tables[N], N, L, f) for i, (N, L, f) in enumerate(zip(Ns, Ls, Fs))])
    assert plan.launches == 1
    g_fwd = _capture(lambda s: plan.fwd(stream=s))
    g_inv = _capture(lambda s: plan.inv(stream=s))
    for rep in range(2):
        xs = [r.uniform_limbs(pool[f:f + L], N) for N, L, f in zip(Ns, Ls, Fs)]
        for t, x in zip(ds, xs):
            _load(t, x)
        g_fwd.replay()
        for i, (N, L, f) in enumerate(zip(Ns, Ls, Fs)):
            assert np.array_equal(host(ds[i]), oracle.ntt_fwd(xs[i], pool[f:f + L])), (rep, i)
        g_inv.replay()
        for i in range(len(xs)):
            assert np.array_equal(host(ds[i]), xs[i]), (rep, i)


def test_mul_relin_rescale_graph_replay():
    N = 8192
    data, P = he.chain_primes(N, [60, 40, 40], 60)
    ctx = he.Context(N, data, P)
    r = Rng(820)
    evk = np.stack([np.stack([r.uniform_limbs(data + [P], N) for _ in range(2)]) for _ in range(3)])
    key = he.RelinKey(ctx, evk)
    level, count = 2, 5
    ca, cb = empty(count, 2, level + 1, N), empty(count, 2, level + 1, N)
    out = empty(count, 2, level, N)
    scratch = empty(ctx.mrr_scratch_bytes(level, count) // 8)
    g = _capture(lambda s: he.mul_relin_rescale(out, ca, cb, count, key, ctx, level, scratch, stream=s))
    for rep in range(2):
        A = np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)]) for _ in range(count)])
        B = np.stack([np.stack([r.uniform_limbs(data, N) for _ in range(2)]) for _ in range(count)])
        _load(ca, A)
        _load(cb, B)
        g.replay()
        got = host(out)
        for c in range(count):
            assert np.array_equal(got[c], oracle.mul_relin_rescale(A[c], B[c], evk, data, P, level)), (rep, c)
