"""Serving loop: open-loop arrivals, admission under a memory budget, continuous
batching; results checked against the oracle, alone and in the mix."""
import numpy as np
import pytest

import oracle
from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N_F, N_G = 16, 8          # factor / GEMM actors


def _setup(rt, wl, pool):
    f_actors = [rt.spawn(C.FACTOR_U64, mailbox_capacity=256) for _ in range(N_F)]
    g_actors = [rt.spawn(C.GEMM_SPLIT_BF16X3, mailbox_capacity=256) for _ in range(N_G)]
    reqs = np.zeros(wl.count, C.SERVE_REQ_DTYPE)
    isf = wl.kind == C.FACTOR_U64
    reqs["actor"] = np.where(isf, np.array(f_actors, np.uint64)[wl.actor % N_F],
                             np.array(g_actors, np.uint64)[wl.actor % N_G])
    reqs["t_arrival"] = wl.t
    reqs["u64"] = wl.n
    reqs["n"] = wl.size
    base = pool.data_ptr()
    reqs["A"] = np.where(isf, 0, base + 4 * wl.a_off.astype(np.uint64))
    reqs["B"] = np.where(isf, 0, base + 4 * wl.b_off.astype(np.uint64))
    return reqs, isf


def _gemm_out(arena_np, res, n):
    off = int(res["c_offset"])
    return arena_np[off:off + 4 * n * n].view(np.float32).reshape(n, n)


@pytest.mark.parametrize("backend", [C.BACKEND_PERSISTENT, C.BACKEND_PER_MESSAGE_LAUNCH])
def test_serving_mix_budget_and_results(backend):
    import torch
    count = 2000 if backend == C.BACKEND_PERSISTENT else 600
    wl = W.config5(seed=51, n_requests=count, rate=4e4, max_gemm=256, factor_hi=1 << 22,
                   pool_elems=1 << 20, n_factor_actors=N_F, n_gemm_actors=N_G)
    pool_np = W.gemm_pool(wl.pool_seed, wl.pool_elems)
    pool = torch.from_numpy(pool_np).cuda()
    arena = torch.zeros(64 << 20, dtype=torch.uint8, device="cuda")
    budget = 4 << 20
    with C.Runtime(max_factor_n=(1 << 44) - 1, max_actors=64, mailbox_capacity=256) as rt:
        reqs, isf = _setup(rt, wl, pool)
        rt.set_backend(backend)
        torch.cuda.synchronize()
        res, st = rt.serve_run(reqs, arena.data_ptr(), arena.numel(), mem_budget_bytes=budget,
                               timeout_ns=120_000_000_000)
    torch.cuda.synchronize()
    assert st["peak_inflight_bytes"] <= budget
    assert np.all(res["status"] == 0)
    assert np.all(res["t_done"] >= res["t_admit"]) and np.all(res["t_admit"] >= wl.t - 1e-9)
    # factorization: generator certificate for all, the oracle's trial division on a sample
    fi = np.nonzero(isf)[0]
    assert np.array_equal(res["r0"][fi], wl.p[fi]) and np.array_equal(res["r1"][fi], wl.q[fi])
    for i in fi[::97]:
        assert (0, int(res["r0"][i]), int(res["r1"][i])) == oracle.factor(int(wl.n[i]))
    # GEMM: split-BF16x3 error bound against the float64 oracle on a sample
    arena_np = arena.cpu().numpy()
    gi = np.nonzero(~isf)[0]
    for i in gi[::max(1, gi.size // 25)]:
        n = int(wl.size[i])
        A = pool_np[wl.a_off[i]:wl.a_off[i] + n * n].reshape(n, n)
        B = pool_np[wl.b_off[i]:wl.b_off[i] + n * n].reshape(n, n)
        assert oracle.rel_frobenius(_gemm_out(arena_np, res[i], n), oracle.gemm_f64(A, B)) <= 1e-5


def test_each_result_same_alone_and_in_the_mix():
    """Requests sampled from a mixed run give bit-identical results when served alone."""
    import torch
    wl = W.config5(seed=52, n_requests=1500, rate=5e4, max_gemm=384, factor_hi=1 << 22,
                   pool_elems=1 << 20, n_factor_actors=N_F, n_gemm_actors=N_G)
    pool = torch.from_numpy(W.gemm_pool(wl.pool_seed, wl.pool_elems)).cuda()
    arena = torch.zeros(96 << 20, dtype=torch.uint8, device="cuda")
    with C.Runtime(max_factor_n=(1 << 44) - 1, max_actors=64, mailbox_capacity=256) as rt:
        reqs, isf = _setup(rt, wl, pool)
        torch.cuda.synchronize()
        mix, _ = rt.serve_run(reqs, arena.data_ptr(), arena.numel(), mem_budget_bytes=8 << 20)
        torch.cuda.synchronize()
        mix_np = arena.cpu().numpy()
        sample = list(np.nonzero(isf)[0][::150]) + list(np.nonzero(~isf)[0][::60])
        for i in sample:
            one = reqs[i:i + 1].copy()
            one["t_arrival"] = 0.0
            alone, _ = rt.serve_run(one, arena.data_ptr(), arena.numel())
            torch.cuda.synchronize()
            assert (alone["status"][0], alone["r0"][0], alone["r1"][0]) == (mix["status"][i], mix["r0"][i], mix["r1"][i])
            if not isf[i]:
                n = int(wl.size[i])
                got = _gemm_out(arena.cpu().numpy(), alone[0], n)
                assert np.array_equal(got.view(np.uint32), _gemm_out(mix_np, mix[i], n).view(np.uint32)), i
