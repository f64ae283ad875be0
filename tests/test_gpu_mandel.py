"""MANDELBROT actors (the OpenCL actor experiment of Sec. 5) against the oracle.

Escape counts are integers decided by a fixed sequence of rounded float32
operations, so every pixel must equal the oracle's count bit for bit, and
the reply must be (pixels, sum of the counts)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1505_07368_gb300 import cafgpu as C
from paper_1505_07368_gb300 import workloads as W

from helpers import to_device

pytestmark = pytest.mark.gpu

IMG = W.mandel_image()                 # the paper's 1920 x 1080 cut
# a boundary-rich region: counts spread over the whole range
EDGE = (np.float32(-0.80), np.float32(0.05), np.float32(0.0031), np.float32(0.0027))


def _desc(out, width, rows, row0, max_iter, geom):
    x0, y0, dx, dy = geom
    return C.MandelDesc(out.data_ptr(), width, rows, row0, max_iter, float(x0), float(y0), float(dx), float(dy))


def _request_slices(rt, actor, width, slices, max_iter, geom):
    """Host requests, one per (row0, rows) slice; returns (images, replies)."""
    import torch
    outs = [torch.full((rows, width), -1, dtype=torch.int32, device="cuda") for _, rows in slices]
    torch.cuda.synchronize()
    descs = [_desc(o, width, rows, row0, max_iter, geom) for o, (row0, rows) in zip(outs, slices)]
    msgs = (C.Msg * len(slices))()
    for i, d in enumerate(descs):
        msgs[i] = C.Runtime.mandel_msg(d, tag=i)
    h = rt.request_batch(np.full(len(slices), actor, dtype=np.uint64), msgs)
    rep = rt.await_batch(h, timeout_ns=120_000_000_000)
    torch.cuda.synchronize()
    return [o.cpu().numpy().view(np.uint32) for o in outs], rep


def _check(images, rep, width, slices, max_iter, geom):
    x0, y0, dx, dy = geom
    for img, r, (row0, rows) in zip(images, rep, slices):
        want, s = oracle.mandel_rows(x0, y0, dx, dy, width, row0, rows, max_iter)
        assert r["status"] == C.REPLY_OK
        assert (r["r0"], r["r1"]) == (rows * width, s)
        bad = np.argwhere(img != want)
        assert bad.size == 0, (row0, bad[:5], img[tuple(bad[0])], want[tuple(bad[0])])


@pytest.fixture(scope="module", params=["persistent", "per_message"])
def rt_actor(request):
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=16) as rt:
        a = rt.spawn(C.MANDELBROT)
        if request.param == "per_message":
            rt.set_backend(C.BACKEND_PER_MESSAGE_LAUNCH)
        yield rt, a


@pytest.mark.parametrize("width, height, parts, max_iter", [
    (200, 150, 1, 300),        # ragged: pixels not a multiple of 32 or of a band
    (200, 150, 7, 300),
    (1, 1, 1, 50),
    (1, 97, 3, 1000),          # one column
    (333, 1, 1, 65536),        # one row, the largest max_iter
    (128, 128, 4, 0),          # max_iter 0: every count 0
    (96, 64, 2, 1),
    (700, 40, 1, 12),          # max_iter equal to one block of 12 updates
    (700, 40, 1, 13),
    (300, 30, 1, 511),         # the last max_iter with blocks of 12
    (300, 30, 1, 512),         # the first with blocks of 16
    (300, 30, 1, 528),
])
def test_edge_region_bit_exact(rt_actor, width, height, parts, max_iter):
    rt, a = rt_actor
    slices = W.mandel_slices(height, parts)
    images, rep = _request_slices(rt, a, width, slices, max_iter, EDGE)
    _check(images, rep, width, slices, max_iter, EDGE)


def test_paper_image_small_problem_bit_exact(rt_actor):
    """The full 1920 x 1080 image with 120 iterations, as 10 slices of 108 rows."""
    rt, a = rt_actor
    slices = W.mandel_slices(W.MANDEL_HEIGHT, 10)
    images, rep = _request_slices(rt, a, W.MANDEL_WIDTH, slices, 120, IMG)
    _check(images, rep, W.MANDEL_WIDTH, slices, 120, IMG)


def test_paper_image_large_problem_sampled_rows(rt_actor):
    """The full image with 1200 iterations in one message; 48 sampled rows and the
    reply's sum checked against the oracle (the full oracle image takes seconds)."""
    rt, a = rt_actor
    images, rep = _request_slices(rt, a, W.MANDEL_WIDTH, [(0, W.MANDEL_HEIGHT)], 1200, IMG)
    img = images[0]
    x0, y0, dx, dy = IMG
    rows = np.random.default_rng(1200).choice(W.MANDEL_HEIGHT, 48, replace=False)
    for j in sorted(rows.tolist()) + [0, W.MANDEL_HEIGHT - 1]:
        want, _ = oracle.mandel_rows(x0, y0, dx, dy, W.MANDEL_WIDTH, j, 1, 1200)
        assert np.array_equal(img[j], want[0]), j
    assert rep[0]["status"] == C.REPLY_OK
    assert rep[0]["r0"] == W.MANDEL_WIDTH * W.MANDEL_HEIGHT
    assert rep[0]["r1"] == int(img.astype(np.uint64).sum())


def test_many_jobs_reuse_records():
    """More messages than job records (256) from several actors at once."""
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=16) as rt:
        actors = [rt.spawn(C.MANDELBROT) for _ in range(4)]
        import torch
        width, max_iter = 96, 400
        n = 600
        outs = torch.zeros((n, 5, width), dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        descs = []
        msgs = (C.Msg * n)()
        for i in range(n):
            row0 = (i * 5) % 200
            descs.append(C.MandelDesc(outs[i].data_ptr(), width, 5, row0, max_iter, *map(float, EDGE)))
            msgs[i] = C.Runtime.mandel_msg(descs[-1], sender=i % 3, tag=i)
        to = np.array([actors[i % 4] for i in range(n)], dtype=np.uint64)
        rep = rt.await_batch(rt.request_batch(to, msgs), timeout_ns=120_000_000_000)
        got = outs.cpu().numpy().view(np.uint32)
        x0, y0, dx, dy = EDGE
        full, _ = oracle.mandel_rows(x0, y0, dx, dy, width, 0, 205, max_iter)
        for i in range(n):
            row0 = (i * 5) % 200
            assert np.array_equal(got[i], full[row0:row0 + 5]), i
            assert rep[i]["status"] == C.REPLY_OK
            assert (rep[i]["r0"], rep[i]["r1"]) == (5 * width, int(full[row0:row0 + 5].astype(np.uint64).sum()))


def test_device_batch_and_rejects():
    """Device-resident messages name device descriptors; bad descriptors are rejected."""
    import torch
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=8) as rt:
        a = rt.spawn(C.MANDELBROT)
        width, max_iter = 150, 500
        out = torch.zeros((4, 30, width), dtype=torch.int32, device="cuda")
        d = np.zeros(7, C.MANDEL_DESC_DTYPE)
        for i in range(4):
            d[i] = (out[i].data_ptr(), width, 30, 30 * i, max_iter, *EDGE)
        d[4] = (out[0].data_ptr(), 0, 30, 0, max_iter, *EDGE)                 # width 0
        d[5] = (out[0].data_ptr(), width, 30, 0, (1 << 16) + 1, *EDGE)        # max_iter too large
        d[6] = (out[0].data_ptr() + 2, width, 30, 0, max_iter, *EDGE)         # misaligned out
        d_desc = to_device(d)
        m = np.zeros(8, C.DMSG_DTYPE)
        m["actor"] = a - 1
        m["kind"] = C.MANDELBROT
        m["u64"] = [d_desc.data_ptr() + i * d.itemsize for i in range(7)] + [0]   # last: null descriptor
        m["sender_seq"] = np.arange(8)
        d_m = to_device(m)
        d_r = torch.zeros(8 * C.DREPLY_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        rt.request_batch_device(d_m.data_ptr(), 8, d_r.data_ptr())
        rt.stream_sync()
        rep = d_r.cpu().numpy().view(C.DREPLY_DTYPE)
        got = out.cpu().numpy().view(np.uint32)
        x0, y0, dx, dy = EDGE
        full, _ = oracle.mandel_rows(x0, y0, dx, dy, width, 0, 120, max_iter)
        for i in range(4):
            assert rep[i]["status"] == C.REPLY_OK and rep[i]["done"] == 1
            assert np.array_equal(got[i], full[30 * i:30 * i + 30])
            assert rep[i]["r1"] == int(full[30 * i:30 * i + 30].astype(np.uint64).sum())
        for i in range(4, 8):
            assert rep[i]["status"] == C.REPLY_REJECTED and rep[i]["done"] == 1, i


def test_host_rejects_bad_descriptors():
    import torch
    with C.Runtime(max_factor_n=(1 << 32) - 1, max_actors=8) as rt:
        a = rt.spawn(C.MANDELBROT)
        out = torch.zeros(64, dtype=torch.int32, device="cuda")
        bad = [
            C.MandelDesc(None, 8, 8, 0, 10, *map(float, EDGE)),
            C.MandelDesc(out.data_ptr(), 0, 8, 0, 10, *map(float, EDGE)),
            C.MandelDesc(out.data_ptr(), 8, 0, 0, 10, *map(float, EDGE)),
            C.MandelDesc(out.data_ptr(), 1 << 13, 1 << 12, 0, 10, *map(float, EDGE)),   # 2^25 pixels
            C.MandelDesc(out.data_ptr(), 8, 8, (1 << 24) - 4, 10, *map(float, EDGE)),   # rows past 2^24
            C.MandelDesc(out.data_ptr(), 8, 8, 0, (1 << 16) + 1, *map(float, EDGE)),
            C.MandelDesc(out.data_ptr() + 1, 8, 8, 0, 10, *map(float, EDGE)),
        ]
        for d in bad:
            rc = rt.L.caf_gpu_request(rt.h, a, ctypes.byref(C.Runtime.mandel_msg(d)), ctypes.byref(ctypes.c_uint64()))
            assert rc == C.EINVAL
        good = C.MandelDesc(out.data_ptr(), 8, 8, 0, 10, *map(float, EDGE))
        assert rt.try_send(a, C.Runtime.mandel_msg(good)) == C.EINVAL     # needs a reply
        st, r0, r1 = rt.await_(rt.request(a, C.Runtime.mandel_msg(good)))
        assert (st, r0) == (C.REPLY_OK, 64)


def test_same_counts_alone_and_mixed_with_factor_and_gemm():
    """Bands share the drain with GEMM tiles and factor sweeps; counts do not change."""
    import torch
    from helpers import host_requests
    width, height, max_iter = 640, 96, 800
    slices = W.mandel_slices(height, 6)
    with C.Runtime(max_factor_n=(1 << 56) - 1, max_actors=32) as rt:
        am = rt.spawn(C.MANDELBROT)
        alone, rep_alone = _request_slices(rt, am, width, slices, max_iter, EDGE)
        af = rt.spawn(C.FACTOR_U64)
        ag = rt.spawn(C.GEMM_BF16)
        n = 512
        A = torch.randn(n, n, device="cuda")
        B = torch.randn(n, n, device="cuda")
        Cs = [torch.empty(n, n, device="cuda") for _ in range(8)]
        torch.cuda.synchronize()
        nums, _, _ = W.semiprimes(W.primes_uniform(W.stream_key(77, 1), 128, 1 << 24, 1 << 28))
        hg = [rt.request(ag, C.Runtime.msg(C.GEMM_BF16, n=n, A=A.data_ptr(), B=B.data_ptr(), C=c.data_ptr()))
              for c in Cs]
        outs = [torch.zeros((rows, width), dtype=torch.int32, device="cuda") for _, rows in slices]
        torch.cuda.synchronize()
        descs = [_desc(o, width, rows, row0, max_iter, EDGE) for o, (row0, rows) in zip(outs, slices)]
        hm = [rt.request(am, C.Runtime.mandel_msg(d)) for d in descs]
        fac = host_requests(rt, [af] * len(nums), C.FACTOR_U64, nums)
        rep_mixed = [rt.await_(h, 120_000_000_000) for h in hm]
        for h in hg:
            assert rt.await_(h, 120_000_000_000)[0] == C.REPLY_OK
        torch.cuda.synchronize()
        for o, img, r0, r1 in zip(outs, alone, rep_mixed, rep_alone):
            assert np.array_equal(o.cpu().numpy().view(np.uint32), img)
            assert (r0[0], r0[1], r0[2]) == (r1["status"], r1["r0"], r1["r1"])
        for (s, pp, q), nn in zip(zip(fac["status"], fac["r0"], fac["r1"]), nums):
            assert s == C.REPLY_OK and int(pp) * int(q) == int(nn)
    _check(alone, rep_alone, width, slices, max_iter, EDGE)


def test_fp32_rate_probe():
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    r = C.measure_fp32_rate() / sms
    # 128 float32 lanes per SM at 1-2.1 GHz: about 1.3e11 to 2.7e11 operations/s per SM
    assert 5e10 < r < 4e11, r
