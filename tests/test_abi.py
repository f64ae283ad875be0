"""CPU checks of the C-ABI library: it builds, loads and exports every symbol
that include/caf_gpu.h declares, and the binding's structs match the header."""
import ctypes
import os
import re

import pytest

from paper_1505_07368_gb300 import _build, cafgpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "caf_gpu.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(caf_gpu_\w+)\s*\(", src)))


def test_header_declarations_match_binding():
    assert _declared() == sorted(cafgpu.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    lib_path = _build.build()
    L = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(L, name), name


def test_struct_sizes():
    assert ctypes.sizeof(cafgpu.Msg) == 56
    assert ctypes.sizeof(cafgpu.Reply) == 32
    assert cafgpu.DMSG_DTYPE.itemsize == 32
    assert cafgpu.DREPLY_DTYPE.itemsize == 32
    assert cafgpu.GEMM_DESC_DTYPE.itemsize == 32
    assert cafgpu.MANDEL_DESC_DTYPE.itemsize == 40
    assert ctypes.sizeof(cafgpu.MandelDesc) == 40
    assert cafgpu.LOG_DTYPE.itemsize == 40
    assert cafgpu.SERVE_REQ_DTYPE.itemsize == 48
    assert cafgpu.SERVE_RESULT_DTYPE.itemsize == 48
    assert ctypes.sizeof(cafgpu.ServeCfg) == 32
    assert ctypes.sizeof(cafgpu.ServeStats) == 32
    assert ctypes.sizeof(cafgpu.RuntimeCfg) == 104
    assert ctypes.sizeof(cafgpu.ActorCfg) == 56
    assert ctypes.sizeof(cafgpu.Stats) == 96


def test_strerror_without_gpu():
    L = cafgpu.load()
    assert L.caf_gpu_strerror(cafgpu.EDEAD) == b"actor has terminated"


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(cafgpu.CafGpuError) as e:
        cafgpu.Runtime(max_factor_n=1 << 20)
    assert e.value.code == cafgpu.ECUDA


def test_header_constants_match_binding():
    src = open(HEADER).read()
    defs = dict(re.findall(r"#define\s+CAF_GPU_(\w+)\s+\(?(-?\d+)u?\)?", src))
    want = {
        "FACTOR_U64": cafgpu.FACTOR_U64, "GEMM_BF16": cafgpu.GEMM_BF16,
        "GEMM_SPLIT_BF16X3": cafgpu.GEMM_SPLIT_BF16X3, "RING_TOKEN": cafgpu.RING_TOKEN,
        "SINK": cafgpu.SINK, "SOURCE": cafgpu.SOURCE, "MANDELBROT": cafgpu.MANDELBROT, "FORK": cafgpu.FORK,
        "ACTOR_MASTER": cafgpu.ACTOR_MASTER, "ACTOR_RECREATE": cafgpu.ACTOR_RECREATE,
        "SCHED_GLOBAL": cafgpu.SCHED_GLOBAL, "SCHED_STEAL": cafgpu.SCHED_STEAL,
        "BACKEND_PERSISTENT": cafgpu.BACKEND_PERSISTENT,
        "BACKEND_PER_MESSAGE_LAUNCH": cafgpu.BACKEND_PER_MESSAGE_LAUNCH,
        "REPLY_OK": cafgpu.REPLY_OK, "REPLY_NOFACTOR": cafgpu.REPLY_NOFACTOR,
        "REPLY_DEAD": cafgpu.REPLY_DEAD, "REPLY_REJECTED": cafgpu.REPLY_REJECTED,
        "EINVAL": cafgpu.EINVAL, "ENOMEM": cafgpu.ENOMEM, "EAGAIN": cafgpu.EAGAIN,
        "ETIMEDOUT": cafgpu.ETIMEDOUT, "EDEAD": cafgpu.EDEAD, "EWAITLIMIT": cafgpu.EWAITLIMIT,
        "ESTATE": cafgpu.ESTATE, "ECUDA": cafgpu.ECUDA, "EBOUNDS": cafgpu.EBOUNDS,
    }
    for name, value in want.items():
        assert int(defs[name]) == value, name


@pytest.mark.parametrize("bad", [
    {"factor_warps": 3}, {"factor_batch": 17}, {"ctas_per_sm": 5}, {"mailbox_capacity": 48},
    {"ingress_capacity": 1000}, {"max_factor_n": 1 << 62}, {"gemm_items_per_round": 9},
    {"scheduler": 2}, {"max_actors": (1 << 24) + 1}, {"max_actors": 1 << 20, "fork_pool": (1 << 31) - (1 << 20)},
    {"factor_split": 33}, {"gemm_tile_n": 192},
])
def test_bad_runtime_settings_rejected_before_any_cuda_call(bad):
    # the settings are checked before the runtime touches the device, so this
    # holds with or without a GPU
    with pytest.raises(cafgpu.CafGpuError) as e:
        cafgpu.Runtime(**bad)
    assert e.value.code == cafgpu.EINVAL, bad
