"""Helpers shared by the GPU tests: device batches through the C ABI."""
import ctypes

import numpy as np

from paper_1505_07368_gb300 import cafgpu as C


def to_device(arr: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr).view(np.uint8).copy()).cuda()


def device_batch(rt, actor_idx, kind, u64, sender=None, sender_seq=None, tag=None):
    """Run one device-resident batch; returns the reply records (numpy)."""
    import torch
    cnt = len(u64)
    m = np.zeros(cnt, C.DMSG_DTYPE)
    m["actor"] = actor_idx
    m["kind"] = kind
    m["u64"] = u64
    m["sender"] = 0 if sender is None else sender
    m["sender_seq"] = np.arange(cnt) if sender_seq is None else sender_seq
    m["tag"] = np.arange(cnt) if tag is None else tag
    d_m = to_device(m)
    d_r = torch.zeros(cnt * C.DREPLY_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    rt.request_batch_device(d_m.data_ptr(), cnt, d_r.data_ptr())
    rt.stream_sync()
    return d_r.cpu().numpy().view(C.DREPLY_DTYPE).copy()


def host_requests(rt, actors, kind, u64, sender=0, tags=None, timeout_ns=120_000_000_000):
    cnt = len(u64)
    msgs = (C.Msg * cnt)()
    for i in range(cnt):
        msgs[i] = C.Runtime.msg(kind, int(u64[i]), sender=sender,
                                tag=int(tags[i]) if tags is not None else i)
    h = rt.request_batch(np.asarray(actors, dtype=np.uint64), msgs)
    return rt.await_batch(h, timeout_ns=timeout_ns)


_cudart = None


def d2h(ptr: int, nbytes: int) -> np.ndarray:
    """Copy `nbytes` from a raw device address (cudaMemcpy from the toolkit's libcudart)."""
    global _cudart
    if _cudart is None:
        _cudart = ctypes.CDLL("/usr/local/cuda/lib64/libcudart.so")
        _cudart.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
        _cudart.cudaMemcpy.restype = ctypes.c_int
    out = np.empty(nbytes, dtype=np.uint8)
    rc = _cudart.cudaMemcpy(out.ctypes.data, ptr, nbytes, 2)   # cudaMemcpyDeviceToHost
    assert rc == 0, rc
    return out
