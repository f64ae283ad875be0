"""The autotuner's selection rule, with the timed GPU run stubbed on the host:
the fastest candidate wins only if its results equal the first candidate's;
a faster candidate whose results differ is rejected."""
import numpy as np
import pytest

from paper_1505_07368_gb300 import autotune
from paper_1505_07368_gb300 import cafgpu as C


def _stub(times, sigs, seen):
    def run(cand):
        i = len(seen)
        seen.append(cand)
        return times[i], sigs[i]
    return run


def test_factor_rejects_a_faster_candidate_with_different_results(tmp_path, monkeypatch):
    monkeypatch.setenv("CAFGPU_CACHE_DIR", str(tmp_path))
    cands = [{"factor_batch": 8, "factor_warps": 2, "ctas_per_sm": 2},
             {"factor_batch": 16, "factor_warps": 4, "ctas_per_sm": 2},
             {"factor_batch": 16, "factor_warps": 8, "ctas_per_sm": 2}]
    seen = []
    # candidate 1 is the fastest but its replies differ; candidate 2 is next
    run = _stub([0.30, 0.10, 0.20], [b"ok", b"WRONG", b"ok"], seen)
    n = np.arange(10, dtype=np.uint64)
    best, table = autotune.tune_factor(np.zeros(10, np.uint32), n, 4, 1 << 40, candidates=cands,
                                       timed_run=run, gpu_name="stub")
    assert seen == cands
    assert best == cands[2]
    assert table[1][1] == float("inf")
    # cached: the same workload and candidates do not run again
    best2, table2 = autotune.tune_factor(np.zeros(10, np.uint32), n, 4, 1 << 40, candidates=cands,
                                         timed_run=_stub([], [], []), gpu_name="stub")
    assert best2 == best and table2 == []


def test_gemm_rejects_a_faster_candidate_with_different_checksum(tmp_path, monkeypatch):
    monkeypatch.setenv("CAFGPU_CACHE_DIR", str(tmp_path))
    cands = autotune.GEMM_CANDIDATES_BF16[:4]
    seen = []
    sig_ok = (b"st", b"n", 123.0)
    sig_bad = (b"st", b"n", 123.5)          # one C differs
    run = _stub([0.5, 0.4, 0.1, 0.45], [sig_ok, sig_ok, sig_bad, sig_ok], seen)
    desc = np.zeros(3, C.GEMM_DESC_DTYPE)
    desc["n"] = [64, 128, 256]
    best, table = autotune.tune_gemm(C.GEMM_SPLIT_BF16X3, np.zeros(3, np.uint32), desc, None, 2,
                                     candidates=cands, timed_run=run, use_cache=False, gpu_name="stub")
    assert seen == cands
    assert best == cands[1]
    assert [t for _, t in table] == [0.5, 0.4, float("inf"), 0.45]


def test_bf16_search_covers_both_tile_widths():
    assert {c["gemm_tile_n"] for c in autotune.GEMM_CANDIDATES_BF16} == {128, 256}
    assert all("gemm_tile_n" not in c for c in autotune.GEMM_CANDIDATES)
    # GEMM claims take no per-claim message limit, so no candidate sets one
    assert all("max_msgs_per_claim" not in c for c in autotune.GEMM_CANDIDATES_BF16)


def test_gemm_gpu_timing_is_refused():
    desc = np.zeros(2, C.GEMM_DESC_DTYPE)
    desc["n"] = [64, 128]
    with pytest.raises(RuntimeError):
        autotune.tune_gemm(C.GEMM_BF16, np.zeros(2, np.uint32), desc, None, 1, use_cache=False, gpu_name="stub")
