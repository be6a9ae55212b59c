"""Host-side logic of bench.py (no GPU): the packed 16-bit point format,
the workload descriptions (each says how L2 is handled), the traffic lookup
keyed by the kernel's source, and the host t_n comparison."""
import numpy as np
import pytest

import bench
from paper_1505_00914_gb300 import synth


def test_pack_u16_layout():
    P = np.asarray([[1, 1], [65536, 1], [1, 65536], [300, 7000]], np.int32)
    w = bench.pack_u16(P).view(np.uint32)
    np.testing.assert_array_equal(w & 0xFFFF, P[:, 0] - 1)
    np.testing.assert_array_equal(w >> 16, P[:, 1] - 1)
    # little-endian uint16 pairs (x - 1, y - 1)
    np.testing.assert_array_equal(w.view(np.uint16).reshape(-1, 2), P - 1)


@pytest.mark.parametrize("workload", sorted(bench.WORKLOADS) + ["learned", "batched", "box", "profile_batched",
                                                                 "melkman", "rxy", "sparse"])
def test_every_workload_has_a_config(workload):
    c = bench.workload_config(workload)
    assert c["workload"] == workload
    assert "l2" in c and ("256 MB write" in c["l2"] or "larger than L2" in c["l2"])


def test_small_inputs_are_flushed_and_large_ones_not():
    assert "256 MB write" in bench.workload_config("projected_shells")["l2"]
    assert "256 MB write" in bench.workload_config("plain_small")["l2"]
    assert "no flush" in bench.workload_config("plain_at_scale")["l2"]
    assert "no flush" in bench.workload_config("plain_at_scale_u16")["l2"]


def test_traffic_lookup_follows_the_kernel_source():
    t = bench._traffic("k_reduce_filtered", 1 << 26, 65536)
    assert t is not None and 8 * (1 << 26) <= t <= 1.05 * 8 * (1 << 26)
    t16 = bench._traffic("k_reduce_filtered", 1 << 26, 65536, u16=True)
    assert t16 is not None and 4 * (1 << 26) <= t16 <= 1.05 * 4 * (1 << 26)
    assert bench._traffic("k_reduce_filtered", 1 << 26, 4096) is None  # captured at another p
    assert bench._traffic("k_reduce_private", 1 << 26, 65536) is None


def test_host_t_n_comparison():
    p = 1024
    inputs = [(d, synth.points(d, 50_000, p, seed=3)) for d in ("uniform", "disc")]
    r = bench.cpu_andrew_all_points(p, inputs, m=20_000)
    assert r["speedup_t_n_over_t_r_plus_t_s"] > 0
    assert r["sort_andrew_gpoints_s"] > 0 and r["reduce_then_hull_gpoints_s"] > 0


def test_all_core_reduction_merges_to_one_pass_of_algorithm_1():
    """Per-thread partial arrays merged by min/max equal Algorithm 1 over all
    points (the function raises otherwise); shards smaller than a thread
    count, and empty shards, are covered by the tiny instance."""
    p = 512
    inputs = [("uniform", synth.points("uniform", 200_003, p, seed=5)),
              ("gaussian", synth.points("gaussian", 3, p, seed=6))]
    r = bench.cpu_reduce_all_cores(p, inputs, passes=1)
    assert r["threads"] >= 1 and r["reduce_gpoints_s"] > 0


def test_bench_reads_no_undefined_global():
    """Every global name a function of bench.py reads is defined at module
    level or is a builtin (a stray name fails only when its workload runs)."""
    import builtins
    import os
    import symtable
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py")
    top = symtable.symtable(open(path).read(), path, "exec")
    defined = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()
               or s.is_namespace()} | set(dir(builtins)) | {"__file__", "__name__"}
    missing = []

    def walk(t):
        for s in t.get_symbols():
            if s.is_referenced() and s.is_global() and s.get_name() not in defined:
                missing.append((t.get_name(), s.get_name()))
        for c in t.get_children():
            walk(c)

    walk(top)
    assert not missing, missing


def test_autotune_cache_key_and_lookup(tmp_path, monkeypatch):
    """The tuning cache is keyed by the batch's shape, the candidate chunk
    sizes and CTA shapes and the kernel source; a cached batch is answered
    without a launch."""
    from paper_1505_00914_gb300 import autotune
    monkeypatch.setenv("CH_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    off, ps = np.asarray([0, 10, 30]), np.asarray([16, 256], np.int32)
    k = autotune.batch_key(off, ps)
    assert k == autotune.batch_key(off.copy(), ps.copy())
    assert k != autotune.batch_key(np.asarray([0, 11, 30]), ps)
    assert k != autotune.batch_key(off, np.asarray([16, 1024], np.int32))
    assert k != autotune.batch_key(off, ps, candidates=(8, 16))
    assert k != autotune.batch_key(off, ps, shapes=(0, 768))
    autotune._store({k: {"chunk_mult": 256, "fold_threads": 768,
                         "ms": {"8/0": 2.0, "256/768": 1.5}}})
    best, times = autotune.tune_batched(None, off, ps, None, None, None, None, None)
    assert best == (256, 768) and times == {"8/0": 2.0, "256/768": 1.5}


def test_clock_summary_from_nvidia_smi_rows():
    rows = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2070, 2070, 1000.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "garbage line\n",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
    ]
    c = bench.ClockSampler.summarize(rows)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = rows[:1] + ["0, 1500, 2070, 1400.0, 0x48, Active, Not Active, Active, Not Active\n"]
    assert bench.ClockSampler.summarize(hot)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler.summarize(["garbage\n"]) is None
