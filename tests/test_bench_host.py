"""Host logic of bench.py, on the CPU: the multi-rank plumbing over gloo (two ranks),
the reference arm under torch.distributed.run, the byte model, and the guard that keeps
stale ncu traffic figures out of the JSON line."""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    bench = load_bench()
    bench.barrier(2)
    top = bench.reduce_max(float(10 * (rank + 1)), 2)  # rank 0: 10, rank 1: 20
    bench.barrier(2)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"max": top}, f)


def test_max_over_ranks_and_barrier_with_two_gloo_ranks(tmp_path):
    """The timed region's wall time is the maximum over ranks, taken after a barrier."""
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    for r in range(2):
        assert json.load(open(tmp_path / f"rank{r}.json"))["max"] == 20.0


def test_reference_arm_prints_one_line_from_rank_zero_under_torchrun():
    """With two ranks, rank 0 alone times the oracle and prints; the other rank exits 0."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py",
           "--impl", "reference", "--workload", "tiny", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(x) for x in p.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["value"] == line["value"]


def test_byte_model_hand_computed():
    """One tiny case worked by hand: q = 1000 queries (100 inserts), 400 distinct keys (all
    hits), 50 written, 10,000 live keys after the batch, levels 1..4 of 10,000 / 2,500 /
    625 / 156 keys, P = 1/4, an L2 of 40,000 bytes."""
    bench = load_bench()
    ab = bench.algorithmic_bytes(q=1000, q_ins=100, distinct=400, hits=400, writes=50, live_after=10000,
                                 level_sizes=[0, 10000, 2500, 625, 156], l2_bytes=40000, p=0.25)
    assert ab["io"] == 1000 * 25 + 100 * 8                  # 25,800
    # level 2: 12 B x 2,500 = 30,000 > L2 / 2 = 20,000; level 3: 7,500 and level 4 fit
    assert ab["traversal"] == 400 * 64                       # 25,600
    assert ab["storage"] == 400 * 32 + 400 * 32 + 50 * 96   # 30,400
    assert ab["rebuild"] == 9 * 10000 + 12 * 10000 / 3       # 130,000: N' p / (1 - p) = N' / 3 entries
    assert ab["total"] == 25800 + 25600 + 30400 + 130000
    ab2 = bench.algorithmic_bytes(1000, 100, 400, 400, 50, 10000, [0, 10000, 2500, 625, 156], 10000, 0.25)
    assert ab2["traversal"] == 400 * 64 * 2                  # level 3 (7,500 B) no longer fits in half the L2


def test_stale_ncu_figures_are_not_reported(tmp_path, monkeypatch):
    """The per-kernel ncu figures count only for the sources and the workload they were
    captured with; index-size kernels are scaled by keys, the others by batch size."""
    bench = load_bench()
    data = {"workload": "skewed", "digest": bench.source_digest(), "capture": {"keys": 1000, "batch": 100},
            "kernels": {"k_locate": {"launches_per_batch": 1, "dram_bytes": 5000, "scales_with": "queries"},
                        "k_relevel_write": {"launches_per_batch": 1, "dram_bytes": 700, "scales_with": "index"},
                        "k_sort_count": {"launches_per_batch": 4, "dram_bytes": 10, "scales_with": "queries"}}}
    f = tmp_path / "k.json"
    f.write_text(json.dumps(data))
    monkeypatch.setattr(bench, "KERNEL_PROFILE", str(f))
    total, kern, note = bench.kernel_profile("skewed", 4000, 200)
    assert total == 5000 * 2 + 700 * 4 + 4 * 10 * 2 and "lower bound" in note
    assert bench.kernel_profile("mid", 4000, 200)[0] is None
    data["digest"] = "0" * 16
    f.write_text(json.dumps(data))
    total, kern, note = bench.kernel_profile("skewed", 4000, 200)
    assert total is None and kern is None and "changed" in note


def test_tuned_tables_are_well_formed():
    """The committed tuning tables hold a valid kernel variant per size class (clusters
    only with 16 or 32 warps and 8-bit digits) and a lowest level per class, and the
    bench reads the plain path's table for the sizes it tuned."""
    bench = load_bench()
    classes = bench.tuned_classes()
    assert classes and [c[0] for c in classes] == sorted(c[0] for c in classes)
    for c in classes:
        hi, warps, bits = c[:3]
        cluster = c[3] if len(c) > 3 else 1
        assert warps in (8, 16, 32) and bits in (4, 8)
        assert cluster in (0, 1, 2, 4, 8, 16)
        if cluster > 1:
            assert warps in (16, 32) and bits == 8
    for n in (1 << 12, 1 << 16, 1 << 20, 1 << 26):
        assert bench.tuned_lowest(n) in (0, 2, 3, 4, 5, 6)
    plain = bench.tuned_plain(1 << 27)
    assert plain.get("lowest_level") in (2, 3, 4, 5) and plain.get("sort_passes") in (0, 1, 2, 3, 4, 8)
    assert bench.tuned_plain(1 << 16) == {}  # no tuned size within a factor of two


def test_autotune_variant_names_round_trip():
    from paper_1601_00159_gb300 import autotune
    for v in autotune.VARIANTS:
        assert autotune.parse_kernel(autotune.kernel_name(v)) == v
    assert autotune.kernel_name((32, 8, 1)) == "32x8" and autotune.parse_kernel("16x8c4") == (16, 8, 4)
    assert all(w in (16, 32) and b == 8 for (w, b, c) in autotune.VARIANTS if c > 1)
