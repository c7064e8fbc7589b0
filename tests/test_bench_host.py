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
    """One tiny case worked by hand: q = 1000 queries (100 inserts), 400 distinct keys, 50
    written, 10,000 storage nodes after the batch, levels 1..4 of 10,000 / 2,500 / 625 /
    156 keys, lowest built level 3 at P = 1/4 (gap 16 nodes), an L2 of 40,000 bytes."""
    bench = load_bench()
    ab = bench.algorithmic_bytes(q=1000, q_ins=100, distinct=400, hits=400, writes=50, size_after=10000,
                                 level_sizes=[0, 10000, 2500, 625, 156], l2_bytes=40000, sort_passes=8,
                                 lowest=3, inv_p=4)
    assert ab["io"] == 1000 * 25 + 100 * 8                  # 25,800
    assert ab["traversal"] == 0                              # 12 B x 625 = 7,500 < L2 / 2 = 20,000
    assert ab["storage"] == 400 * 128 + 400 * 32 + 50 * 96   # 68,800
    assert ab["rebuild"] == 9 * 10000 + 12 * (625 + 156)     # 99,372
    assert ab["total"] == 25800 + 0 + 68800 + 99372
    ab2 = bench.algorithmic_bytes(1000, 100, 400, 400, 50, 10000, [0, 10000, 2500, 625, 156], 10000, 8, 3, 4)
    assert ab2["traversal"] == 400 * 64                      # level 3 (7,500 B) no longer fits in half the L2


def test_stale_ncu_figures_are_not_reported(tmp_path, monkeypatch):
    bench = load_bench()
    text = open(bench.DRAM_PROFILE).read()
    good = bench.dram_profile("skewed")
    assert good[2] in ("ncu capture of this workload at full size", "kernel sources changed since the ncu capture")
    stale = tmp_path / "stale.md"
    data = json.loads(text.split("```json\n")[1].split("\n```")[0])
    data["digest"] = "0" * 16
    stale.write_text(text.split("```json\n")[0] + "```json\n" + json.dumps(data) + "\n```\n")
    monkeypatch.setattr(bench, "DRAM_PROFILE", str(stale))
    per_launch, per_batch, note = bench.dram_profile("skewed")
    assert per_launch is None and per_batch is None and "changed" in note
    data["digest"] = bench.source_digest()
    data["workload"] = "mid"
    stale.write_text("```json\n" + json.dumps(data) + "\n```\n")
    assert bench.dram_profile("skewed")[0] is None
    assert bench.dram_profile("mid")[0] is not None
