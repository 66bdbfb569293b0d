"""Host-side logic of bench.py that needs no GPU: the max-over-ranks /
sum-over-ranks reduction of a multi-replica run (world size 2 over gloo on
CPU), the algorithmic byte counts and the reference (CPU oracle) arm."""
import json
import os
import socket
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    t, u = bench.reduce_step(10.0 + 3 * rank, 5.0 + rank, world)
    bench.barrier(world)
    out.put((rank, t, u))
    dist.destroy_process_group()


def test_reduce_step_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 13.0, 11.0), (1, 13.0, 11.0)]


def test_algorithmic_bytes():
    """Per-individual model of the method: evaluation 16m + 8n, crossover
    4 E_S n + 4n, mutation 8n + M_P (16m + 8n), times N_p; the node-major
    access model beside it."""
    sys.path.insert(0, ROOT)
    import bench
    b = bench.algorithmic_bytes(n=1000, m=5000, np_=100, p_mut=0.2)
    assert b["evaluate"] == 100 * (16 * 5000 + 8 * 1000)
    assert b["crossover"] == 100 * (4 * 4 * 1000 + 4 * 1000)
    assert abs(b["mutation"] - 100 * (8 * 1000 + 0.2 * (16 * 5000 + 8 * 1000))) < 1e-6
    a = bench.access_bytes(n=1000, m=5000, np_=100, p_mut=0.2)
    csr = 4 * 1001 + 4 * 10000
    assert a["crossover"] == 16 * 100 * 1000
    oriented = 4 * 1001 + 4 * 5000 + 4 * 1000  # the evaluation's oriented CSR (each edge once) and node order
    assert a["evaluate"] == 4 * 100 * 1000 + 4 * 100 * 5000 + oriented + 4 * 100 * 1000
    assert a["mutation"] == 8 * 100 * 1000 + 4 * 0.2 * 100 * 10000 + csr + 8 * 100 * 1000
    r = bench.kernel_roofline("mutation", 0.5, 1000, 5000, 100, 0.2, 1000.0, "measured", "none")
    assert abs(r["achieved"] - b["mutation"] / 0.5e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1000.0) < 1e-12
    assert abs(r["frac_access"] - a["mutation"] / 0.5e-3 / 1e9 / 1000.0) < 1e-12


def test_recorded_traffic_only_for_the_current_source(tmp_path, monkeypatch):
    """A profile's DRAM traffic line counts only while the kernel source it
    was captured on is unchanged (matched by the source hash); otherwise the
    bench reports null traffic."""
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "paper_2506_01752_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k_eval.cu").write_text("// version 1\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    digest = bench.source_digest("evaluate")
    (tmp_path / "profiles" / "evaluate_kernel_lfr-40k.md").write_text(
        f"traffic_bytes_per_launch[evaluate@lfr-40k]: 12345 source_sha256_16: {digest}\n"
        "traffic_bytes_per_launch[evaluate@lfr-1m]: 999 source_sha256_16: 0000000000000000\n")
    assert bench.recorded_traffic("evaluate", "lfr-40k") == 12345.0
    assert bench.recorded_traffic("evaluate", "lfr-1m") is None      # captured on another source
    assert bench.recorded_traffic("mutation", "lfr-40k") is None     # no line for this kernel
    (src / "k_eval.cu").write_text("// version 2\n")
    assert bench.recorded_traffic("evaluate", "lfr-40k") is None     # kernel changed since


def test_reference_arm_prints_one_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "planted-1k", "--steps", "3", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, check=True)
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "planted-1k", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=120, env=env)
    assert out.returncode == 0 and out.stdout.strip() == ""
