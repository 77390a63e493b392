"""Host logic of bench.py on CPU: the N > 1 path over gloo (127.0.0.1) and the traffic record.

The hot path does not shard (replicas only): each rank renders whole frames of its own views
and the job's rate is all ranks' rays over the slowest rank's time.  Checks the helpers bench.py
uses for that (the per-rank view assignment, the max-over-ranks reduction, the aggregate rate,
the reference arm's rank-0 rule) and the rule that ties the reported DRAM traffic to the
kernel sources it was captured on.
"""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(ms, dist)
        views = [bench.replica_view(f, rank, world) for f in range(8)]
        rate = bench.job_rate(1920 * 1080, 4, world, slowest)
        dist.barrier()
        q.put((rank, slowest, views, rate))
    finally:
        dist.destroy_process_group()


def test_two_replicas_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (r0, m0, v0, rate0), (r1, m1, v1, rate1) = out
    # the job's time is the slowest rank's, on every rank
    assert m0 == m1 == 150.0
    # both ranks report the same whole-job rate: all ranks' rays over that time
    assert rate0 == rate1 == pytest.approx(1920 * 1080 * 4 * 2 / 0.150 / 1e6)
    # at every step the two replicas render different views of the 16-view orbit
    assert all(a != b for a, b in zip(v0, v1))
    assert sorted(set(v0) | set(v1)) == list(range(16))


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(12.5) == 12.5
    assert [bench.replica_view(f, 0, 1) for f in range(3)] == [0, 1, 2]
    assert bench.job_rate(1000, 2, 1, 1.0) == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    # under torchrun the reference arm (the oracle on the host cores) runs on rank 0 alone; the other
    # ranks return at once, printing nothing
    import types

    import bench

    monkeypatch.setenv("RANK", "1")
    args = types.SimpleNamespace(dims=512, width=1920, height=1080, steps=2, warmup=3, gpus=2)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    # the bench reports a committed DRAM-traffic capture of a smaller frame, scaled by the frames' sample
    # evaluations, only for the workload it names and only while the kernel's sources hash to the
    # captured ones
    import hashlib
    import json
    import types

    import bench

    fake = tmp_path / "root"
    (fake / "profiles").mkdir(parents=True)
    (fake / "src").mkdir()
    (fake / "src" / "k.cu").write_text("kernel source\n")
    h = hashlib.sha256((fake / "src" / "k.cu").read_bytes()).hexdigest()
    rec = {"kernel": "gen_count_kernel", "workload": "a small workload", "scales_to": "a workload",
           "sample_evals": 1000, "dram_bytes_read": 3.0e9, "dram_bytes_write": 1.0e9, "sources": ["src/k.cu"],
           "sources_sha256": h}
    (fake / "profiles" / "gen_count_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(fake))
    wl = types.SimpleNamespace(name="a workload")
    assert bench.gen_traffic(wl, 1000) == 4.0e9
    assert bench.gen_traffic(wl, 8000) == 32.0e9
    assert bench.gen_traffic(types.SimpleNamespace(name="another workload"), 1000) is None
    # the kernel source differs by one byte
    (fake / "src" / "k.cu").write_text("kernel source\n\n")
    assert bench.gen_traffic(wl, 1000) is None
