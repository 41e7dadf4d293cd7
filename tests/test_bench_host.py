"""Host logic of bench.py that needs no GPU: the multi-rank aggregation of the
replica runs (two gloo ranks on the CPU), the whole-job throughput, and the
reference arm's rule that only rank 0 does work under torchrun."""
import json
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, torch.device("cpu"))   # rank 1 is slower
        value = bench.replica_throughput(world, 200_000, ms)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"ms": ms, "value": value}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_rank(tmp_path):
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for g in got:
        assert g["ms"] == 15.0                              # the max over ranks
        assert g["value"] == pytest.approx(2 * 200_000 / 0.015)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, None, None) == 12.5
    assert bench.replica_throughput(1, 1000, 2.0) == pytest.approx(500_000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        gpus, steps, warmup = 2, 1, 0

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""                    # no line, no oracle work


def test_algorithmic_work_of_the_c2_pass_by_hand():
    """12x12 signals, D 12x24, s = 6: C0 in the cheaper association
    2 (12*12*24 + 24*12*24) = 20 736; correlation updates 2*576*(0+1+...+5) =
    17 280; Cholesky and solves sum_t (2t^2 + 4t + 4) = 194; D1-side epilogue
    2*12*6 + 3*36 = 252: 38 462 FLOP per signal, 7.69e9 per 200k-signal pass.
    Bytes: the signal (576) and, in the second pass, the code (8 s + 4)."""
    assert bench.flops_per_signal_pass(12, 12, 24, 24, 6, 1) == 20736 + 17280 + 194 + 252
    assert bench.flops_per_signal_pass(12, 12, 24, 24, 6, 1) * 200_000 == pytest.approx(7.69e9, rel=1e-3)
    assert bench.bytes_per_signal_pass(12, 12, 6, 1) == 576
    assert bench.bytes_per_signal_pass(12, 12, 6, 2) == 576 + 52
