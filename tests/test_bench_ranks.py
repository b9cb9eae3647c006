"""Host logic of the multi-GPU (replica) benchmark on CPU: two gloo ranks reduce their step
times to the maximum and their kernel-launch counts to the sum, the whole-job value counts
the work of every rank over the slowest time, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, n = bench.reduce_over_ranks(dist, torch.device("cpu"), 10.0 + 5.0 * rank, 100 + rank)
    out[rank] = (ms, n)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_summed_launches():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (15.0, 201)


def test_whole_job_value_and_single_rank_identity():
    assert bench.reduce_over_ranks(None, None, 12.5, 7) == (12.5, 7)
    # 2 ranks of 1e12 flops each over 0.5 s = 4 TFLOP/s
    assert bench.aggregate_value(2, 1e12, 500.0) == pytest.approx(4.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    import argparse
    ns = argparse.Namespace(impl="reference", gpus=2, steps=1, warmup=0, workload="p3",
                            prec="f32", rr="tc32", no_fp64_compare=True, no_cpu_baseline=True)
    assert bench.run_reference(ns) == 0
    assert capsys.readouterr().out == ""
