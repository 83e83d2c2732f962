"""The multi-GPU path's host logic on CPU: two gloo ranks, as bench.py runs
one process per GPU under torchrun.  Realizations are independent, so ranks
draw disjoint seeded shards and share nothing on the data path; the timing is
reduced to the slowest rank, and the job's rate counts every rank's
realizations.  The one exchange an ensemble over GPUs needs (the sum of the
ranks' mean densities) is checked against a single process computing all of
it."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle as O
from paper_1602_03395_gb300 import inputs

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        # disjoint shards of the two-cloud workload, distinct data
        B = 3
        starts = bench.rank_realizations(rank, B)
        every = [None] * WORLD
        dist.all_gather_object(every, starts)
        spans = [set(range(s, s + B)) for r in range(WORLD) for s in every[r]]
        assert sum(len(x) for x in spans) == len(set().union(*spans)), "ranks share realizations"
        w = inputs.config_two_cloud()
        arr = w.batch_array(1, start=starts[0])
        sums = [None] * WORLD
        dist.all_gather_object(sums, complex(arr.sum()))
        assert sums[0] != sums[1]
        seeds = [None] * WORLD
        dist.all_gather_object(seeds, [bench.mixed_seed(rank, i) for i in range(1000)])
        assert not set(seeds[0]) & set(seeds[1])

        # the slowest rank's time, on every rank; the job's rate from it
        ms = bench.max_over_ranks(torch, dist, 10.0 + 5.0 * rank, "cpu")
        assert ms == 15.0
        assert bench.job_rate(steps=4, per_rank=B, world=WORLD, ms=ms) == pytest.approx(4 * B * WORLD / 0.015)

        # the ensemble's one exchange: each rank sums the densities of its own
        # realizations (a small 1-D geometry), then one all_reduce
        N, dx, lam, t = 64, 0.2, 7, 3.0
        rng = np.random.default_rng(1000 + rank)
        psi = (rng.normal(size=(2, N)) + 1j * rng.normal(size=(2, N))).astype(np.complex64)
        local = O.expand_density(psi, (dx,), t, (lam,)).sum(axis=0)
        tot = torch.from_numpy(local.astype(np.float64))
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        if rank == 0:
            ref = np.zeros(N)
            for r in range(WORLD):
                g = np.random.default_rng(1000 + r)
                p = (g.normal(size=(2, N)) + 1j * g.normal(size=(2, N))).astype(np.complex64)
                ref += O.expand_density(p, (dx,), t, (lam,)).sum(axis=0)
            assert np.allclose(tot.numpy(), ref, rtol=1e-12, atol=0)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    mp.spawn(_rank_main, args=(_free_port(),), nprocs=WORLD, join=True)


def test_bench_cli_checks(monkeypatch):
    """The unsplit variant exists for the tensor-core form of single-lattice
    workloads only; the end-to-end leg tries up to four lanes."""
    for argv in (["bench.py", "--unsplit"], ["bench.py", "--unsplit", "--form", "dense"],
                 ["bench.py", "--unsplit", "--form", "tc", "--workload", "mixed"]):
        monkeypatch.setattr("sys.argv", argv)
        with pytest.raises(SystemExit):
            bench.parse()
    monkeypatch.setattr("sys.argv", ["bench.py", "--unsplit", "--form", "tc", "--batch", "8"])
    a = bench.parse()
    assert a.unsplit and a.form == "tc" and a.batch == 8 and a.gpus == 1
    assert bench.E2E_MAX_LANES == 4


def test_bench_defaults_and_peak_choice(monkeypatch):
    """The default line is the largest single-GPU configuration (256^3 at
    lam = 100, with the 128x128x1024 companion record); the tensor-core
    roofline divides by the burst bf16 figure for a timed region under a
    second and by the sustained one for longer regions (both scaled by the
    nominal TF32 : BF16 ratio)."""
    monkeypatch.setattr("sys.argv", ["bench.py"])
    a = bench.parse()
    assert a.workload == "large_two_cloud" and not a.no_companion
    assert bench.COMPANION["large_two_cloud"] == "large_quasicondensate"
    pk = {"bf16_tflops": 1884.7, "bf16_tflops_sustained": 1699.1}
    burst, src = bench.tensor_peak(pk, "measured", 400.0)
    assert burst == pytest.approx(1884.7 * 1.1 / 2.25) and src.startswith("bf16_tflops x")
    sus, src = bench.tensor_peak(pk, "measured", 4000.0)
    assert sus == pytest.approx(1699.1 * 1.1 / 2.25) and src.startswith("bf16_tflops_sustained")


def test_bench_hbm_step_record():
    """Whole-step HBM bytes: 12 B per point algorithmic (psi0 in, densities
    out); the BF16 chain's launches move 16 (split) + 2 x 16 + 12 B per point
    on a 3-D lattice, the per-axis passes 16 + 16 + 12, a fused launch the
    algorithmic bytes."""
    import bench

    class W:
        dims = (64, 32, 16)

    pts = 64 * 32 * 16
    r = bench.hbm_step_record(W(), 2, True, False, 2 * pts * 4, 1.0, 1000.0, "measured")
    assert r["algorithmic_bytes"] == 2 * pts * 12
    assert r["implementation_bytes"] == 2 * pts * (16 + 32 + 12)
    assert abs(r["algorithmic_gbs"] - 2 * pts * 12 / 1e-3 / 1e9) < 1e-9
    assert abs(r["implementation_frac"] - r["implementation_gbs"] / 1000.0) < 1e-12
    r = bench.hbm_step_record(W(), 2, False, False, 2 * pts * 4, 1.0, 1000.0, "measured")
    assert r["implementation_bytes"] == 2 * pts * (32 + 12)
    r = bench.hbm_step_record(W(), 2, False, True, 2 * pts * 4, 1.0, 1000.0, "measured")
    assert r["implementation_bytes"] == r["algorithmic_bytes"]
