"""The multi-GPU form is independent replicas (the peel does not shard): the benchmark takes the
slowest rank's time and counts every rank's units.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.reduce_max(100.0 + 50.0 * rank)  # rank 1 is the slower replica
    out[rank] = (t, bench.whole_job_rate(1000, world, 2, t))
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_every_rank():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        t, v = out[rank]
        assert t == 150.0
        assert v == pytest.approx(2 * 1000 * 2 / 0.150)


def test_single_rank_is_unchanged():
    import bench
    assert bench.reduce_max(42.0) == 42.0
    assert bench.whole_job_rate(10, 1, 3, 1000.0) == pytest.approx(30.0)


def test_pair_report_arithmetic():
    """The bench's per-pair figures from a step's counters (CPU, no GPU): the algorithmic bytes
    follow B = 4 E_scan + 8 U_cnt + 16 P_hash + 8 N_link + 12 frontier + 4 stamp reads."""
    import bench as b
    stats = {"rounds": 7, "scan_elements": 100, "s_cliques_listed": 50, "decrements": 20, "hash_probes": 3,
             "link_calls": 10, "frontier_total": 40, "stamp_reads": 60}
    info = {(2, 3): {"n_r": 40, "n_s": 30, "n_nodes": 3, "stats": stats}}
    oracle_res = {"2,3": {"n_s": 30, "seconds": 0.6, "core_equal": True}}
    rep = b.pair_report(info, {(2, 3): 2.0}, {(2, 3): 1.0}, {(2, 3): 5.0}, 1000.0, oracle_res)["2,3"]
    alg = 4 * 100 + 8 * 20 + 16 * 3 + 8 * 10 + 12 * 40 + 4 * 60
    assert b.algorithmic_peel_bytes(stats) == alg
    assert rep["s_cliques_peeled_per_s"] == 30 / 0.002
    assert abs(rep["peel_algorithmic_gbs"] - round(alg / 0.002 / 1e9, 3)) < 1e-12
    assert rep["method"] == b.METHOD[(2, 3)]
    assert rep["peel_frac_of_hbm_peak"] == (alg / 0.002 / 1e9) / 1000.0
    assert rep["oracle_seconds"] == 0.6 and rep["gpu_peel_and_hierarchy_vs_oracle"] == 0.6 / 0.003
    assert rep["oracle_core_equal"] is True
    rep4 = b.pair_report({(2, 4): info[(2, 3)]}, {(2, 4): 2.0}, {(2, 4): 1.0}, {}, 1000.0, oracle_res)["2,4"]
    assert "not run" in rep4["oracle_seconds"]
