"""Host logic of bench.py on CPU: rank aggregation over gloo (world size 2) and
the clock-record parser."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    r, w, _ = bench.dist_setup(use_cuda=False)
    bench.barrier()
    out[rank] = bench.max_over_ranks(10.0 + 5.0 * rank)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0] == 15.0 and out[1] == 15.0


def test_single_process_needs_no_process_group():
    assert bench.max_over_ranks(3.5) == 3.5


def test_clock_parser_flags_throttling():
    rows = ["0, 1965, 2070, 1100.5, 0x0, Not Active, Not Active, Not Active, Active",
            "0, 1980, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1400, 2070, 900.0, 0x0, Active, Not Active, Not Active, Not Active"]
    c = bench.parse_clock_csv(rows)
    assert c["sm_mhz"] == 1965.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]


def _tiny_system(n_orb):
    # two atoms of n_orb / 2 orbitals, one pair: only what the roofline helpers read
    half = n_orb // 2
    return {"orb_offset": [0, half, n_orb], "blk_ijl": [[0, 0, 0, 0, 0], [0, 1, 0, 0, 0], [1, 1, 0, 0, 0]]}


def test_roofline_counts_algorithmic_flops_per_product():
    """Separate launches: each tcgen05 product counts 3 split terms x 8 N^3 (unpadded N)."""
    n = 1000
    stats = {"gemm1": (4, 4 * 0.2), "gemm2": (4, 4 * 0.1)}
    tiles = {"product1": {"schedule": "classic, zero k-panels skipped"}, "product2": {"schedule": "classic"}}
    peaks = {"bf16_tflops_sustained": 1000.0, "bf16_tflops": 1200.0}
    p1, p2 = bench.split_product_rooflines([_tiny_system(n)], [1], stats, tiles, peaks)
    assert p1["flops_per_launch"] == 24.0 * n ** 3 and p2["flops_per_launch"] == 24.0 * n ** 3
    assert p1["achieved"] == pytest.approx(24.0 * n ** 3 / 0.2e-3 / 1e12, rel=1e-3)
    assert p1["frac"] == pytest.approx(p1["achieved"] / 1000.0, rel=1e-3)
    assert bench.launches_per_step(tiles) == 6


def test_roofline_of_the_one_launch_products():
    """Both products in one launch: one roofline over 2 x 24 N^3, timed as product 1."""
    n = 512
    stats = {"gemm1": (2, 2 * 0.05), "gemm2": (2, 2 * 0.001)}
    sched = "classic, zero k-panels skipped, both products in one launch"
    tiles = {"product1": {"schedule": sched}, "product2": {"schedule": "classic, both products in one launch"}}
    pc, p2 = bench.split_product_rooflines([_tiny_system(n)], [1], stats, tiles, {"bf16_tflops_sustained": 800.0})
    assert p2 is None
    assert pc["flops_per_launch"] == 48.0 * n ** 3
    assert pc["frac"] == pytest.approx(48.0 * n ** 3 / 0.05e-3 / 1e12 / 800.0, rel=1e-3)
    assert bench.launches_per_step(tiles) == 5
