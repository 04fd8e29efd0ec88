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
