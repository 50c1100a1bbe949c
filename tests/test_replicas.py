"""Host logic of the multi-replica bench (one process per GPU, no data-path
collective): the whole-job throughput is the particle-steps of all ranks over
the slowest rank's time.  Two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    p_steps = [3.0e9, 5.0e9][rank]
    ms = [40.0, 50.0][rank]
    value, ms_max = bench.job_throughput(p_steps, ms, dist, device="cpu")
    out[rank] = (value, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_sums_work_over_slowest_rank():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        value, ms_max = res[rank]
        assert ms_max == 50.0
        assert value == pytest.approx((3.0e9 + 5.0e9) / 0.050, rel=1e-12)


def test_job_throughput_single_process():
    import bench
    value, ms = bench.job_throughput(1e9, 20.0)
    assert ms == 20.0 and value == pytest.approx(5e10)
