"""The multi-replica bookkeeping of bench.py on CPU: two gloo ranks, each
with its own step time; both see the slowest rank's time and the whole-job
rate (weak scaling: every rank processes the full workload on its own field).
No GPU, no estimator arithmetic."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out_dir):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms, e2e = times[rank]
        ms_max, e2e_max = bench.max_over_ranks(dist, [ms, e2e])
        rate = bench.whole_job_rate(world, 7885, ms_max / 1e3)
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as fh:
            fh.write("%r %r %r\n" % (ms_max, e2e_max, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_two_gloo_ranks(tmp_path):
    times = [(80.0, 0.09), (95.5, 0.07)]  # rank 1 slowest on device, rank 0 end to end
    mp.spawn(_rank_main, args=(2, _free_port(), times, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        ms_max, e2e_max, rate = (float(v) for v in open(tmp_path / ("rank%d.txt" % r)).read().split())
        assert ms_max == 95.5 and e2e_max == 0.09
        assert rate == pytest.approx(2 * 7885 / 0.0955)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(None, [1.5, 2]) == [1.5, 2.0]
    assert bench.whole_job_rate(1, 10, 2.0) == 5.0


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 times the oracle; other ranks exit 0 and print nothing."""
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(os.path.dirname(HERE), "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
