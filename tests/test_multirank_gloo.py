"""Host logic of the multi-rank benchmark on CPU: two gloo ranks, each with its
own canyon case (independent problems, no data-path exchange), timed by the
slowest rank; the reference arm runs on rank 0 only."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from canyon_inputs.mesh import canyon_mesh
    from oracle.oracle import Oracle
    from tests.conftest import oracle_params_for

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.env_rank()
    # each rank's own case: the case id changes the Philox key, so the ensembles differ
    mesh = canyon_mesh(offset=0.05, h=0.3, seed=1)
    o = Oracle(oracle_params_for(mesh, seed=5, case_id=r), mesh)
    o.seed(4)
    P = o.particles()
    # per-rank timings; the job is timed by the slowest rank
    my_seconds = 1.0 + 0.5 * r
    t = bench.reduce_max(my_seconds, dist, "cpu")
    value = bench.whole_job_value(w, len(P["x"]), 10, t)
    np.savez(os.path.join(out_dir, f"rank{r}.npz"), u=P["u"], t=t, value=value, world=w, local=local)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_independent_cases_and_max_time(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    a, b = (np.load(tmp_path / f"rank{k}.npz") for k in (0, 1))
    assert int(a["world"]) == 2 and int(b["local"]) == 1
    assert float(a["t"]) == float(b["t"]) == 1.5  # the slowest rank's time on every rank
    n = a["u"].size
    assert float(a["value"]) == pytest.approx(2 * n * 10 / 1.5)
    assert a["u"].shape == b["u"].shape and not np.allclose(a["u"], b["u"])  # different Philox keys


def test_reference_arm_is_rank_zero_only(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(None, None, None, None) is None
    assert capsys.readouterr().out == ""
