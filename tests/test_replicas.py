"""Multi-rank host logic of the replica bench (weak scaling, no data-path
collective), run as two gloo ranks on the CPU: each rank's draw ids and
Philox uniforms are its own, the slowest rank's time is what every rank
reports, and the whole-job rate counts every rank's samples.
"""
import json
import os
import socket

import numpy as np
import pytest

from paper_2301_12584_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    from oracle.philox import sampler_uniforms
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ids = list(replicas.draw_ids(rank, 0, 5))
        elapsed = 10.0 + 7.0 * rank                     # the slower rank sets the job's time
        ms = replicas.max_over_ranks(elapsed, dist, "cpu")
        rate = replicas.whole_job_rate(1000, world, ms)
        u_eig, u_row = sampler_uniforms(1, ids[0], 64, 3)
        with open(os.path.join(out_dir, f"{rank}.json"), "w") as f:
            json.dump({"ids": ids, "ms": ms, "rate": rate, "u": u_eig[:, :8].ravel().tolist()}, f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"{r}.json")) for r in range(world)]
    assert set(res[0]["ids"]).isdisjoint(res[1]["ids"])
    assert res[0]["ms"] == res[1]["ms"] == 17.0
    assert res[0]["rate"] == pytest.approx(2 * 1000 / 0.017)
    assert not np.allclose(res[0]["u"], res[1]["u"])


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.rank_env() == (0, 0, 1)
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.whole_job_rate(65536, 1, 2.0) == pytest.approx(65536 / 0.002)
    with pytest.raises(ValueError):
        replicas.draw_ids(0, replicas.DRAW_STRIDE - 1, 2)
    with pytest.raises(ValueError):
        replicas.whole_job_rate(1, 1, 0.0)
