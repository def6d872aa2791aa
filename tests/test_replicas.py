"""Multi-rank replica path on CPU: world_size 2 over gloo."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, inputs, out):
    import torch.distributed as dist

    from paper_1807_00699_gb300.replicas import combine_best
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        E, r = inputs[rank]
        out[rank] = combine_best(E, r)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("inputs,expect", [
    ({0: (-10.5, 3), 1: (-12.25, 7)}, (-12.25, 1, 7)),
    ({0: (-3.0, 2), 1: (-3.0, 0)}, (-3.0, 0, 2)),  # tie: lowest rank wins
])
def test_combine_best_gloo_world2(inputs, expect):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(k, 2, port, inputs, out)) for k in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == expect and out[1] == expect
