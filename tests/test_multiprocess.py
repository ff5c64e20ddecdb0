"""Multi-rank path of the render on CPU: gloo ranks, world size 2 and 3.

Each rank traces its own path-id range with the FP64 oracle (standing in for
the GPU kernel, which needs a device) and the per-rank estimates are combined
with the same all-reduce helper the benchmark uses.  The result must equal a
single render of all paths.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, method, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import oracle as O
        from paper_2402_03106_gb300 import scenes as S, sharding
        sc, sp = S.cube_workload(paths=n, seed=17)
        sp.method = method
        sp.max_bounces = 10
        h, _, _ = O.render(sc, sp, method, n_paths=n, offset=sharding.path_offset(rank, n), threads=2)
        t = torch.from_numpy(h)
        sharding.combine(t, world)
        if rank == 0:
            q.put(t.numpy().copy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,method", [(2, 0), (3, 0), (2, 1)])
def test_sharded_render_equals_single_render(world, method):
    import oracle as O
    from paper_2402_03106_gb300 import scenes as S
    n = 4096
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, method, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    sc, sp = S.cube_workload(paths=n * world, seed=17)
    sp.method = method
    sp.max_bounces = 10
    ref, _, _ = O.render(sc, sp, method, threads=4)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-300)
