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


def _camera_worker(rank, world, port, spp, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import oracle as O
        from paper_2402_03106_gb300 import scenes as S, sharding
        sc = S.box_camera_scene(seed=1, width=4, height=4, n_bins=32, t_max=8.0)
        sp = S.Sampling(seed=21, paths_per_element=spp, max_bounces=6)
        n = S.total_paths(sc, sp)
        off = sharding.path_offset(rank, n)
        h, sq, _ = O.render(sc, sp, O.ORC_DARTS, offset=off, threads=2)
        bins = O.trace_paths(sc, sp, off, n)["bin"]
        t = torch.from_numpy(h)
        s2 = torch.from_numpy(sq)
        sharding.combine(t, world)
        dist.all_reduce(s2)
        if rank == 0:
            q.put((t.numpy().copy(), s2.numpy().copy()))
        q.put((rank, bins))
    finally:
        dist.destroy_process_group()


def test_sharded_camera_render_is_a_consistent_estimate():
    """Camera shards (path offset = rank x frame) keep the pixel layout and
    continue the DARTS sample index: their average agrees with a single
    render of world x spp within standard errors, and the ranks' paths land
    on different bins of each pixel."""
    import oracle as O
    from paper_2402_03106_gb300 import scenes as S
    world, spp = 2, 200
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_camera_worker, args=(r, world, port, spp, q)) for r in range(world)]
    for p in procs:
        p.start()
    items = [q.get(timeout=300) for _ in range(world + 1)]
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    hist = [it for it in items if isinstance(it[0], np.ndarray)][0]
    bins = dict(it for it in items if not isinstance(it[0], np.ndarray))
    h, sq = hist
    sc = S.box_camera_scene(seed=1, width=4, height=4, n_bins=32, t_max=8.0)
    sp = S.Sampling(seed=22, paths_per_element=spp * world, max_bounces=6)
    ref, sqref, _ = O.render(sc, sp, O.ORC_DARTS, threads=4)
    # per-pixel totals (sums over bins) with their standard errors
    B = 32
    tot, tref = h.reshape(16, B).sum(1), ref.reshape(16, B).sum(1)
    se = np.sqrt(np.maximum(sq.reshape(16, B).sum(1) / world ** 2, 0.0) / 1.0)
    se_ref = np.sqrt(sqref.reshape(16, B).sum(1))
    z = (tot - tref) / np.sqrt(se ** 2 + se_ref ** 2 + 1e-300)
    assert np.max(np.abs(z)) < 4.5, z
    # rank 1 covers the bins spp further along in each pixel
    b0, b1 = bins[0], bins[1]
    assert np.array_equal(b0 // B, b1 // B)
    assert np.array_equal((b0 % B + spp) % B, b1 % B)


def _pipelined_worker(rank, world, port, n, steps, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import oracle as O
        from paper_2402_03106_gb300 import scenes as S, sharding
        sc, sp = S.cube_workload(paths=n, seed=19)
        sp.max_bounces = 8
        pipe = sharding.PipelinedCombine(lambda: torch.zeros(256, dtype=torch.float64), world)
        seen = []
        for k in range(steps):
            buf = pipe.begin_step()
            seen.append(id(buf))
            h, _, _ = O.render(sc, sp, O.ORC_DARTS, n_paths=n,
                               offset=(k * world + rank) * n, threads=2)
            buf.copy_(torch.from_numpy(h))
            pipe.end_step(buf)
        last = pipe.finish()
        other = [b for b in pipe.buffers if b is not last][0]
        if rank == 0:
            q.put((last.numpy().copy(), other.numpy().copy(), len(set(seen))))
    finally:
        dist.destroy_process_group()


def test_pipelined_combine_averages_the_last_step():
    """Two buffers alternate between steps; each step's render overlaps the
    all-reduce of the previous step's buffer.  After finish() the last
    buffer holds the ranks' average of the last step, equal to a single
    render of its world x n paths."""
    import oracle as O
    from paper_2402_03106_gb300 import scenes as S
    world, n, steps = 2, 2048, 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_pipelined_worker, args=(r, world, port, n, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    got, prev, nbuf = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    assert nbuf == 2
    sc, sp = S.cube_workload(paths=n * world, seed=19)
    sp.max_bounces = 8
    # the last step's ids: [(steps - 1) * world * n, steps * world * n)
    ref, _, _ = O.render(sc, sp, O.ORC_DARTS, n_paths=world * n, offset=(steps - 1) * world * n, threads=4)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-300)
    # the other buffer holds the ranks' sum of the step before, exchanged
    # while the last step rendered
    ref1, _, _ = O.render(sc, sp, O.ORC_DARTS, n_paths=world * n, offset=(steps - 2) * world * n, threads=4)
    np.testing.assert_allclose(prev, world * ref1, rtol=1e-12, atol=1e-300)


def _gradient_worker(rank, world, port, n, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import oracle as O
        from paper_2402_03106_gb300 import scenes as S, sharding
        sc, sp, spa, target = _gradient_case(S)
        off = sharding.path_offset(rank, n)
        h, g = sharding.sharded_gradient(
            lambda: torch.from_numpy(O.render(sc, sp, O.ORC_DARTS, n_paths=n, offset=off, threads=2)[0]),
            lambda w: torch.from_numpy(O.adjoint(sc, spa, w.numpy(), n_paths=n, offset=off, threads=2)[0]),
            lambda h: 2.0 * (h - torch.from_numpy(target)), world)
        if rank == 0:
            q.put((h.numpy().copy(), g.numpy().copy()))
    finally:
        dist.destroy_process_group()


def _gradient_case(S):
    sc, sp = S.cube_workload(paths=1 << 12, seed=23)
    sc.gate.n_bins = 32
    sp.max_bounces = 6
    spa = S.Sampling(seed=24, paths_per_element=sp.paths_per_element, max_bounces=6)
    target = np.linspace(0.0, 0.05, 32)
    return sc, sp, spa, target


def test_sharded_gradient_equals_single_process():
    """Render shards, average the histogram, form the L2 loss weights,
    replay each shard with the adjoint seed, average the gradients: equal to
    one render and one adjoint pass over all the paths."""
    import oracle as O
    from paper_2402_03106_gb300 import scenes as S
    world, n = 2, 4096
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gradient_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    h, g = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    sc, sp, spa, target = _gradient_case(S)
    # one pass over all world x n paths: the per-element budget is world x n
    sp.paths_per_element = spa.paths_per_element = world * n
    href, _, _ = O.render(sc, sp, O.ORC_DARTS, threads=4)
    np.testing.assert_allclose(h, href, rtol=1e-12, atol=1e-300)
    gref, _ = O.adjoint(sc, spa, 2.0 * (href - target), threads=4)
    np.testing.assert_allclose(g, gref, rtol=1e-10, atol=1e-300)
    assert np.all(np.abs(gref) > 0)
