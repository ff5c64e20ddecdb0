"""GPU path-replay adjoint (darts_adjoint, autograd) against the FP64 oracle's
score estimator, CRN finite differences of the GPU render, and autograd."""
import dataclasses
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2402_03106_gb300 import scenes as S  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2402_03106_gb300 import capi
    c = capi.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("K", [1, 3, 50])
def test_adjoint_matches_oracle_score(ctx, K):
    """Same seed and paths: the GPU and the oracle accumulate the same
    per-path scores (FP32 vs FP64; near-tie trace flips allowed)."""
    sc, _ = S.cube_workload()
    n = 1 << 16
    sp = S.Sampling(seed=41, paths_per_element=n, max_bounces=K)
    w = np.cos(np.linspace(0.0, 7.0, 256))
    g, q = ctx.adjoint(sc, sp, torch.from_numpy(w), sumsq=True)
    g = g.cpu().numpy()
    q = q.cpu().numpy()
    gref, qref = O.adjoint(sc, sp, w)
    se = np.sqrt(np.maximum(qref - gref ** 2 / n, 0.0))
    # trace flips replace a path by another draw: bounded by a small fraction of one SE
    assert np.all(np.abs(g - gref) <= 0.25 * se + 1e-6 * np.abs(gref)), (g, gref, se)
    np.testing.assert_allclose(q, qref, rtol=0.1)


def test_adjoint_matches_crn_finite_differences(ctx):
    sc = S.slab_scene(1.0, 0.05, 0.4, n_bins=32, t_min=0.85, t_max=3.0)
    n = 1 << 20
    w = np.linspace(1.0, -0.5, 32)
    sp = S.Sampling(seed=7, paths_per_element=n, max_bounces=20)
    g, q = ctx.adjoint(sc, sp, torch.from_numpy(w), sumsq=True)
    g, q = g.cpu().numpy(), q.cpu().numpy()
    se_adj = np.sqrt(np.maximum(q - g ** 2 / n, 0.0))
    h = 1e-3
    nb = 16
    wt = torch.from_numpy(w).cuda()
    for j, name in enumerate(("sigma_s", "sigma_a", "g")):
        fds = []
        for b in range(nb):
            vals = []
            for sgn in (1, -1):
                m = dataclasses.replace(sc.medium, **{name: getattr(sc.medium, name) + sgn * h})
                spb = dataclasses.replace(sp, seed=100 + b, paths_per_element=n // 4)
                hist = ctx.render(dataclasses.replace(sc, medium=m), spb)
                vals.append(float(torch.dot(wt, hist)))
            fds.append((vals[0] - vals[1]) / (2 * h))
        fds = np.array(fds)
        fd, se_fd = fds.mean(), fds.std(ddof=1) / math.sqrt(nb)
        z = (g[j] - fd) / math.sqrt(se_adj[j] ** 2 + se_fd ** 2)
        assert abs(z) < 4.5, (name, g[j], fd, se_adj[j], se_fd)


def test_autograd_function(ctx):
    from paper_2402_03106_gb300 import autograd as A
    sc, _ = S.cube_workload()
    sp = S.Sampling(seed=3, paths_per_element=1 << 18, max_bounces=10)
    params = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in (1.0, 0.01, 0.7)]
    target = torch.zeros(256, dtype=torch.float64, device="cuda")
    h = A.render(*params, sc, sp, adjoint_seed=99, dctx=ctx)
    loss = ((h - target) ** 2).sum()
    loss.backward()
    grads = torch.stack([p.grad for p in params])
    sp_adj = dataclasses.replace(sp, seed=99)
    ref = ctx.adjoint(sc, sp_adj, (2.0 * (h - target)).detach()).cpu()
    torch.testing.assert_close(grads, ref, rtol=1e-6, atol=0.0)
    assert torch.all(torch.isfinite(grads))


def test_adjoint_rejects_baselines(ctx):
    from paper_2402_03106_gb300 import capi
    sc, sp = S.cube_workload(paths=1024)
    sp.method = S.PLAIN_UNIFORM_T
    with pytest.raises(capi.DartsError) as ei:
        ctx.adjoint(sc, sp, torch.ones(256, dtype=torch.float64))
    assert ei.value.status == 6
