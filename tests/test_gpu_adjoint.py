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


def test_sigma_a_gradient_is_the_exact_path_length_identity(ctx):
    """With sigma_s fixed every path is attenuated by exp(-sigma_a v t), so
    dh(t)/dsigma_a = -v t h(t) exactly (no diffusion approximation).  With
    the render's own paths (same seed; the adjoint replays them), the
    sigma_a gradient of sum_b h_b equals -v sum_b t_b h_b up to where in its
    bin each contribution falls: |G_a + v sum t_c h| <= v (dt / 2) sum h."""
    sc = S.infinite_scene(10.0, 0.01, 0.3, separation=1.0, n_bins=64, t_min=4.0, t_max=12.0, half_width=1e4)
    sp = S.Sampling(seed=12, paths_per_element=1 << 18, max_bounces=1024)
    h = ctx.render(sc, sp).cpu().numpy()
    g = ctx.adjoint(sc, sp, torch.ones(64, dtype=torch.float64)).cpu().numpy()
    dt = (12.0 - 4.0) / 64
    tc = 4.0 + (np.arange(64) + 0.5) * dt
    est = -np.sum(tc * h)
    assert abs(g[1] - est) <= (0.5 * dt) * h.sum() * 1.001 + 1e-12, (g[1], est, 0.5 * dt * h.sum())
    assert g[1] < 0


def _da_bins(r, edges, ss, sa, g, v=1.0):
    """Time-integrated DA fluence per bin (Eq. 9) and its analytic derivatives
    in sigma_s and sigma_a, by 32-point Gauss-Legendre per bin."""
    xg, wg = np.polynomial.legendre.leggauss(32)
    D = 1.0 / (3.0 * (sa + ss * (1.0 - g)))
    F, Fs, Fa = [], [], []
    for a, b in zip(edges[:-1], edges[1:]):
        t = 0.5 * (a + b) + 0.5 * (b - a) * xg
        w = 0.5 * (b - a) * wg
        phi = v / (4.0 * math.pi * v * D * t) ** 1.5 * np.exp(-r * r / (4.0 * v * D * t) - sa * v * t)
        dlog_dD = -1.5 / D + r * r / (4.0 * v * D * D * t)
        F.append(np.sum(w * phi))
        Fs.append(np.sum(w * phi * dlog_dD * (-3.0 * (1.0 - g) * D * D)))
        Fa.append(np.sum(w * phi * (dlog_dD * (-3.0 * D * D) - v * t)))
    return np.array(F), np.array(Fs), np.array(Fa)


@pytest.mark.parametrize("ss,sa,t0,t1", [(10.0, 0.01, 4.0, 12.0), (5.0, 0.005, 8.0, 24.0)])
def test_adjoint_matches_diffusion_derivative_at_high_albedo(ctx, ss, sa, t0, t1):
    """Albedo 0.999, infinite medium, late times (hundreds of scattering
    events): the transport is diffusive, so the adjoint gradient of the summed
    fluence follows the analytic derivative of the DA Green's function (Eq. 9)
    in sigma_s and sigma_a, within the DA's own accuracy (5 %) and 4 SE."""
    sc = S.infinite_scene(ss, sa, 0.0, separation=1.0, n_bins=8, t_min=t0, t_max=t1, half_width=1e4)
    n = 1 << 20
    sp = S.Sampling(seed=6, paths_per_element=n, max_bounces=1024)
    g, q = ctx.adjoint(sc, sp, torch.ones(8, dtype=torch.float64), sumsq=True)
    g, q = g.cpu().numpy(), q.cpu().numpy()
    se = np.sqrt(np.maximum(q - g * g / n, 0.0))
    F, Fs, Fa = _da_bins(1.0, np.linspace(t0, t1, 9), ss, sa, 0.0)
    h = ctx.render(sc, S.Sampling(seed=7, paths_per_element=n, max_bounces=1024)).cpu().numpy()
    assert abs(h.sum() - F.sum()) <= 0.06 * F.sum()
    for j, ref in ((0, Fs.sum()), (1, Fa.sum())):
        assert abs(g[j] - ref) <= 4.0 * se[j] + 0.05 * abs(ref), (j, g[j], ref, se[j])


def test_differentiable_camera_configuration(ctx):
    """The differentiable configuration: the unit-cube medium seen by a 32x32
    camera, 256 bins, L2 loss against a target rendered at (sigma_s, sigma_a,
    g) = (1.3, 0.02, 0.6); gradient at (1.0, 0.01, 0.7).  The loss gradient's
    weights w = 2 (h - target) come from independent renders, then the adjoint
    of w . h is checked against central differences (step 1e-3, common random
    numbers per seed), within 4.5 combined SE."""
    sc = S.cube_camera_scene(32, 32)
    star = dataclasses.replace(sc, medium=dataclasses.replace(sc.medium, sigma_s=1.3, sigma_a=0.02, g=0.6))
    target = ctx.render(star, S.Sampling(seed=1000, paths_per_element=256, max_bounces=20)).reshape(-1)
    h0 = ctx.render(sc, S.Sampling(seed=1001, paths_per_element=256, max_bounces=20)).reshape(-1)
    w = (2.0 * (h0 - target)).cpu().numpy()
    spa = S.Sampling(seed=7, paths_per_element=256, max_bounces=20)
    n = S.total_paths(sc, spa)
    g, q = ctx.adjoint(sc, spa, torch.from_numpy(w), sumsq=True)
    g, q = g.cpu().numpy(), q.cpu().numpy()
    se_adj = np.sqrt(np.maximum(q - g ** 2 / n, 0.0))
    wt = torch.from_numpy(w).cuda()
    step, nb = 1e-3, 8
    for j, name in enumerate(("sigma_s", "sigma_a", "g")):
        fds = []
        for b in range(nb):
            vals = []
            for sgn in (1, -1):
                m = dataclasses.replace(sc.medium, **{name: getattr(sc.medium, name) + sgn * step})
                spb = S.Sampling(seed=200 + b, paths_per_element=64, max_bounces=20)
                vals.append(float(torch.dot(wt, ctx.render(dataclasses.replace(sc, medium=m), spb).reshape(-1))))
            fds.append((vals[0] - vals[1]) / (2 * step))
        fds = np.array(fds)
        fd, se_fd = fds.mean(), fds.std(ddof=1) / math.sqrt(nb)
        z = (g[j] - fd) / math.sqrt(se_adj[j] ** 2 + se_fd ** 2)
        assert abs(z) < 4.5, (name, g[j], fd, se_adj[j], se_fd)
