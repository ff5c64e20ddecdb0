"""The checked build (libdarts_checked.so: every output, tile and table
index tested on the device, DARTS_ERR_BOUNDS instead of an out-of-range
access) runs the main configurations without a single flag and gives the
production build's results.  Each library runs in a process of its own (one
libdarts per process)."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[3])
import torch
from paper_2402_03106_gb300 import capi, scenes as S
capi.load(capi.CHECKED_LIB_PATH if sys.argv[1] == "checked" else capi.LIB_PATH)
ctx = capi.Context(0)
out = {}
sc, sp = S.cube_workload(paths=1 << 16, seed=2)                   # point sensor: shared tiles
h, q = ctx.render(sc, sp, sumsq=True)
out["cube"], out["cube_sq"] = h.cpu().numpy(), q.cpu().numpy()
sc.gate.n_bins = 8192                                              # tiles do not fit: atomics
out["cube_8192"] = ctx.render(sc, sp).cpu().numpy()
cam, spc = S.box_camera_workload(seed=2)                           # camera: per-pixel atomics
spc.paths_per_element = 4
out["camera"] = ctx.render(cam, spc).cpu().numpy()
full = S.Sampling(seed=2, paths_per_element=4, method=S.DARTS_FULL_GATE)
out["full_gate"] = ctx.render(cam, full).cpu().numpy()
w = torch.ones(out["camera"].size, dtype=torch.float64)
out["adjoint"] = ctx.adjoint(cam, spc, w).cpu().numpy()
sv, spv = S.cube_workload(paths=1 << 14, seed=2)                 # RIS variants (trace_var.cu)
for k, fl in enumerate((S.FLAG_IID_CANDIDATES, S.FLAG_EQUIANGULAR, S.FLAG_RESERVOIR, S.FLAG_NO_EDA)):
    spv.flags = fl
    out["variant%d" % k] = ctx.render(sv, spv).cpu().numpy()
sw, spw = S.cube_workload(paths=1 << 14, seed=2)                 # temporal response W
sw.gate.weights = [0.0 if 40 <= b < 200 else 1.0 + (b % 7) for b in range(sw.gate.n_bins)]
for m in (S.DARTS, S.PLAIN_UNIFORM_T):
    spw.method = m
    out["weighted%d" % m] = ctx.render(sw, spw).cpu().numpy()
media = S.batched_media(n_media=6, seed=2, log2_budget=(10.0, 12.0))
outs = ctx.render_batch([m[0] for m in media], [m[1] for m in media])
out["batch"] = torch.cat(outs).cpu().numpy()
ctx.sync()   # raises on any device flag, DARTS_ERR_BOUNDS included
np.savez(sys.argv[2], **out)
"""


def _run(kind, path):
    r = subprocess.run([sys.executable, "-c", SCRIPT, kind, path, ROOT], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(path)


def test_checked_build_raises_no_flag_and_matches(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2402_03106_gb300 import capi
    assert os.path.exists(capi.CHECKED_LIB_PATH)
    chk = _run("checked", str(tmp_path / "checked.npz"))
    prod = _run("production", str(tmp_path / "production.npz"))
    for key in prod.files:
        a, b = chk[key], prod[key]
        assert a.shape == b.shape, key
        assert np.isfinite(a).all(), key
        scale = float(np.abs(b).max()) or 1.0
        # same arithmetic; the atomics' FP64 summation order may differ
        np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-12 * scale, err_msg=key)
        assert float(np.abs(b).sum()) > 0.0, key
