"""Host logic of bench.py and the sharding helpers (no device): the
committed ncu summaries belong to the current kernels, the roofline
arithmetic, and the single-rank combine."""
import importlib.util
import os

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("workload,paths", [("spheres_512", 1 << 24), ("box_camera", 65536), ("cube", 1 << 24)])
def test_profiles_match_the_current_kernels(bench, workload, paths):
    """bench.py reports DRAM traffic only from an ncu summary taken on the
    current path-kernel sources; a kernel change without a new capture
    shows up here."""
    t = bench.profiled_traffic(workload, paths)
    assert t is not None, f"profiles/darts_trace_kernel_{workload}.md is stale or missing"
    assert 0 < t < 1e9


@pytest.mark.parametrize("workload", ["spheres_512", "box_camera", "cube"])
def test_roofline_arithmetic(bench, workload):
    """The numerator is the oracle's op count per vertex (profiles/op_counts.md)
    times the vertices the launch reports, over the kernel time."""
    per = {"vertices": 1000.0}
    w = bench.algorithmic_work(workload)
    assert w is not None and w["flops_per_vertex"] > 0
    r = bench.roofline(per, 1.0, workload)
    flops = w["flops_per_vertex"] * 1000
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["flops_per_launch"] == pytest.approx(flops)
    assert r["achieved"] == pytest.approx(flops / 1e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    clock = bench.measured_peaks().get("sm_max_mhz", 2070.0)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * clock * 1e6 / 1e12)


def test_bench_sample_pieces_cover_one_64th_of_the_frame(bench):
    """The oracle's sample of the 512x512 frame: 8 whole rows spread over
    the image, each a contiguous path range of its own window."""
    from paper_2402_03106_gb300 import scenes as S
    pieces, _ = bench.oracle_sample("spheres_512", S)
    assert len(pieces) == 8
    rows = set()
    for first, count, (e0, ne) in pieces:
        assert count == 512 * 64 and ne == 512 and first == e0 * 64 and e0 % 512 == 0
        rows.add(e0 // 512)
    assert len(rows) == 8 and sum(ne for _, _, (_, ne) in pieces) * 64 == 512 * 512


def test_single_rank_combine_is_a_no_op():
    from paper_2402_03106_gb300 import sharding
    pipe = sharding.PipelinedCombine(lambda: torch.zeros(4, dtype=torch.float64), 1)
    assert len(pipe.buffers) == 1
    for k in range(3):
        b = pipe.begin_step()
        b.fill_(k + 1.0)
        pipe.end_step(b)
    assert torch.equal(pipe.finish(), torch.full((4,), 3.0, dtype=torch.float64))
    h = torch.ones(3, dtype=torch.float64)
    assert sharding.combine(h, 1) is h and torch.equal(h, torch.ones(3, dtype=torch.float64))
    assert sharding.path_offset(3, 1000) == 3000
