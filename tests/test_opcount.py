"""The oracle's op-count mode (oracle/opcount.hpp, oracle/opcount.py).

The roofline numerator of the benchmark is the oracle's own arithmetic per
vertex, tallied by compiling the oracle with a counting number type.  These
tests pin the counting type on expressions whose operation counts are known
by inspection, check that counting does not change the paths the oracle
traces, and that the committed summary profiles/op_counts.md belongs to the
current oracle sources and agrees with a fresh count on a smaller sample.
"""
import json
import os
import subprocess
import textwrap

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_counting_type_tallies_each_operation(tmp_path):
    src = tmp_path / "probe.cc"
    src.write_text(textwrap.dedent("""
        #include <stdio.h>
        static double f(double a, double b) {
          double r = a * b + a / b - sqrt(a);   /* mul 1, div 1, add 2, sqrt 1 */
          r += exp(a) * log1p(b);               /* exp 1, log 1, mul 1, add 1 */
          r = -fabs(r);                         /* not counted */
          if (a < b) r -= 2.0 * 3.0;            /* cmp 1, add 1 (constant folded) */
          double c = 1.5 > b ? 0.0 : r;         /* cmp 1 */
          return c + atan2(a, b) + pow(a, 2.0); /* trig 1, pow 1, add 2 */
        }
        int main() {
          double v = f(1.25, 2.5);
          printf("%d", (int)(v != 0.0));   /* cmp 1 */
          for (int k = 0; k < orc_oc::N; ++k) printf(" %llu", (unsigned long long)orc_oc::tally.n[k]);
          printf("\\n");
          return 0;
        }
    """))
    exe = tmp_path / "probe"
    subprocess.run(["g++", "-std=c++17", "-O0", "-x", "c++", "-include",
                    os.path.join(ROOT, "oracle", "opcount.hpp"), str(src), "-o", str(exe), "-lm"],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    counts = dict(zip(("add", "mul", "div", "sqrt", "cmp", "exp", "log", "trig", "pow", "philox"),
                      map(int, out[1:])))
    assert counts == {"add": 6, "mul": 2, "div": 1, "sqrt": 1, "cmp": 3, "exp": 1, "log": 1,
                      "trig": 1, "pow": 1, "philox": 0}


def test_counted_oracle_traces_the_same_paths():
    import oracle as O
    from oracle import opcount as oc
    from paper_2402_03106_gb300 import scenes as S
    sc = S.spheres_camera_scene(seed=0, width=64, height=64, n_bins=200)
    sp = S.Sampling(seed=3, paths_per_element=4, max_bounces=100)
    t, nv = oc.count_paths(sc, sp, 1000, 1500)
    ref = O.trace_paths(sc, sp, 1000, 1500)
    assert np.array_equal(nv.astype(np.int32), ref["nvert"])
    # every vertex draws at least one Philox block, and every path its init blocks
    assert np.all(t[:, 9] >= nv) and np.all(t[:, 0] > 0)


def test_philox_blocks_per_path_follow_the_layout():
    """K = 1 in the unit cube: a path draws the element block, the emitter
    block (group 2 of the init vertex) and the group-1 block of vertex 0,
    which the oracle evaluates twice (once for the direction, once for the
    connection's S): four blocks.  (The integer count is reported beside the
    roofline, not in its numerator.)"""
    from oracle import opcount as oc
    from paper_2402_03106_gb300 import scenes as S
    sc, sp = S.cube_workload(paths=4096, seed=0)
    sp.max_bounces = 1
    t, nv = oc.count_paths(sc, sp, 0, 256)
    assert np.all(nv == 1)
    assert np.all(t[:, 9] == 4)


def _committed():
    rows = {}
    text = open(os.path.join(ROOT, "profiles", "op_counts.md")).read()
    for line in text.splitlines():
        if line.startswith("data: "):
            d = json.loads(line[6:])
            rows[d["workload"]] = d
    return text, rows


def test_committed_summary_belongs_to_the_current_oracle():
    from oracle import opcount as oc
    text, rows = _committed()
    assert f"oracle_source_hash: {oc.source_hash()}" in text, \
        "profiles/op_counts.md is stale: rerun python oracle/opcount.py"
    assert set(rows) == {"spheres_512", "box_camera", "cube"}


@pytest.mark.parametrize("workload", ["spheres_512", "cube"])
def test_committed_counts_agree_with_a_fresh_smaller_sample(workload):
    from oracle import opcount as oc
    _, rows = _committed()
    fresh = oc.count_workload(workload, fraction=32, workers=1)
    ref = rows[workload]
    for k in ("flops_per_vertex", "special_per_vertex", "int_per_vertex"):
        assert fresh[k] == pytest.approx(ref[k], rel=0.05), k
