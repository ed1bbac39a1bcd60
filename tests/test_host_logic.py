"""Host-side logic that needs no GPU: the autotuner's problem classes and saved table, the
library build reusing only objects that are up to date and made on this kind of machine, the
cache layout and geometry helpers against the oracle, and the binding's tensor checks."""
import json
import os
import shutil
import time

import pytest


def test_autotuner_buckets_problem_classes():
    from paper_1904_08463_gb300.autotune import Autotuner

    # plane and visibility counts fall into power-of-two buckets; sizes and supports do not
    assert Autotuner.key("grid", 4096, 512, 127, 8388608) == "grid:N4096:P512:S127:V8388608"
    assert Autotuner.key("grid", 4096, 300, 127, 5_000_000) == "grid:N4096:P512:S127:V8388608"
    assert Autotuner.key("grid", 4096, 257, 127, 1) == "grid:N4096:P512:S127:V1"
    assert Autotuner.key("grid", 4096, 256, 127, 0) == "grid:N4096:P256:S127:V0"
    assert Autotuner.key("kernelgen", 1024, 33, 63) != Autotuner.key("kernelgen", 1024, 33, 127)


def test_autotuner_table_round_trip_answers_without_timing(tmp_path):
    from paper_1904_08463_gb300.autotune import Autotuner

    path = str(tmp_path / "tune.json")
    t = Autotuner(path)
    key = Autotuner.key("grid", 2048, 64, 63, 100_000)
    t.table[key] = {"best": [9, 64], "ms": {"[9, 64]": 1.0, "[3, 64]": 2.0}}
    t.save()
    assert json.load(open(path))[key]["best"] == [9, 64]

    def run(_):
        raise AssertionError("a tuned class is never timed again")

    again = Autotuner(path)
    assert again.choose(key, [[3, 64], [9, 64]], run) == [9, 64]


@pytest.mark.skipif(not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")), reason="needs nvcc")
def test_build_recompiles_only_stale_objects_and_never_foreign_ones():
    from paper_1904_08463_gb300 import build

    build.build()
    objs = {os.path.basename(s): os.path.join(build.BUILD, os.path.basename(s) + ".o") for s in build.sources()}
    before = {k: os.path.getmtime(o) for k, o in objs.items()}
    # a touched source: only its own object is rebuilt
    src = os.path.join(build.CSRC, "planes.cu")
    time.sleep(1.1)
    os.utime(src, None)
    build.build()
    after = {k: os.path.getmtime(o) for k, o in objs.items()}
    assert after["planes.cu"] > before["planes.cu"]
    assert all(after[k] == before[k] for k in objs if k != "planes.cu")
    # objects stamped for another machine or other flags are never reused
    stamp = os.path.join(build.BUILD, "stamp.txt")
    good = open(stamp).read()
    try:
        with open(stamp, "w") as fh:
            fh.write("another-machine " + good)
        time.sleep(1.1)
        os.utime(src, None)
        build.build()
        rebuilt = {k: os.path.getmtime(o) for k, o in objs.items()}
        assert all(rebuilt[k] > after[k] for k in objs)
        assert open(stamp).read() == good
    finally:
        if open(stamp).read() != good:
            with open(stamp, "w") as fh:
                fh.write(good)


def test_python_layout_and_geometry_agree_with_the_oracle():
    """The library's host helpers through the Python binding: the compact cache layout of given
    supports and the derived geometry equal the oracle's (os^2 (2S+1)^2 taps per plane; K_out,
    du, r_max from the plan)."""
    import numpy as np

    import paper_1904_08463_gb300 as wp
    from oracle import oracle as o

    rng = np.random.default_rng(5)
    for N, os_, s_max in ((256, 8, 15), (4096, 8, 127), (640, 2, 140), (96, 5, 12)):
        dl = np.deg2rad(4.0) / N
        plan = wp.Plan(N, dl, os_, s_max, 1, 0.0, 512)
        g = o.Geometry(N, dl, os_, s_max, 1, 0.0, 512)
        sup = rng.integers(1, s_max + 1, 17)
        assert wp.api.kernel_layout(plan, sup.tolist()) == o.layout(g, sup).tolist()
        assert wp.api.kernel_layout_max(plan, 3) == [0, *(o.layout(g, [s_max] * 3)[1:]).tolist()]
        geo = plan.geometry()
        assert geo.k_out == g.k_out
        assert geo.du == pytest.approx(g.du, rel=1e-15) and geo.r_max == pytest.approx(g.r_max, rel=1e-15)


def test_python_binding_refuses_host_tensors_before_any_device_work():
    import torch

    import paper_1904_08463_gb300 as wp

    with pytest.raises(ValueError, match="CUDA tensor"):
        wp.plane_values(torch.zeros(30, dtype=torch.float32), 4)
