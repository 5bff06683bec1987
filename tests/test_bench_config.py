"""The two arms of bench.py describe their workload with one `config` object
(bench.workload_config): the reference arm's line, run here on the CPU for one
step of the oracle, carries exactly the config the GPU arm prints."""
import argparse
import io
import json
import os
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_workload_config_of_the_couette_workload():
    sys.path.insert(0, ROOT)
    import bench
    args = argparse.Namespace(workload="couette", tiles="autotune")
    c = bench.workload_config("couette", args, 1)
    assert c["workload"] == "couette_d2q81_512x256_kn{0.01,0.1,1}"
    assert (c["lattice"], c["k"], c["nodes"], c["instances"]) == ("D2Q81", 3, 512 * 256, 3)
    assert "255 MB > 129 MB L2" in c["l2"]  # 2 buffers x 81 x 512 x 256 x 3 x 4 B
    assert "fit in the 129 MB L2" in bench.workload_config("sod", args, 1)["l2"]
    assert "2 rank(s)" in bench.workload_config("couette", args, 2)["parallelism"]


def test_reference_arm_prints_the_same_config():
    sys.path.insert(0, ROOT)
    import bench
    args = argparse.Namespace(workload="couette", tiles="autotune", steps=1, warmup=0,
                              gpus=1, impl="reference")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["config"] == bench.workload_config("couette", args, 1)
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0
