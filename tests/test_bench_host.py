"""Host-side logic of bench.py (no GPU): the per-kernel roofline table, the ncu traffic
annotations and JSON serialisation of the line."""
import json

import numpy as np

import bench
from paper_2607_27440_b300 import workloads as wl


def test_kernel_rooflines_c3():
    spec, es = wl.c3()
    groups = {"solve_pass1_df64": (250.0, 2222), "orth1_df": (410.0, 2220), "orth2_dots_df": (220.0, 2220),
              "orth2_update_df": (200.0, 2220), "orth_scale": (30.0, 2220), "rotate": (150.0, 34),
              "schur_qr": (290.0, 35), "cap_solve": (45.0, 2222)}
    infos = [{"restarts": 34, "reorths": 2220}]
    k = bench.kernel_rooflines(groups, spec, es, infos, 1, {"hbm_gbs": 6327.4}, path="df64")
    # cost-modelled groups carry a bound, a peak and a fraction; the rest only their times
    for name in ("solve_pass1_df64", "orth1_df", "orth2_dots_df", "orth2_update_df", "rotate"):
        assert k[name]["peak"] > 0 and 0 < k[name]["frac"] < 2, name
    assert "frac" not in k["schur_qr"] and "frac" not in k["cap_solve"]
    assert k["solve_pass1_df64"]["bound"] == "alu" and k["orth1_df"]["bound"] == "hbm"
    # pass 1 of Gram-Schmidt reads the basis twice per step, the second dots once
    assert abs(k["orth1_df"]["achieved"] * 410.0 / (k["orth2_dots_df"]["achieved"] * 220.0) - 2.0) < 1e-9
    # ncu traffic annotations exist only at the captured size
    assert 0.9 < k["orth1_df"]["ncu_traffic"]["ratio"] < 1.2
    small = bench.kernel_rooflines(groups, wl.c2()[0], wl.c2()[1], infos, 1, {"hbm_gbs": 6327.4}, path="df64")
    assert all("ncu_traffic" not in v for v in small.values())


def test_kernel_rooflines_fp64_path():
    """The float64 path's groups are bounded by the float64 pipe (against the DGEMM peak given)."""
    spec, es = wl.c3()
    groups = {"solve_pass1_c128": (520.0, 1822), "orth1_f32dots_f64update": (450.0, 1820),
              "orth2_f64": (800.0, 1820), "rotate": (570.0, 34), "schur_qr": (300.0, 35)}
    infos = [{"restarts": 34, "reorths": 1820}]
    k = bench.kernel_rooflines(groups, spec, es, infos, 1, {"hbm_gbs": 6327.4}, path="fp64", fp64_peak=1.1)
    for name in ("solve_pass1_c128", "orth1_f32dots_f64update", "orth2_f64", "rotate"):
        assert k[name]["bound"] == "alu" and k[name]["peak"] == 1.1 and 0 < k[name]["frac"] < 2, name
    # the second pass does twice the float64 work of the first per step
    r = (k["orth2_f64"]["achieved"] * 800.0) / (k["orth1_f32dots_f64update"]["achieved"] * 450.0)
    assert abs(r - 2.0) < 1e-9


def test_json_line_serialises_numpy_values():
    line = {"a": np.float64(1.5), "b": np.int64(3), "c": np.arange(3), "d": np.complex128(1 + 2j).real}
    back = json.loads(json.dumps(line, default=bench._jsonable))
    assert back == {"a": 1.5, "b": 3, "c": [0, 1, 2], "d": 1.0}
