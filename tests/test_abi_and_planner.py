"""C ABI exports and the host planner against the oracle planner (CPU only).

rimo_plan_estimate runs the planner of Section 3.4 on the host without touching a
GPU, so the product's planning decisions are compared here with the oracle's.
"""
import math
import os
import re

import numpy as np
import pytest

import synth
from oracle import plan as opl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "rimo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rimo_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function(rimo_lib):
    names = header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(rimo_lib, n), n


def test_version_and_last_error_without_gpu(rimo_lib):
    assert b"sm_103a" in rimo_lib.rimo_version()
    assert isinstance(rimo_lib.rimo_last_error(), bytes)


def _params(pkg, n, fov, **kw):
    return pkg.default_params(n, n, fov, fov, **kw)


def test_invalid_arguments_are_rejected(rimo_lib):
    import paper_2605_26347_gb300 as pkg
    uvw = synth.make_uvw(100, 60, 1.28e9, 3)
    for bad in (dict(nx=100), dict(oversampling=3), dict(kb_support=6), dict(max_wsupport=11),
                dict(w_norm_frac=0.0), dict(plan_fraction=2.0), dict(tile_size=48), dict(wkernel_table=8),
                dict(wkernel_table=-1)):
        p = _params(pkg, 256, math.radians(1.0))
        for k, v in bad.items():
            setattr(p, k, v)
        with pytest.raises(pkg.RimoError) as e:
            pkg.estimate(uvw, p)
        assert e.value.status == 1


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf, 2.0 ** 60])
@pytest.mark.parametrize("col", [0, 1, 2])
def test_unplaceable_uvw_is_rejected_before_any_device_work(rimo_lib, bad, col):
    # rimo_plan_create checks the coordinates before it touches a GPU, so both calls
    # return INVALID_ARG here
    import ctypes as C
    import paper_2605_26347_gb300 as pkg
    uvw = np.ascontiguousarray(synth.make_uvw(5000, 60, 1.28e9, 3))
    p = _params(pkg, 256, math.radians(1.0), n_wbins=4)
    uvw[4321, col] = bad
    with pytest.raises(pkg.RimoError) as e:
        pkg.estimate(uvw, p)
    assert e.value.status == 1 and b"uvw" in rimo_lib.rimo_last_error()
    out = C.c_void_p()
    st = rimo_lib.rimo_plan_create(uvw.ctypes.data, uvw.shape[0], C.byref(p), None, C.byref(out))
    assert st == 1 and out.value is None and b"uvw" in rimo_lib.rimo_last_error()
    # a large but placeable coordinate still plans
    uvw[4321, col] = 1e12
    assert pkg.estimate(uvw, p)["P"] == 4


@pytest.mark.parametrize("case", [
    dict(n=256, fov=1.0, m=20000, steps=60, seed=1001, bins=4),
    dict(n=256, fov=1.0, m=20000, steps=60, seed=1001, bins=0),
    dict(n=512, fov=2.5, m=60000, steps=28800, seed=77, bins=0, budget=0),
    dict(n=1024, fov=2.5, m=200000, steps=28800, seed=1002, bins=0, budget=40 * 2**30),
])
def test_planner_matches_oracle(case, rimo_lib):
    import paper_2605_26347_gb300 as pkg
    uvw = synth.make_uvw(case["m"], case["steps"], 1.28e9, case["seed"])
    fov = math.radians(case["fov"])
    kw = dict(n_wbins=case["bins"], mem_budget_bytes=case.get("budget", 0))
    est = pkg.estimate(uvw, _params(pkg, case["n"], fov, **kw))
    ref = opl.choose(uvw, opl.PlanParams(nx=case["n"], ny=case["n"], fov_x=fov, fov_y=fov,
                                         n_wbins=case["bins"], mem_budget_bytes=kw["mem_budget_bytes"]))
    assert est["P"] == ref["P"]
    assert est["mode"] == ref["mode"]
    assert est["p_star"] == ref["p_star"]
    assert est["subset"] == ref["subset"]
    m = {d["P"]: d for d in ref["models"]}[est["P"]]
    assert abs(est["est_m_g"] - m["m_G"]) <= 1e-9 * m["m_G"]
    assert abs(est["est_cost"] - m["cost"]) <= 1e-9 * m["cost"]
    assert abs(est["wsclean_p"] - opl.wsclean_bound(uvw[:, 2], fov, fov)) < 1e-9 * est["wsclean_p"]


def _random_cases(n_cases, seed):
    rng = np.random.default_rng(seed)
    for _ in range(n_cases):
        yield dict(n=int(rng.choice([64, 128, 256, 512, 1024])), nyf=int(rng.choice([1, 2])),
                   fov=float(rng.uniform(0.5, 4.0)), m=int(rng.integers(500, 60000)),
                   steps=int(rng.choice([60, 600, 28800])), seed=int(rng.integers(1, 10**6)),
                   bins=int(rng.choice([0, 0, int(rng.integers(1, 48))])),
                   J=int(rng.choice([5, 7, 9])), Sw=int(rng.choice([3, 5, 7, 9])),
                   frac=float(rng.choice([0.01, 0.05, 0.3])), pseed=int(rng.integers(0, 2**40)),
                   budget_frac=float(rng.choice([0.0, 0.5, 1.0, 2.0])))


@pytest.mark.parametrize("case", list(_random_cases(10, 2024)), ids=lambda c: f"n{c['n']}-m{c['m']}-P{c['bins']}")
def test_planner_matches_oracle_on_random_workloads(case, rimo_lib):
    # every planning decision of the host planner (k-means on the sorted subset, per-P
    # models in parallel) against the oracle's plain implementation
    import paper_2605_26347_gb300 as pkg
    uvw = synth.make_uvw(case["m"], case["steps"], 1.28e9, case["seed"])
    nx = case["n"]
    ny = max(64, nx // case["nyf"])
    fx = math.radians(case["fov"])
    fy = fx * ny / nx
    kw = dict(n_wbins=case["bins"], kb_support=case["J"], max_wsupport=case["Sw"],
              plan_fraction=case["frac"], seed=case["pseed"])
    ref0 = opl.choose(uvw, opl.PlanParams(nx=nx, ny=ny, fov_x=fx, fov_y=fy, **kw))
    budget = int(case["budget_frac"] * min(d["m_G"] for d in ref0["models"]))
    ref = opl.choose(uvw, opl.PlanParams(nx=nx, ny=ny, fov_x=fx, fov_y=fy, mem_budget_bytes=budget, **kw))
    est = pkg.estimate(uvw, pkg.default_params(nx, ny, fx, fy, mem_budget_bytes=budget, **kw))
    assert (est["P"], est["mode"], est["p_star"], est["subset"]) == (ref["P"], ref["mode"], ref["p_star"], ref["subset"])
    m = {d["P"]: d for d in ref["models"]}[est["P"]]
    assert abs(est["est_m_g"] - m["m_G"]) <= 1e-9 * m["m_G"]
    assert abs(est["est_cost"] - m["cost"]) <= 1e-9 * m["cost"]
    assert est["truncated"] == int(m["truncated"])


def test_planner_budget_regimes_match_oracle(rimo_lib):
    # Fig. 2 regimes forced by the budget: stored G at P*, nearest feasible P, holographic
    import paper_2605_26347_gb300 as pkg
    uvw = synth.make_uvw(30000, 60, 1.28e9, 5)
    fov = math.radians(1.0)
    ref = opl.choose(uvw, opl.PlanParams(nx=256, ny=256, fov_x=fov, fov_y=fov))
    mG = sorted(d["m_G"] for d in ref["models"])
    for budget in (0, int(mG[len(mG) // 2]), int(mG[0] * 1.0001), 1000):
        est = pkg.estimate(uvw, _params(pkg, 256, fov, mem_budget_bytes=budget))
        r = opl.choose(uvw, opl.PlanParams(nx=256, ny=256, fov_x=fov, fov_y=fov, mem_budget_bytes=budget))
        assert (est["P"], est["mode"]) == (r["P"], r["mode"]), budget


def test_briggs_weights_match_oracle_on_the_host(rimo_lib):
    # host logic of the library (no GPU): Briggs' robust weights against the oracle's
    import paper_2605_26347_gb300 as pkg
    from oracle import weighting
    uvw = synth.make_uvw(20000, 60, 1.28e9, 9)
    fov = math.radians(1.5)
    for R in (-2.0, 0.0, 0.5, 2.0):
        got = pkg.briggs_weights(uvw, 128, 96, fov, 0.8 * fov, R)
        want = weighting.briggs_weights(uvw, 128, 96, fov, 0.8 * fov, R)
        assert np.max(np.abs(got - want) / want) < 1e-6, R
    with pytest.raises(pkg.RimoError):
        pkg.briggs_weights(uvw, 0, 96, fov, fov, 0.0)
    bad = uvw.copy()
    bad[3, 0] = np.nan
    with pytest.raises(pkg.RimoError):
        pkg.briggs_weights(bad, 128, 96, fov, fov, 0.0)


def test_python_structures_match_the_c_header(tmp_path, rimo_lib):
    # the ctypes views of rimo_plan_params and rimo_plan_info against the header's layout,
    # compiled by the host C compiler (sizes and every field offset)
    import ctypes as C
    import shutil
    import subprocess
    from paper_2605_26347_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rimo.h"', 'int main(void) {']
    for cname, py in (("rimo_plan_params", _lib.PlanParams), ("rimo_plan_info", _lib.PlanInfo)):
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    want = {}
    for line in out:
        if line:
            name, field, val = line.split()
            want[(name, field)] = int(val)
    for cname, py in (("rimo_plan_params", _lib.PlanParams), ("rimo_plan_info", _lib.PlanInfo)):
        assert C.sizeof(py) == want[(cname, "size")], cname
        for f, _ in py._fields_:
            assert getattr(py, f).offset == want[(cname, f)], (cname, f)


def test_product_path_fails_loudly_without_the_library(tmp_path):
    # no fallback: every entry point needs librimo.so, and its absence is an ImportError
    import subprocess
    import sys
    code = ("import math, numpy as np, paper_2605_26347_gb300 as pkg\n"
            "uvw = np.zeros((10, 3))\n"
            "pkg.estimate(uvw, pkg.default_params(64, 64, 0.01, 0.01))\n")
    env = dict(os.environ, RIMO_LIBRARY=str(tmp_path / "librimo.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "build the CUDA library first" in r.stderr
