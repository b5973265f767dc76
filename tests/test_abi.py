"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every function include/plan.h declares, and plan_init rejects invalid
configurations before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2212_02224_gb300 import binding, build, scenegen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding.load()


def _declared():
    hdr = open(os.path.join(ROOT, "include", "plan.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(plan_[a-z0-9_]+)\s*\(", hdr)))


def test_header_declares_the_binding_names():
    assert _declared() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = _lib()
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings():
    lib = _lib()
    assert lib.plan_status_str(0) == b"ok"
    assert lib.plan_status_str(binding.PLAN_ECAPACITY) == b"capacity exceeded"
    assert lib.plan_status_str(12345) == b"unknown status"


@pytest.mark.parametrize("field,value,needle", [
    ("m", 4, "m must be"),
    ("n_coef", 17, "n_coef"),
    ("n_seg", 5, "n_seg"),
    ("inner_iters", 0, "inner_iters"),
    ("n_elite", 0, "n_elite"),
    ("eta", 0.0, "eta"),
    ("v_max", 0.05, "v_min < v_max"),
    ("n_elite_c", 4096, "2048"),
])
def test_init_rejects_invalid_config(field, value, needle):
    lib = _lib()
    prm = scenegen.Params()
    cfg = binding.make_config(prm, binding.PLAN_PREC_FP32, 8, 64)
    setattr(cfg, field, value)
    ctx = ctypes.c_void_p()
    st = lib.plan_init(ctypes.byref(cfg), ctypes.byref(ctx))
    assert st == binding.PLAN_EINVAL
    assert ctx.value is None
    assert needle in binding.last_error(None)


def test_fp32_kernel_coefficient_counts():
    lib = _lib()
    prm = scenegen.Params(n_coef=9)
    cfg = binding.make_config(prm, binding.PLAN_PREC_FP32, 8, 64)
    ctx = ctypes.c_void_p()
    assert lib.plan_init(ctypes.byref(cfg), ctypes.byref(ctx)) == binding.PLAN_EINVAL
    assert "n_coef" in binding.last_error(None)


def test_null_context_is_rejected():
    lib = _lib()
    assert lib.plan_solve(None, None, None, 0, None, None, None, None, None) == binding.PLAN_EINVAL
    assert lib.plan_destroy(None) == binding.PLAN_OK


@pytest.mark.parametrize("prec", [binding.PLAN_PREC_TF32, binding.PLAN_PREC_BF16,
                                  binding.PLAN_PREC_TF32X3])
def test_tensor_core_modes_need_short_horizons(prec):
    lib = _lib()
    prm = scenegen.Params(m=200)
    cfg = binding.make_config(prm, prec, 8, 64)
    ctx = ctypes.c_void_p()
    assert lib.plan_init(ctypes.byref(cfg), ctypes.byref(ctx)) == binding.PLAN_EINVAL
    assert "m <= 128" in binding.last_error(None)


def test_unknown_precision_is_rejected():
    lib = _lib()
    cfg = binding.make_config(scenegen.Params(), 5, 8, 64)
    ctx = ctypes.c_void_p()
    assert lib.plan_init(ctypes.byref(cfg), ctypes.byref(ctx)) == binding.PLAN_EINVAL
    assert "prec" in binding.last_error(None)


def test_diagnostics_check_their_arguments_before_the_device():
    lib = _lib()
    assert lib.plan_probe_alu(None, None) == binding.PLAN_EINVAL
    for bad in (0, 100001):
        assert lib.plan_probe_wait_timeout(bad, None) == binding.PLAN_EINVAL
        assert "wait_us" in binding.last_error(None)


@pytest.mark.parametrize("what", ["ego_nan", "obstacle_inf", "kappa_road_nan", "a_max", "c_max",
                                  "lane_margin", "goal_narrow_basis", "goal_flag"])
def test_noalloc_rejects_what_plan_solve_rejects(what):
    """The allocation-free entry point checks its configuration and scene as
    plan_init and plan_solve do; these rejections happen before any device
    call, so they run without a GPU."""
    lib = _lib()
    prm = scenegen.Params()
    sc = scenegen.make_scene(5, n_lanes=3, n_obs=2)
    if what == "ego_nan":
        sc.ego[2] = float("nan")
    elif what == "obstacle_inf":
        sc.obstacles[1, 0] = float("inf")
    elif what == "kappa_road_nan":
        sc.kappa_road = float("nan")
    elif what == "a_max":
        prm.a_max = 0.0
    elif what == "c_max":
        prm.c_max = -1.0
    elif what == "lane_margin":
        prm.lane_margin = -0.5
    elif what == "goal_narrow_basis":
        prm.goal, prm.n_coef = True, 5
    cfg = binding.make_config(prm, binding.PLAN_PREC_FP64, 8, 8)
    if what == "goal_flag":
        cfg.goal = 2
    arr, keep = binding.make_scenes([sc])
    st = lib.plan_solve_fp64_noalloc(ctypes.byref(cfg), arr, None, 0, None, None, None, None)
    assert st == binding.PLAN_EINVAL, binding.last_error(None)
