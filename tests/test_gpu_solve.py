"""Parity of the lower-level solve (Step 1, Alg. 2, scoring) through the C ABI
against the FP64 oracle, for both the plain FP64 path and the fused FP32
kernel.  Sizes span several tiles and a ragged last slot of timesteps."""
import numpy as np
import pytest
import torch

from oracle import lower
from oracle.basis import bernstein
from paper_2212_02224_gb300 import binding, scenegen as sg

from gpu_common import compare, planner, scene_with, to_dev

pytestmark = pytest.mark.gpu
PRECS = ["fp64", "fp32"]


def _run(prec, prm, sc, p, max_obs=32):
    pl = planner(prm, prec, max_obs=max_obs, max_samples=max(len(p), 1))
    xi, r, cu = pl.solve(sc, to_dev(p))
    torch.cuda.synchronize()
    out = xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy()
    pl.close()
    return out


def _oracle(prm, sc, p):
    return lower.solve(p, sc, prm, bernstein(prm.m, prm.n_coef, prm.dt))


@pytest.mark.parametrize("prec", PRECS)
def test_small_plain_workload(prec):
    """2 lanes, 4 obstacles, B = 64, 50 iterations."""
    prm, sc, B = sg.workload(0)
    p = sg.make_samples(101, sc, B, prm.n_seg)
    compare(prec, prm, *_run(prec, prm, sc, p), *_oracle(prm, sc, p), sc=sc, p=p)


@pytest.mark.parametrize("prec", PRECS)
def test_dense_traffic_scene(prec):
    """4 lanes, 12 obstacles, 100 iterations, 96 samples."""
    prm, sc, _ = sg.workload(1)
    p = sg.make_samples(202, sc, 96, prm.n_seg)
    compare(prec, prm, *_run(prec, prm, sc, p), *_oracle(prm, sc, p), sc=sc, p=p)


@pytest.mark.parametrize("prec", PRECS)
def test_dense_traffic_full_batch(prec):
    """Full size (B = 1000, the bench's launch) on the GPU; every sample is
    compared with the oracle."""
    prm, sc, B = sg.workload(1)
    p = sg.make_samples(303, sc, B, prm.n_seg)
    compare(prec, prm, *_run(prec, prm, sc, p), *_oracle(prm, sc, p), sc=sc, p=p)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["no_obstacles", "single_sample", "four_segments",
                                  "ragged_horizon", "wide_basis", "static_obstacles"])
def test_edge_cases(prec, case):
    if case == "no_obstacles":
        prm, sc, _ = sg.workload(0, inner_iters=30)
        sc.obstacles = np.zeros((0, 6))
        p = sg.make_samples(1, sc, 40, prm.n_seg)
    elif case == "single_sample":
        prm, sc, _ = sg.workload(1, inner_iters=40)
        p = sg.make_samples(2, sc, 1, prm.n_seg)
    elif case == "four_segments":
        prm, sc, _ = sg.workload(1, inner_iters=40, n_seg=4)
        p = sg.make_samples(3, sc, 50, 4)
    elif case == "ragged_horizon":
        prm = sg.Params(m=37, n_coef=8, inner_iters=30)
        sc = scene_with(4, 3, 5, obs_x=(5.0, 30.0))
        p = sg.make_samples(4, sc, 33, 1)
    elif case == "wide_basis":
        prm, sc, _ = sg.workload(4, inner_iters=40)
        p = sg.make_samples(5, sc, 20, prm.n_seg)
    else:
        prm = sg.Params(m=100, n_coef=11, inner_iters=60)
        sc = scene_with(6, 3, 6, obs_x=(12.0, 50.0), obs_vx=(0.0, 0.0))
        p = sg.make_samples(6, sc, 70, 1)
    compare(prec, prm, *_run(prec, prm, sc, p, max_obs=max(sc.n_obs, 1)), *_oracle(prm, sc, p), sc=sc, p=p)


@pytest.mark.parametrize("prec,shape", [("fp64", None), ("fp32", None), ("fp32", (2, 1)),
                                         ("fp32", (4, 1))])
def test_maximum_obstacle_count(prec, shape):
    """64 obstacles, the largest scene the library accepts: the fused kernel
    walks its obstacle tables in two chunks of 32, and points of the
    trajectories fall inside obstacles of both chunks."""
    prm = sg.Params(m=100, n_coef=11, inner_iters=20)
    sc = scene_with(64064, 4, 64, obs_x=(8.0, 260.0))
    p = sg.make_samples(65, sc, 40, 1)
    pl = planner(prm, prec, max_obs=64, max_samples=len(p))
    if shape:
        pl.set_tuning(*shape)
    xi, r, cu = pl.solve(sc, to_dev(p))
    torch.cuda.synchronize()
    out = xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy()
    pl.close()
    compare(prec, prm, *out, *_oracle(prm, sc, p), sc=sc, p=p)


@pytest.mark.parametrize("prec,shape", [("fp64", None), ("fp32", None), ("fp32", (1, 8)),
                                         ("fp32", (2, 4))])
def test_longest_horizon(prec, shape):
    """m = 256 timesteps with 16 coefficients, the largest horizon and basis
    the fused kernel takes: eight full timestep slots per lane for one warp
    per sample, and the most shared memory per CTA at eight samples per CTA."""
    prm = sg.Params(m=256, n_coef=16, inner_iters=20)
    sc = scene_with(256, 4, 10, obs_x=(10.0, 200.0))
    p = sg.make_samples(257, sc, 16, 1)
    pl = planner(prm, prec, max_obs=10, max_samples=len(p))
    if shape:
        pl.set_tuning(*shape)
    xi, r, cu = pl.solve(sc, to_dev(p))
    torch.cuda.synchronize()
    out = xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy()
    pl.close()
    compare(prec, prm, *out, *_oracle(prm, sc, p), sc=sc, p=p)


@pytest.mark.parametrize("prec", PRECS)
def test_batched_scenes_uneven(prec):
    """Several scenes of uneven obstacle and sample counts in one call."""
    prm, scenes, Bs = sg.batched_workload(S=5, seed=77, B_range=(1, 40), N_range=(0, 14),
                                          inner_iters=40)
    ps = [sg.make_samples(500 + i, scenes[i], Bs[i], prm.n_seg) for i in range(5)]
    pl = planner(prm, prec, max_obs=20, max_samples=sum(Bs), max_scenes=5)
    xi, r, cu = pl.solve_batch(scenes, Bs, to_dev(np.concatenate(ps)))
    torch.cuda.synchronize()
    xi, r, cu = xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy()
    pl.close()
    off = 0
    for i in range(5):
        sl = slice(off, off + Bs[i])
        compare(prec, prm, xi[sl], r[sl], cu[sl], *_oracle(prm, scenes[i], ps[i]), sc=scenes[i], p=ps[i])
        off += Bs[i]


def test_capacity_and_argument_errors():
    prm, sc, _ = sg.workload(0)
    pl = planner(prm, "fp32", max_obs=2, max_samples=16)
    p = to_dev(sg.make_samples(1, sc, 32, 1))
    with pytest.raises(binding.PlanError) as e:
        pl.solve(sc, p)           # 4 obstacles > max_obs
    assert e.value.status == binding.PLAN_ECAPACITY
    sc.obstacles = sc.obstacles[:2]
    with pytest.raises(binding.PlanError) as e:
        pl.solve(sc, p)           # 32 samples > max_samples
    assert e.value.status == binding.PLAN_ECAPACITY
    bad = sg.make_scene(1, n_lanes=2, n_obs=1)
    bad.obstacles[0, 4] = 0.0     # zero ellipse axis
    with pytest.raises(binding.PlanError) as e:
        pl.solve(bad, p[:4].contiguous())
    assert e.value.status == binding.PLAN_EINVAL
    xi, r, cu = pl.solve(sc, p[:0].contiguous())   # B = 0 is a no-op
    assert r.numel() == 0
    pl.close()


SHAPES = [(1, 1), (1, 4), (1, 8), (2, 1), (2, 2), (2, 4), (4, 1)]


@pytest.fixture(scope="module")
def dense_case():
    prm, sc, _ = sg.workload(1, inner_iters=60)
    p = sg.make_samples(404, sc, 45, prm.n_seg)
    return prm, sc, p, _oracle(prm, sc, p)


@pytest.mark.parametrize("wps,spc", SHAPES)
def test_fused_kernel_shapes(wps, spc, dense_case):
    """Every warps-per-sample / samples-per-CTA shape gives oracle parity."""
    prm, sc, p, ref = dense_case
    pl = planner(prm, "fp32", max_obs=16, max_samples=len(p))
    pl.set_tuning(wps, spc)
    xi, r, cu = pl.solve(sc, to_dev(p))
    torch.cuda.synchronize()
    compare("fp32", prm, xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy(), *ref, sc=sc, p=p)
    pl.close()


@pytest.mark.parametrize("wps,spc", [(1, 1), (2, 1), (2, 2), (4, 1)])
def test_long_and_ragged_horizons_per_shape(wps, spc):
    for m, n in ((37, 8), (200, 16)):
        prm = sg.Params(m=m, n_coef=n, inner_iters=25)
        sc = scene_with(40 + m, 4, 7, obs_x=(8.0, 60.0))
        p = sg.make_samples(41, sc, 9, 1)
        pl = planner(prm, "fp32", max_obs=8, max_samples=9)
        pl.set_tuning(wps, spc)
        xi, r, cu = pl.solve(sc, to_dev(p))
        torch.cuda.synchronize()
        compare("fp32", prm, xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy(),
                *_oracle(prm, sc, p), sc=sc, p=p)
        pl.close()


def test_autotune_returns_a_valid_shape(tmp_path, monkeypatch):
    prm, sc, B = sg.workload(1, inner_iters=10)
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("PLAN_TUNE_CACHE", str(cache))
    pl = planner(prm, "fp32", max_obs=16, max_samples=256)
    w, s = pl.autotune(sc, 256)
    assert (w, s) in {(1, 1), (1, 2), (1, 4), (1, 5), (1, 6), (1, 7), (1, 8), (2, 1), (2, 2), (2, 4),
                      (4, 1)}
    assert cache.read_text().split()[4:6] == [str(w), str(s)]
    assert pl.autotune(sc, 256) == (w, s)          # served from the cache file
    with pytest.raises(binding.PlanError):
        pl.set_tuning(3, 1)
    pl.close()


def test_arithmetic_probe():
    """The roofline's denominators measured on the device: positive, the SM
    count of the device, FP32 FMA no faster than SMs x 128 lanes x 2 flop at
    the maximum SM clock (a little slack for clock reporting)."""
    out = binding.plan_probe_alu()
    props = torch.cuda.get_device_properties(0)
    assert out["sms"] == props.multi_processor_count
    assert out["fp32_tflops"] > 0 and out["fp64_tflops"] > 0 and out["rsqrt_tops"] > 0
    assert out["fp32_tflops"] <= 1.1 * out["sms"] * 128 * 2 * 2.1e9 / 1e12


def test_repeated_solves_reuse_or_refresh_the_upload():
    """plan_solve skips re-uploading scenes whose bytes equal the previous
    call's (it waits on that upload's event instead).  Alternating scenes,
    sample counts and streams must each give the result of a fresh context."""
    prm, sc1, _ = sg.workload(1, inner_iters=20)
    sc2 = scene_with(77, 4, 9, obs_x=(10.0, 60.0))
    p1 = to_dev(sg.make_samples(81, sc1, 64, prm.n_seg))
    p2 = to_dev(sg.make_samples(82, sc2, 48, prm.n_seg))
    ref = {}
    for name, sc, p in (("a", sc1, p1), ("b", sc2, p2)):
        pl = planner(prm, "fp32", max_obs=16, max_samples=64)
        ref[name] = [t.cpu().numpy() for t in pl.solve(sc, p)]
        pl.close()
    pl = planner(prm, "fp32", max_obs=16, max_samples=64)
    side = torch.cuda.Stream()
    for name, sc, p, stream in (("a", sc1, p1, None), ("a", sc1, p1, None), ("b", sc2, p2, None),
                                ("a", sc1, p1, side), ("a", sc1, p1, None), ("b", sc2, p2, side)):
        if stream is not None:
            stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(stream):
                out = pl.solve(sc, p, stream=stream)
            torch.cuda.current_stream().wait_stream(stream)
        else:
            out = pl.solve(sc, p)
        torch.cuda.synchronize()
        for got, want in zip(out, ref[name]):
            assert np.array_equal(got.cpu().numpy(), want)
    pl.close()
