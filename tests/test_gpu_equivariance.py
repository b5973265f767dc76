"""A sample's result does not depend on the rest of the batch: permuting the
batch permutes the results bit for bit, and a sample solved alone gives the
bits it gets inside the batch (every path, every fused-kernel shape)."""
import numpy as np
import pytest
import torch

from paper_2212_02224_gb300 import scenegen as sg

from gpu_common import planner, to_dev

pytestmark = pytest.mark.gpu


def _solve(prm, sc, p, prec, shape=None):
    pl = planner(prm, prec, max_obs=sc.n_obs, max_samples=len(p))
    if shape:
        pl.set_tuning(*shape)
    xi, r, cu = pl.solve(sc, to_dev(p))
    torch.cuda.synchronize()
    out = xi.cpu().numpy(), r.cpu().numpy(), cu.cpu().numpy()
    pl.close()
    return out


@pytest.mark.parametrize("prec,shape", [("fp64", None), ("fp32", (1, 7)), ("fp32", (2, 2)),
                                        ("fp32", (4, 1)), ("tf32x3", None)])
def test_permuted_batch_permutes_results(prec, shape):
    prm, sc, _ = sg.workload(1, inner_iters=40)
    p = sg.make_samples(515, sc, 61, prm.n_seg)
    perm = np.random.default_rng(3).permutation(len(p))
    a = _solve(prm, sc, p, prec, shape)
    b = _solve(prm, sc, p[perm], prec, shape)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x[perm], y)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sample_alone_matches_sample_in_batch(prec):
    prm, sc, _ = sg.workload(1, inner_iters=40)
    p = sg.make_samples(616, sc, 33, prm.n_seg)
    whole = _solve(prm, sc, p, prec)
    for j in (0, 16, 32):
        alone = _solve(prm, sc, p[j:j + 1], prec)
        for x, y in zip(whole, alone):
            np.testing.assert_array_equal(x[j:j + 1], y)
