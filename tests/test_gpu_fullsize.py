"""Parity at the benchmark's full size and launch configuration: the six
512^2 images of the sweep ({Einasto, cored-NFW, Kerr} x i in {17, 80} deg,
a = 0.9, three refinement levels) traced in one batched plan with the default
persistent grids, exactly as bench.py times them, in both precisions.

The oracle cannot trace whole images this size in a test, so sampled base
pixels (most of them refined, where the method does its work) are computed
one by one with their refinement subtrees and compared: the pixel value
within 1e-6 (FP64 path) or 1e-4 (mixed path) of the image maximum, the base
ray's class exactly, except where the oracle shows the class to be
undetermined at the path's precision (the exemption rules of parity.py); a
pixel whose refinement depth differs holds such a ray in its subtree and is
counted, not compared.
"""
import numpy as np
import pytest

from parity import class_sensitive, oracle_class_is_undetermined, oracle_flat, pixel_centre

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_05635_gb300 as B
    B.lib()
    return B


@pytest.mark.parametrize("precision,tol", [(1, 1e-4), (0, 1e-6)])
def test_fullsize_sweep_sampled_pixels(B, oracle, precision, tol):
    from paper_2605_05635_gb300 import workloads
    flats = workloads.sweep_512(precision=precision)
    plan = B.Plan([B.from_flat(d) for d in flats])
    plan.launch()
    plan.check()
    outs = [{k: v.cpu().numpy() for k, v in o.items()} for o in plan.outputs]
    plan.close()
    rng = np.random.default_rng(512 + precision)
    compared, skipped_depth = 0, 0
    for img, d in enumerate(flats):
        g = outs[img]
        refined = np.argwhere(g["refine_level"] > 0)          # (j, i)
        picks = [tuple(refined[k]) for k in rng.choice(len(refined), 5, replace=False)]
        picks += [tuple(x) for x in rng.integers(0, 512, (2, 2))]
        ij = np.array([[i, j] for j, i in picks], dtype=np.int32)
        P = oracle.problem(**{**oracle_flat(d, oracle), "rtol": 1e-10, "atol": 1e-12})
        ref = oracle.trace_pixels(P, ij)
        base = oracle.trace_points(P, [pixel_centre(d, i, j) for i, j in ij])
        scale = float(np.abs(g["I"]).max())
        exempt = class_sensitive if precision == 1 else oracle_class_is_undetermined
        for k, (i, j) in enumerate(ij):
            X, Y = pixel_centre(d, i, j)
            if (g["status"][j, i], g["ncross"][j, i]) != (base[k]["status"], base[k]["ncross"]):
                assert exempt(oracle, d, X, Y), (img, i, j)
                continue
            if g["refine_level"][j, i] != ref["level"][k]:
                skipped_depth += 1
                continue
            assert abs(float(g["I"][j, i]) - ref["val"][k, 0]) <= tol * scale, \
                (img, i, j, float(g["I"][j, i]), ref["val"][k, 0])
            compared += 1
    assert compared >= 30 and skipped_depth <= 6
