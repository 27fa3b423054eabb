"""Batched sweeps: one persistent launch per refinement level over many
images, plans replayed as CUDA graphs, and the autotuner.

Every ray's computation is independent of the schedule, so a batch must give
bit-identical planes to the same images traced one by one; the refinement
key sets must match too.  A sample of the 96-image sweep (jittered halo
parameters, mixed metrics) is checked against the oracle pixel by pixel.
"""
import math

import numpy as np
import pytest

from parity import oracle_class_is_undetermined, oracle_flat, pixel_centre

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_05635_gb300 as B
    B.lib()
    return B


def _np(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_single_images(B, precision):
    from paper_2605_05635_gb300 import workloads
    flats = workloads.sweep_96(n=20)[::9]        # 11 images, all metrics, spins, inclinations
    for d in flats:
        d.update(levels=2)
        if precision == 1:
            d.update(workloads.MIXED_INTEG)
    items = [B.from_flat(d) for d in flats]
    batch = [_np(o) for o in B.trace_batch(items, keys_cap=1 << 18)]
    for it, b in zip(items, batch):
        single = _np(B.trace_batch([it], keys_cap=1 << 18)[0])
        for k in ("I", "I_n", "ncross", "status", "refine_level", "R_em", "g"):
            assert np.array_equal(b[k], single[k]), k
        assert np.array_equal(np.sort(b["refine_keys"]), np.sort(single["refine_keys"]))


def test_plan_graph_replay_and_autotune(B):
    import torch
    from paper_2605_05635_gb300 import workloads
    flats = workloads.sweep_96(n=24)[::16]
    items = [B.from_flat(d) for d in flats]
    plan = B.Plan(items)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.launch(use_graph=False, stream=s)
        ref = [_np(o) for o in plan.outputs]
        plan.launch(use_graph=True, stream=s)    # capture + first replay
        plan.launch(use_graph=True, stream=s)    # replay
        s.synchronize()
        plan.check(s)
        for o, r in zip(plan.outputs, ref):
            for k in ("I", "ncross", "status", "refine_level"):
                assert np.array_equal(o[k].cpu().numpy(), r[k])
        rep = plan.autotune(stream=s)
        assert rep["candidates"] >= 2 and rep["blocks"][0] > 0
        plan.launch(use_graph=True, stream=s)
        s.synchronize()
        for o, r in zip(plan.outputs, ref):
            assert np.array_equal(o["I"].cpu().numpy(), r["I"])
        st = plan.stats(s)
        assert st["status"] == 0 and sum(st["rays"]) >= sum(st["cells"][:1])
    plan.close()


def test_sweep96_sampled_pixels_match_oracle(B, oracle):
    """96 images (3 metrics x 8 spins x 4 inclinations, jittered halos) at a
    reduced 32^2 with one refinement level (a screen this coarse refines most
    of its pixels), one batched FP64 call; sampled pixels (value, class, depth)
    against the oracle's per-pixel computation."""
    from paper_2605_05635_gb300 import workloads
    flats = workloads.sweep_96(n=32)
    for d in flats:
        d.update(levels=1)
    items = [B.from_flat(d) for d in flats]
    outs = [_np(o) for o in B.trace_batch(items)]
    rng = np.random.default_rng(9)
    checked = 0
    for k in rng.choice(len(flats), 12, replace=False):
        d = flats[k]
        P = oracle.problem(**oracle_flat(d, oracle))
        scale = max(float(np.abs(outs[k]["I"]).max()), 1e-30)
        for _ in range(3):
            i, j = (int(x) for x in rng.integers(0, 32, 2))
            px = oracle.trace_pixel(P, i, j)
            g = outs[k]
            if (g["status"][j, i], g["ncross"][j, i]) != (px["status"], px["ncross"]):
                assert oracle_class_is_undetermined(oracle, d, *pixel_centre(d, i, j))
                continue
            if g["refine_level"][j, i] != px["level"]:
                continue  # a refined descendant's class is undetermined
            assert abs(g["I"][j, i] - px["I"]) <= 1e-6 * scale
            checked += 1
    assert checked >= 25


def test_plan_fixed_launch_shapes_give_identical_planes(B):
    """Every ray's computation is independent of the persistent grid: a plan
    confined to a small grid (and either kernel build) gives the same planes
    bit for bit."""
    import torch
    from paper_2605_05635_gb300 import workloads
    flats = workloads.sweep_96(n=24)[::24]
    for d in flats:
        d.update(workloads.MIXED_INTEG)
    plan = B.Plan([B.from_flat(d) for d in flats])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.launch(stream=s)
        ref = [_np(o) for o in plan.outputs]
        for shape in ((0, 152, 64, 1, 1, 76, 128, 1), (0, 19, 128, 0, 1, 38, 64, 0)):
            plan.set_launch(*shape[:4])
            plan.set_launch(*shape[4:])
            plan.launch(stream=s)
            plan.check(s)
            for o, r in zip(plan.outputs, ref):
                for k in ("I", "ncross", "status", "refine_level", "R_em"):
                    assert np.array_equal(o[k].cpu().numpy(), r[k]), k
        with pytest.raises(B.BHRTError):
            plan.set_launch(0, 0, 128, 0)
    plan.close()


def test_sweep96_mixed_every_pixel_vs_fp64(B):
    """The 96-image sweep as bench.py times it (256^2, three levels, mixed,
    one batched plan) against single-image FP64 traces (rtol 1e-10, pinned to
    the oracle by test_gpu_trace.py) of eight images, one per spin: every
    pixel within 1e-4 of each image's maximum."""
    from paper_2605_05635_gb300 import workloads
    base = workloads.sweep_96()
    flats = [dict(d, **workloads.MIXED_INTEG) for d in base]
    plan = B.Plan([B.from_flat(d) for d in flats])
    plan.launch()
    plan.check()
    for k in range(0, 96, 12):
        ref = B.trace_batch([B.from_flat(dict(base[k], **workloads.FP64_INTEG))])[0]
        a = plan.outputs[k]["I"].double()
        b = ref["I"].double()
        err = float(((a - b).abs() / b.abs().max()).max())
        assert err <= 1e-4, (k, err)
    plan.close()
