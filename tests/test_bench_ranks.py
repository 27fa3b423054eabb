"""The bench's multi-rank aggregation on two gloo ranks (CPU): each rank
traces its own batch (weak scaling, no collective on the data path); the job
value is the sum of the ranks' rays over the longest rank's time."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rays, ms = 1000.0 * (rank + 1), 50.0 + 25.0 * rank
    out = bench.aggregate_ranks(rays, ms, world, torch.device("cpu"))
    q.put((rank, out))
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert res[r] == (3000.0, 75.0)


def test_aggregate_single_rank():
    torch = pytest.importorskip("torch")
    import bench
    assert bench.aggregate_ranks(123.0, 4.5, 1, torch.device("cpu")) == (123.0, 4.5)


def test_added_workload_generators():
    """The seeded inputs of the shadow, scan and amplitude-curve benches have
    the shapes and parameters their metric strings state."""
    import math

    import numpy as np

    from paper_2605_05635_gb300 import workloads
    flats, psi, lo, hi, tol = workloads.shadow_fig5()
    assert [d["metric"] for d in flats] == [0, 1, 2] and len(psi) == 4096
    assert flats[1]["lam_E"] == 0.3 and flats[2]["eta"] == 0.02 and flats[2]["lam_c"] == 10.0
    assert all(d["chi"] == 0.5 and abs(d["incl"] - math.radians(60.0)) < 1e-15 for d in flats)
    assert (lo, hi, tol) == (1.0, 9.0, 1e-10) and psi[0] == 0.0 and psi[-1] < 2 * math.pi
    metric, chi, lam_E, eta, lam_c, theta = workloads.geometry_grid(8, 4)
    assert metric.shape == (128,) and np.all(metric[:64] == 1) and np.all(metric[64:] == 2)
    assert chi.min() == 0.0 and chi.max() == 1.2 and lam_E[:64].min() == 0.05
    assert eta[64:].max() == 0.3 and np.all(lam_c == 10.0) and theta[-1] == 0.5 * math.pi
    imgs = workloads.fig12_images()
    assert [d["metric"] for d in imgs] == [0, 1, 2]
    assert all(d["nx"] == 1024 and d["chi"] == 0.95 and d["levels"] == 3 for d in imgs)
    vol = workloads.sweep_512(precision=1, volumetric=True)
    assert all(d["volumetric"] == 1 for d in vol) and len(vol) == 6


def test_clock_summary_and_step_defaults():
    """The clock record is the median SM clock of the samples with the
    throttle reasons they show; a sample with an unreadable clock is skipped
    and no sample gives None. Millisecond-long workloads default to enough
    timed calls for the sampler to see the timed region."""
    import bench
    lines = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage"]
    c = bench.summarise_clocks(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    hot = bench.summarise_clocks(["0, 1500, 2070, 1400, 0x8, Not Active, Active, Not Active, "
                                  "Not Active"])
    assert hot["reasons"] == ["hw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0
    assert bench.summarise_clocks([]) is None
    assert bench.default_steps("sweep512") == 5
    assert bench.default_steps("vis1024") * 0.7e-3 >= 0.5      # about 0.75 ms per call
    assert bench.default_steps("viscurves") * 2.9e-3 >= 0.5
    assert bench.default_steps("kerr64") * 30e-3 >= 0.5
