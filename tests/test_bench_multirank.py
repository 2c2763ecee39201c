"""The benchmark's multi-process path on the CPU: two gloo ranks shard the batched runs by
seed with no overlap and no gap, and the whole-job figures are the max of the ranks' times
and the sum of their counts.  (The GPU path runs the same functions over NCCL.)"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, n_units, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        mine = bench.shard(n_units, rank, ws)
        # a rank's wall time and counts: made up, different per rank
        mx, sm = bench.job_reduce([10.0 + rank], [len(mine), rank], "cpu")
        got = [None] * ws
        dist.all_gather_object(got, mine)
        out[rank] = (got, mx, sm)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,n_units", [(2, 256), (2, 7)])
def test_two_ranks_shard_and_reduce(ws, n_units):
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.start_processes(_rank, args=(ws, port, n_units, out), nprocs=ws, start_method="spawn", join=True)
        res = dict(out)
    for rank in range(ws):
        shards, mx, sm = res[rank]
        flat = sorted(u for s in shards for u in s)
        assert flat == list(range(n_units))                 # every unit once
        assert mx == [10.0 + ws - 1]                        # max of the ranks' times
        assert sm == [float(n_units), float(sum(range(ws)))]


def test_single_process_is_a_no_op():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.job_reduce([3.0], [4, 5]) == ([3.0], [4.0, 5.0])


def test_batch_failures_counts_causes():
    """The batched leg's outcome counts: one count per status bit (1 non-positive volume or
    density, 2 NaN, 4 step below dt_min), failed runs split by projectile, and clean runs
    whose crater half-width reaches the absorbing strip (nr - pml_r cells from the axis),
    and failed runs split by whether their cavity had reached a strip."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from paper_2403_04267_gb300 import workloads as W

    def spec(projectile):
        sp = W.batched_run(W.batched_draw(7), 100)
        sp["materials"][-1] = W.iron() if projectile == "iron" else W.basalt()
        return sp

    specs = [spec(p) for p in ("iron", "basalt", "basalt", "iron", "basalt", "basalt")]
    strip = (specs[0]["grid"]["nr"] - specs[0]["grid"]["pml_r"]) * specs[0]["grid"]["dx"]
    status = [0, 1, 5, 2, 0, 0]
    polled = np.array([[20.0, 1e-3, 100, s, 20.0] for s in status])
    half = [strip, None, None, None, strip - 1.0, strip + 5.0]
    assert bench.batch_failures(polled, specs, half) == [2, 1, 1, 1, 2, 2, 0, 3]
    # failed runs 1 and 3 stopped with their cavity in a strip, run 2 did not
    cav = [None, True, False, True, None, None]
    assert bench.batch_failures(polled, specs, half, cav) == [2, 1, 1, 1, 2, 2, 2, 1]
    assert bench.batch_failures(np.zeros((0, 5)), [], []) == [0, 0, 0, 0, 0, 0, 0, 0]


def test_cavity_in_strip_reads_the_strip_cells_below_the_surface():
    """A strip cell below the initial surface with less than half matter marks the run;
    emptied cells above the surface, or inside the domain, do not."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from paper_2403_04267_gb300 import workloads as W
    sp = W.batched_run(W.batched_draw(7), 120)
    g = sp["grid"]
    nr, nz, pb, pr = g["nr"], g["nz"], g["pml_b"], g["pml_r"]
    ks = int(round(sp["z_surface"] / g["dx"]))
    phi = np.zeros((nz, nr))
    phi[:ks, :] = 1.0
    assert not bench.cavity_in_strip(phi, sp)
    cav = phi.copy()
    cav[pb + 5:ks, :10] = 0.0                     # a deep cavity inside the domain
    assert not bench.cavity_in_strip(cav, sp)
    cav[pb - 1, 3] = 0.3                          # it reaches the bottom strip
    assert bench.cavity_in_strip(cav, sp)
    side = phi.copy()
    side[ks - 3, nr - pr] = 0.0                   # the crater rim reaches the right strip
    assert bench.cavity_in_strip(side, sp)
    # matter torn open to a near-vacuum density at full fraction: in the strip it marks the
    # run, inside the domain it does not
    ratio = np.ones((nz, nr))
    ratio[pb + 5, 0] = 0.005
    assert not bench.cavity_in_strip(phi, sp, ratio)
    ratio[pb - 3, 1] = 0.005
    assert bench.cavity_in_strip(phi, sp, ratio)
    ratio[pb - 3, 1] = 0.02
    assert not bench.cavity_in_strip(phi, sp, ratio)
