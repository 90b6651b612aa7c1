"""The sharded sweep on one GPU: a one-rank shard (a real gloo process group of size 1) runs
the library's batched handle on every instance and gives bit for bit the results of the
unsharded handle, and its combined statistics equal the handle's own."""
import os
import socket

import numpy as np
import pytest

from paper_1812_00394_gb300 import fvlbm, meshgen as mg
from paper_1812_00394_gb300.shard import ShardedSweep

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_one_rank_shard_equals_the_unsharded_handle():
    import torch.distributed as dist
    cases = mg.batched_sweep(seed=5, scale=0.05)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    dist.init_process_group("gloo", rank=0, world_size=1)
    sw = None
    try:
        sw = ShardedSweep(cases, lambda cs: fvlbm.Solver(cs, precision=fvlbm.FVLBM_FP32_DEV, device=0),
                          dist=dist, device="cpu")
        assert sw.mine == list(range(len(cases)))
        sw.step(4)
        st = sw.step(1, stats=True)
        forces = sw.gather_forces()
        fields = sw.gather_fields()
    finally:
        if sw is not None:
            sw.close()
        dist.destroy_process_group()
    ref = fvlbm.Solver(cases, precision=fvlbm.FVLBM_FP32_DEV, device=0)
    ref.step(4)
    st_ref = ref.step(1, stats=True)
    assert st == st_ref
    for g in range(len(cases)):
        fr = ref.forces(g)
        assert np.array_equal(forces[g], [fr["fx"], fr["fy"], fr["cd"], fr["cl"]])
        fl = ref.fields(g)
        for key in ("rho", "u", "v"):
            assert np.array_equal(fields[g][key], fl[key]), (g, key)
    ref.close()
