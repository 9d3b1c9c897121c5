"""The distributed slab driver on a GPU with a one-rank NCCL group: the slab handle runs on
the current stream, the (empty) halo plan posts no transfers, and the records go through an
NCCL all-reduce on device tensors.  With one slab the run is the whole system's, so the spins
equal the undecomposed handle's bit for bit.  (More ranks need more GPUs; the halo sequence of
two ranks is covered on CPU with gloo.)"""
import os
import socket

import numpy as np
import pytest

from paper_1310_6143_gb300 import lattice as L

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_distributed_slab_one_rank_nccl(precision):
    import torch
    import torch.distributed as dist

    from paper_1310_6143_gb300.slab import DistributedSlab
    from paper_1310_6143_gb300.system import SpinSystem

    lat = L.film(48, 40, 8)
    kw = dict(alpha=0.1, dt=1e-16, T=500.0, seed=3, precision=precision)
    with SpinSystem(lat, **kw) as whole:
        whole.step(12)
        S_ref, rec_ref = whole.spins(), whole.record(0, 12)
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1)
    try:
        with SpinSystem(lat, slab=(1, 0), **kw) as h:
            d = DistributedSlab(h, lat.row_ptr, lat.col)
            assert d.plan == [] and d.send == {} and d.recv == {}
            d.refresh_halo()
            d.step(12)
            rec = d.record(0, 12)
            torch.cuda.synchronize()
            S = h.spins()[:lat.n]
    finally:
        dist.destroy_process_group()
    np.testing.assert_array_equal(S, S_ref)
    scale = np.maximum(np.abs(rec_ref).max(axis=(0, 1)), 1e-300)
    np.testing.assert_allclose(rec / scale, rec_ref / scale, rtol=0, atol=1e-12)
