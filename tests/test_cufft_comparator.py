"""The cuFFT comparator of bench.py (plain PyTorch step, timed beside the
library) computes the same scheme: run on CPU tensors against the FP64
oracle on small grids."""

import numpy as np
import pytest

from helpers import oracle_from_config, rel_l2
from paper_1408_4675_gb300 import inputs

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("cfgid,n,steps", [(1, 16, 30), (2, 16, 30), (3, 32, 40)])
def test_comparator_matches_oracle(cfgid, n, steps):
    import bench
    cfg = inputs.make_config(cfgid, n=n, n_steps=steps)
    st = bench.CufftStep(cfg, device="cpu")
    st.step(steps)
    osim, oids = oracle_from_config(cfg)
    osim.step(steps)
    of = osim.fields()
    assert rel_l2(st.p.numpy(), of["p"]) <= 1e-4
    for i, name in enumerate(("ux", "uy", "uz")):
        assert rel_l2(st.u[i].numpy(), of[name]) <= 1e-4
    for (ii, pm, p2), oi, (idx, rec) in zip(st.sens, oids, cfg["sensors"]):
        if rec & 1:
            assert rel_l2(pm.numpy(), osim.read(oi, 1)) <= 1e-4
