"""The autotuner on the GPU: it returns an admissible launch shape whose
results equal the default shape's bit for bit, and rejects none."""
import numpy as np
import pytest

from paper_2106_13465_gb300 import hydro as H
from paper_2106_13465_gb300 import problems as pr
from paper_2106_13465_gb300.autotune import autotune

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [64, 32])
def test_autotune_small_batch(precision):
    pbs = [pr.random_modes(96, 64, seed=1), pr.sedov(40, 70)]
    res = autotune(pbs, precision=precision, steps=2, warmup=1,
                   y_tiles=(0, 16, 64), x_spans=(0, 60, 240), ctas=(0, 1))
    assert res.rejected == []
    assert res.sweep_ms > 0 and len(res.trials) == 1 + 2 + 2 + 1
    grids = [(p.nx, p.ny, p.h, p.bc) for p in pbs]
    outs = []
    for tuning in ({}, res.tuning()):
        with H.Context(grids, precision=precision) as c:
            if tuning:
                c.set_tuning(**tuning)
            for g, p in enumerate(pbs):
                c.set_state(g, p.U)
            c.step(6)
            outs.append([c.get_state(g) for g in range(len(pbs))])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
