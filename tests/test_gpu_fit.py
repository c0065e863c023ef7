"""Uneven-batch inverse rendering: the Adam loop driven by the CUDA path on the whole 256-mesh batch tracks the
same loop driven by the FP64 oracle's gradients on four items of that batch (the fewest triangles, the most,
and two in between): final vertex RMSE over those items."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2405_02508_gb300 import scenes
from paper_2405_02508_gb300.fit import UnevenFit

pytestmark = pytest.mark.gpu


def test_uneven_batch_fit_tracks_oracle_driven_subset():
    from oracle.fitloop import oracle_fit, subset_of_batch

    items = scenes.uneven_batch(n_items=256)
    fit = UnevenFit(items, sigma=0.01, seed=11)
    steps = 60
    v_gpu = fit.run(steps, lr=1e-3)
    sub = subset_of_batch(256)
    rows = np.concatenate([np.arange(fit.vert_off[k], fit.vert_off[k + 1]) for k in sub])
    r0, r_gpu = fit.rmse(fit.v_init, sub), fit.rmse(v_gpu, sub)
    v_orc = oracle_fit([items[k] for k in sub], fit.v_init[torch.from_numpy(rows).cuda()].cpu().numpy(), steps,
                       lr=1e-3)
    d = v_orc - fit.v_true[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    r_orc = float(np.sqrt((d ** 2).sum(axis=1).mean()))
    print(f"subset {sub}: rmse {r0:.6f} -> gpu {r_gpu:.6f} / oracle-driven {r_orc:.6f} after {steps} steps; "
          f"whole batch {fit.rmse(fit.v_init):.6f} -> {fit.rmse(v_gpu):.6f}")
    # the two loops follow the same trajectory
    assert abs(r_gpu - r_orc) <= 0.02 * r_orc, (r0, r_gpu, r_orc)
    assert abs(r_gpu - r0) > 1e-5  # the loop moved the vertices
