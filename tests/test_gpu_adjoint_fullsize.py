"""The bubble-collapse wall-impulse gradient at 256 x 256 cells over 500
CFL steps, a size and horizon where the collapse's pressure waves reach the
x = 1 wall (at 1024^2 they need about 1400 steps).  MFC_FP64, binomial
checkpointing with 20 snapshots; the gradient along two seeded directions
of the initial volume fraction against the oracle's forward-mode
derivatives of the same 500 steps, stored in
tests/golden/wall_impulse_jvp_256.txt by make_wall_impulse_jvp.py (oracle
only).  Central differences cannot check this map at this size: they move
by 1 % between h = 1e-6 and 1e-7 (the map is only piecewise smooth)."""
import os

import numpy as np
import pytest
import torch

from paper_2503_07953_gb300 import adjoint as adj
from paper_2503_07953_gb300 import workloads as wl
from tests.helpers import solver_for

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "wall_impulse_jvp_256.txt")


def load_golden():
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


def test_wall_impulse_gradient_256_against_oracle_forward_mode(mfc_lib, cuda_device):
    gold = load_golden()
    case, W = wl.bubble_collapse_2d(256)
    S = solver_for(mfc_lib, case)
    a1 = torch.as_tensor(W[case.nf + case.ndim + 1].copy(), dtype=torch.float64, device=cuda_device)
    q0 = adj.alpha_to_state(S, case, W, a1).detach()
    _, _, dts, _ = adj.rollout_gradient(S, q0, 500, lambda n, q: q.sum() * 0.0, 1)
    loss = adj.wall_pressure_objective(S, case, dts)
    J, gq, _, st = adj.rollout_gradient(S, q0, 500, loss, 20, dts)
    assert st.max_live_snapshots <= 20
    assert J == pytest.approx(gold["J"], rel=1e-12)
    a = a1.clone().requires_grad_(True)
    (adj.alpha_to_state(S, case, W, a) * gq).sum().backward()
    band = ((a1 > 1e-3) & (a1 < 1 - 1e-3)).double()
    gen = torch.Generator(device="cpu").manual_seed(0)
    for k in range(2):
        d = torch.randn(a1.shape, generator=gen, dtype=torch.float64).to(cuda_device) * band
        d = d / float(d.abs().max())
        ad = float((a.grad * d).sum())
        assert ad == pytest.approx(gold[f"dJ_direction_{k}"], rel=1e-9), (k, ad)
