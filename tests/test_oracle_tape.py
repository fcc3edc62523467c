"""Pins of the PyTorch tape restatement (oracle/tape.py) against the C oracle:
two independent restatements of the plain step (Sec. 2 with the box faces)
agree to round-off, so the tape's autograd gradient is a reference for the
adjoint."""
import numpy as np
import pytest
import torch

import synth
from oracle import tape


@pytest.mark.parametrize("faces,lbgk", [((0,) * 6, False), ((1, 1, 0, 0, 2, 3), False), ((0,) * 6, True)])
def test_tape_step_equals_oracle(orc, faces, lbgk):
    shape = (7, 6, 5)
    nu = 0.02
    beta = orc.beta_from_nu(nu)
    rho, u, xi = synth.parity_fields(shape, 21)
    o = orc.Oracle(shape, nu=nu, faces=faces, u_face=(0.03, -0.01, 0.02),
                   gamma_mode=orc.MODE_LBGK if lbgk else orc.MODE_ANALYTIC)
    o.init_state(rho, u, xi, 1e-3)
    f0 = o.get_f()
    box = tape.Box(shape, faces, u_face=(0.03, -0.01, 0.02))
    f = torch.tensor(f0, dtype=torch.float64)
    for _ in range(3):
        f = box.step(f, beta, lbgk)
    o.step(3)
    ref = o.get_f()
    assert np.abs(f.numpy() - ref).max() / np.abs(ref).max() < 1e-13


def test_tape_collision_conserves_and_is_differentiable():
    rho, u, xi = synth.parity_fields((3, 2, 2), 4)
    f = tape.equilibrium(torch.tensor(rho), torch.tensor(np.moveaxis(u, -1, 0)))
    f = (f + 1e-3 * tape.W.reshape(27, 1, 1, 1) * torch.tensor(xi)).requires_grad_(True)
    out = tape.collide(f, 0.9)
    assert torch.allclose(out.sum(0), f.sum(0), atol=1e-15, rtol=0)
    for a in range(3):
        ca = tape.C[:, a].reshape(27, 1, 1, 1)
        assert torch.allclose((ca * out).sum(0), (ca * f).sum(0), atol=1e-15, rtol=0)
    out.pow(2).sum().backward()
    assert torch.isfinite(f.grad).all()
