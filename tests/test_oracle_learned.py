"""Oracle pins for the learned draft: the force-matching loss and its exact gradient (the double backward through
descriptors and MLP) agree with central finite differences in the weights."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W


def _setup(n_rbf, n_ang, n_layers, width, seed=0):
    s = W.small_system(n_cells=1, a=4.6, n_species=2, seed=seed, L=9.2)
    d0 = W.input_dim(2, n_rbf, n_ang)
    w = W.mlp_weights(d0, n_layers, width, 4) * 2.0
    w[width * d0:width * d0 + width] = np.linspace(-0.5, 0.5, width)   # non-zero first-layer biases
    pot = W.Potential(lj_eps=np.array([0.01, 0.005]), lj_sigma=np.array([2.6, 2.9]), lj_cutoff=4.4, n_rbf=n_rbf,
                      n_ang=n_ang, n_layers=n_layers, width=width, desc_cutoff=4.0, head="linear", head_scale=1.0,
                      weights=w)
    rng = np.random.default_rng(seed + 1)
    frames_q = np.stack([s.positions + 0.1 * rng.standard_normal(s.positions.shape) for _ in range(2)])
    frames_F = 0.3 * rng.standard_normal(frames_q.shape)
    return s, pot, frames_q, frames_F


@pytest.mark.parametrize("n_rbf,n_ang,n_layers,width", [(8, 0, 1, 6), (6, 16, 2, 5)])
def test_force_matching_gradient_matches_finite_differences(n_rbf, n_ang, n_layers, width):
    """T13: dL/dtheta of L = mean |F~(theta) - F*|^2 equals the central difference on every weight."""
    s, pot, fq, fF = _setup(n_rbf, n_ang, n_layers, width)
    loss, g = O.force_match(s, pot, fq, fF)
    h = 1e-5
    w0 = pot.weights.copy()
    fd = np.zeros_like(w0)
    for k in range(w0.size):
        wp = w0.copy(); wp[k] += h
        wm = w0.copy(); wm[k] -= h
        lp, _ = O.force_match(s, W.replace(pot, weights=wp), fq, fF, grad=False)
        lm, _ = O.force_match(s, W.replace(pot, weights=wm), fq, fF, grad=False)
        fd[k] = (lp - lm) / (2 * h)
    assert g[-1] == 0.0 and abs(fd[-1]) < 1e-9        # the output bias does not change forces
    err = np.linalg.norm(g - fd) / np.linalg.norm(fd)
    assert err < 1e-6, err


def test_force_matching_loss_definition():
    """The loss is the mean squared force residual over frames and components."""
    s, pot, fq, fF = _setup(8, 0, 1, 6)
    loss, _ = O.force_match(s, pot, fq, fF, grad=False)
    F = np.stack([O.forces(s, pot, q) for q in fq])
    assert loss == pytest.approx(np.mean((F - fF) ** 2), rel=1e-12)
