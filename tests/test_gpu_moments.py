"""The target's angular descriptors and their adjoint through Cartesian moments (lsd_set_angular_moments): the
sixteen triplet sums of every row as (1/2)(ordered pairs - diagonal) of polynomials in u_p.u_q, evaluated from the
165 moments sum_p w_p u_p^alpha.  Against the FP64 oracle, which forms the pair sums themselves, the moment path
meets the same FP32 bars as the pair-sum path (descriptors, dE/dX and forces within 1e-5 relative, per norm and
per element; lists and decisions identical), at 27, 256 and 4,096 atoms; and it agrees with the pair-sum path of
the same library to FP32 rounding."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W
from parity_bounds import FORCE_TOL, elem, rel

pytestmark = pytest.mark.gpu

AGREE = 2e-6   # moment form against the pair sums of the same library: FP32 rounding of either form


def _handle(w, target, moments):
    from paper_2606_02455_b300 import lsd
    h = lsd.LSD(w.system, w.draft, target, w.integ)
    h.set_angular_moments(moments)
    return h


def _configs(system, n, scale, seed):
    rng = np.random.default_rng(seed)
    return np.stack([system.positions + scale * rng.standard_normal(system.positions.shape) for _ in range(n)])


def _small():
    from test_gpu_parity import _small_ragged
    return _small_ragged()


@pytest.mark.parametrize("name", ["ragged27", "c2"])
def test_moment_descriptors_and_forces_match_oracle(name):
    """K configurations in one batched call with the moment form forced on (these sparse systems default to the
    pair sums): X, dE/dX and forces within the FP32 bars of the oracle's pair sums."""
    import torch
    w = _small() if name == "ragged27" else W.config2()
    s = w.system
    K = w.integ.K
    qs = _configs(s, K, 0.08, seed=321)
    out = {}
    for mom in (True, False):
        h = _handle(w, w.target, mom)
        F = h.target_forces(torch.tensor(qs, device="cuda")).cpu().numpy()
        X, G = h.descriptors(K)
        out[mom] = (F, X, G)
        h.close()
    F, X, G = out[True]
    for c in range(K):
        ref = O.energy_forces(s, w.target, qs[c], want=("F", "X", "dEdX"))
        assert rel(X[c], ref["X"]) < FORCE_TOL and elem(X[c], ref["X"]) < FORCE_TOL, c
        assert rel(G[c], ref["dEdX"]) < FORCE_TOL and elem(G[c], ref["dEdX"]) < FORCE_TOL, c
        assert rel(F[c], ref["F"]) < FORCE_TOL and elem(F[c], ref["F"]) < FORCE_TOL, (c, rel(F[c], ref["F"]))
        for a, b in zip(out[True], out[False]):
            assert rel(a[c], b[c]) < AGREE, c


def test_moment_window_matches_oracle_c2():
    """One 256-atom window with rejections (head scale 1.5) with the moment form: the window arrays, log ratios
    and decisions against the oracle's window, as for the pair-sum form."""
    from test_gpu_parity import _window_compare
    w = W.config2()
    target = W.replace(w.target, head_scale=1.5)
    h = _handle(w, target, True)
    h.draft_window()
    nc, first = h.verify_window()
    win = h.get_window()
    h.close()
    ref = O.lsd_window(w.system, w.draft, target, w.integ, w.system.seed, 0, w.integ.K, w.system.positions,
                       w.system.momenta)
    _window_compare(win, ref, w.integ.K, w, target)
    assert nc == ref["n_committed"]


def test_moment_forces_dense_sampled_and_against_pair_sums():
    """4,096 atoms at 0.1 atoms/A^3 (86-90 descriptor neighbours: the moment form is the default) with the target
    network in FP32 arithmetic: sampled atoms' forces within the FP32 bars of the oracle, and every atom's force
    within FP32 rounding of the pair-sum form."""
    import torch
    w = W.config4()
    s = w.system
    target = W.replace(w.target, precision="fp32-cuda-cores")
    q = s.positions.copy()
    F = {}
    for mom in (True, False):
        h = _handle(w, target, mom)
        F[mom] = h.target_forces(torch.tensor(q[None], device="cuda")).cpu().numpy()[0]
        h.close()
    sel = np.sort(np.random.default_rng(4).choice(s.n_atoms, 32, replace=False))
    ref = O.forces_subset(s, target, q, sel)
    assert rel(F[True][sel], ref) < FORCE_TOL and elem(F[True][sel], ref) < FORCE_TOL, rel(F[True][sel], ref)
    assert rel(F[True], F[False]) < AGREE, rel(F[True], F[False])


def test_moments_default_by_density_and_unsupported_without_angular_terms():
    from paper_2606_02455_b300 import lsd
    w = W.config1()   # radial-only target
    h = lsd.LSD(w.system, w.draft, w.target, w.integ)
    with pytest.raises(lsd.LSDError):
        h.set_angular_moments(True)
    h.set_angular_moments(False)
    h.close()
