"""Long-run statistics of LSD on the GPU: the committed trajectory is target distributed (Thm 3.1, Thm D.2), so over
20,000 committed steps

* the rejections match Eq. 6: every committed step was tested, in order, and step j is rejected with probability
  p_j = erf(|delta_j| / sqrt 8) given its past, so (rejections - sum p_j) / sqrt(sum p_j (1 - p_j)) is a martingale
  z-score; it must lie within 4;
* the mean kinetic temperature <T_kin> = <sum p^2 / m> / (3 N k_B) and the mean target energy <E_pot> of LSD agree
  with those of plain target Langevin on the same GPU (an independent run of the same length, another noise key)
  within 3 standard errors of the difference, each side's error from 20 block averages.

The trajectories are seeded and the kernels deterministic, so each outcome is fixed (no flakiness)."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W

pytestmark = pytest.mark.gpu

N_STEPS = 20000
EVERY = 50
BLOCKS = 20


def _observables(h, w, n_steps, lsd_run):
    """(T_kin, E_pot) every EVERY steps: lsd_step or plain steps of EVERY, then the state and the target energy."""
    import torch
    s = w.system
    kb = O.kboltz()
    kap = O.kappa()
    minv = 1.0 / s.masses[s.species]
    T, E = [], []
    for _ in range(n_steps // EVERY):
        if lsd_run:
            h.step(EVERY)
        else:
            h.plain_step(EVERY)
        q, p, _ = h.get_state()
        # kinetic energy in eV: sum p^2 / (2 m) is in amu A^2/fs^2, divided by kappa
        ekin = 0.5 * np.sum(p * p * minv[:, None]) / kap
        T.append(2.0 * ekin / (3 * s.n_atoms * kb))
        _, Ea = h.target_forces(torch.tensor(q[None], device="cuda"), energies=True)
        E.append(float(Ea.double().sum()))
    return np.array(T), np.array(E)


def _block_mean_err(x):
    b = x[: len(x) // BLOCKS * BLOCKS].reshape(BLOCKS, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / np.sqrt(BLOCKS)


@pytest.mark.parametrize("cfg", [1, 2])
def test_long_run_statistics_match_plain_target_langevin(cfg):
    from paper_2606_02455_b300 import lsd
    w = W.CONFIGS[cfg]()
    s = w.system
    h = lsd.LSD(s, w.draft, w.target, w.integ)
    h.plain_step(2000)                       # equilibrate
    q0, p0, n0 = h.get_state()
    h.close()

    h = lsd.LSD(s, w.draft, w.target, w.integ)
    h.set_state(q0, p0, n0)
    h.set_pipelining(True)
    st0 = h.stats()
    T_l, E_l = _observables(h, w, N_STEPS, True)
    st1 = h.stats()
    h.close()
    committed = st1["committed"] - st0["committed"]
    rejected = st1["rejected"] - st0["rejected"]
    pred = st1["pred_rejected"] - st0["pred_rejected"]
    assert committed == N_STEPS
    # the martingale's variance is sum p (1 - p) = pred - sum p^2 <= pred (1 - pred / committed) (Cauchy-Schwarz):
    # the z-score below is conservative
    var = pred * (1.0 - pred / committed)
    z = (rejected - pred) / np.sqrt(max(var, 1e-12))
    assert rejected > 0, "no rejection in %d steps: the rejection law is not exercised" % N_STEPS
    assert abs(z) < 4.0, (rejected, pred, z)

    s2 = W.replace(s, seed=s.seed + 1000)   # an independent plain run
    h = lsd.LSD(s2, w.draft, w.target, w.integ)
    h.set_state(q0, p0, n0)
    T_p, E_p = _observables(h, w, N_STEPS, False)
    h.close()
    for a, b, name in ((T_l, T_p, "T_kin"), (E_l, E_p, "E_pot")):
        ma, ea = _block_mean_err(a)
        mb, eb = _block_mean_err(b)
        assert abs(ma - mb) < 3.0 * np.hypot(ea, eb), (name, ma, ea, mb, eb)
    # and the kinetic temperature is the thermostat's (equipartition; ABOBA's kinetic bias is O(dt^2 gamma^2))
    mT, eT = _block_mean_err(np.concatenate([T_l, T_p]))
    assert abs(mT - w.integ.temperature) < 4.0 * eT + 0.01 * w.integ.temperature, (mT, eT)
