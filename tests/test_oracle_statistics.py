"""Statistical pins of the oracle (T9, T10).

T9: a draft with a non-conservative shear field F_x += A sin(2 pi y / L_y) overheats under plain draft Langevin
dynamics; LSD with that draft and the conservative target keeps the target's kinetic temperature, as plain target
dynamics does (the synthetic analogue of the heating experiment, Tab. 1).

T10: 10-step trajectories from one equilibrated state, with independent noise keys per trajectory: the maximum mean
discrepancy (RBF kernel, median bandwidth, unbiased estimate) between LSD and target trajectories is as small as
between two target samples, and far below the draft's (App. F)."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W


def _system():
    w = W.config1(8)
    lj = dict(lj_eps=w.draft.lj_eps, lj_sigma=w.draft.lj_sigma, lj_cutoff=w.draft.lj_cutoff)
    return w, W.Potential(**lj), W.Potential(**lj, shear=0.25)


def _tkin(traj_p, system):
    m = system.masses[system.species][None, :, None]
    ke = 0.5 * (traj_p ** 2 / m).sum(axis=(1, 2)) / O.kappa()          # eV per frame
    return 2.0 * ke / (3 * system.n_atoms * O.kboltz())


@pytest.mark.slow
def test_t9_shear_draft_overheats_but_lsd_keeps_the_target_temperature():
    w, target, draft = _system()
    s = w.system
    integ = W.replace(w.integ, K=8)
    eq = O.plain_run(s, target, integ, 5, 500, s.positions, s.momenta)
    n = 2500
    plain_t = O.plain_run(s, target, integ, 6, n, eq["q"], eq["p"], traj=True)
    plain_d = O.plain_run(s, draft, integ, 6, n, eq["q"], eq["p"], traj=True)
    lsd = O.lsd_run(s, draft, target, integ, 6, n, 8, eq["q"], eq["p"], traj=True)
    T = integ.temperature
    t_target = _tkin(plain_t["traj_p"][500:], s).mean()
    t_draft = _tkin(plain_d["traj_p"][500:], s).mean()
    t_lsd = _tkin(lsd["traj_p"][500:], s).mean()
    assert t_draft > 1.3 * T, t_draft                       # the shear field pumps energy in
    assert abs(t_target / T - 1) < 0.12, t_target
    assert abs(t_lsd / T - 1) < 0.12, t_lsd
    assert abs(t_lsd - t_target) < 0.12 * T
    assert lsd["stats"]["rejected"] > 50                    # the draft is far from the target


def _mmd2(X, Y, bw):
    def k(A, B):
        d = (A * A).sum(1)[:, None] + (B * B).sum(1)[None, :] - 2 * A @ B.T
        return np.exp(-np.maximum(d, 0) / (2 * bw * bw))
    m, n = len(X), len(Y)
    kxx, kyy, kxy = k(X, X), k(Y, Y), k(X, Y)
    return ((kxx.sum() - np.trace(kxx)) / (m * (m - 1)) + (kyy.sum() - np.trace(kyy)) / (n * (n - 1))
            - 2 * kxy.mean())


@pytest.mark.slow
def test_t10_mmd_of_lsd_trajectories_matches_target():
    w, target, draft = _system()
    s = w.system
    integ = W.replace(w.integ, K=4)
    eq = O.plain_run(s, target, integ, 5, 400, s.positions, s.momenta)
    M, steps = 250, 10

    def trajs(kind, seed0):
        out = []
        for j in range(M):
            if kind == "lsd":
                r = O.lsd_run(s, draft, target, integ, seed0 + j, steps, 4, eq["q"], eq["p"], traj=True)
            else:
                r = O.plain_run(s, target if kind == "target" else draft, integ, seed0 + j, steps, eq["q"], eq["p"],
                                traj=True)
            out.append((r["traj_q"] - eq["q"][None]).ravel())
        return np.array(out)

    tgt, tgt2 = trajs("target", 1000), trajs("target", 3000)
    lsd, dft = trajs("lsd", 2000), trajs("draft", 4000)
    pooled = np.concatenate([tgt, dft])
    d = np.sqrt(((pooled[:, None, :] - pooled[None, :, :]) ** 2).sum(-1))
    bw = np.median(d[d > 0])
    m_tt, m_lt, m_dt = _mmd2(tgt2, tgt, bw), _mmd2(lsd, tgt, bw), _mmd2(dft, tgt, bw)
    print("T10 MMD^2: target'-target %.2e, LSD-target %.2e, draft-target %.2e" % (m_tt, m_lt, m_dt))
    assert m_dt > 5 * max(abs(m_tt), abs(m_lt), 1e-12)
    assert abs(m_lt) < 5 * max(abs(m_tt), 2.0 / M)
