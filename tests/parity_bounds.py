"""Tolerances of the GPU parity tests, each derived from the arithmetic it bounds (imported by the test files).

FORCE_TOL   FP32 forces, descriptors, dE/dX: within 1e-5 of the FP64 oracle, as a norm ratio per configuration and
            per element relative to the configuration's largest |value|.
BF16_TOL    the same for BF16 MLP arithmetic: 2e-2.
XI_ERR      the GPU's FP32 Box-Muller normal differs from the exact (FP64) one by at most 1e-6 per component for
            |xi| < 6 (a few ulp of logf, sqrtf and sincospif times the radius).
LOGR_RTOL   end-to-end log ratio of a drafted step (the GPU drafts and evaluates both potentials in FP32, the oracle
            in FP64): within 1e-4 max(1, |log r|).  Decisions are compared outside that same band, so a log ratio
            within its tolerance cannot flip a compared decision; none may fall inside it at the test seeds.
"""
import numpy as np

import oracle.oracle as O

FORCE_TOL = 1e-5
BF16_TOL = 2e-2
XI_ERR = 1e-6
LOGR_RTOL = 1e-4
REFLECT_ERR = 1e-4   # error of a reflected momentum, in sigma: 2 |z.delta^| |d delta^| with |d delta^| <~ 2e-5 here


def rel(a, b):
    """Norm ratio |a - b| / |b|."""
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def elem(a, b):
    """Largest element difference relative to the largest |b|."""
    b = np.asarray(b, np.float64)
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-300))


def logr_tol(logr):
    return LOGR_RTOL * np.maximum(1.0, np.abs(logr))


def state_tols(w, target, n_steps, n_refl=0, draft=None):
    """Bounds on |p_gpu - p_oracle| and |q_gpu - q_oracle| after n_steps steps from the same state.

    Per step the momentum differs by the FP32 noise (XI_ERR sigma) and by the FP32 force error, at most FORCE_TOL of
    max|F| per element, of the force that enters the mean (the draft's for an accepted step, the target's for a
    reflected or plain step), times (1+c1)(dt/2)kappa: e_step = sigma XI_ERR + aF 1e-5 (max|F~| + max|F|), with
    max|F| taken at the start and doubled for the rest of the run.  c1 < 1, so per-step errors add: n e_step.  A
    reflection adds REFLECT_ERR sigma.  Positions follow q_n = q_{n-1} + (dt/2)(p_{n-1} + p_n)/m, so their error
    is at most (dt/2)/m times twice the sum of the momentum errors: hm n (n+1) e_step (plus the reflections').
    The force change these position errors cause over a few tens of steps is below 1e-3 of the force error term
    (stiffness ~0.1 eV/A^2, dt kappa ~ 0.02), inside the doubling."""
    draft = w.draft if draft is None else draft
    c1, aF, hm, sg = O.coefficients(w.system, w.integ)
    fmax = np.abs(O.forces(w.system, target, w.system.positions)).max() + \
        np.abs(O.forces(w.system, draft, w.system.positions)).max()
    e_step = sg.max() * XI_ERR + aF * FORCE_TOL * 2.0 * fmax
    e_refl = REFLECT_ERR * sg.max()
    ptol = n_steps * e_step + n_refl * e_refl
    qtol = hm.max() * (n_steps * (n_steps + 1) * e_step + 2 * n_steps * n_refl * e_refl)
    return ptol, qtol + 1e-13 * np.abs(w.system.positions).max()
