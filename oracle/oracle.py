"""Test-infrastructure oracle: Python front end of ``lsd_oracle.c``.

Plain FP64 CPU reference of Langevin Speculative Dynamics (the ABOBA
integrator of Eq. 2, the BOB Gaussian of Eq. 4, ``reflectionVerify`` of Eq. 5
with the shared post-processing map of Thm 3.1, the synchronous speculative
window of Alg. 1 with the draft/verify steps of Alg. 2, and error correction of
Alg. 3) and of the synthetic potentials it runs on.  Only ``tests/``, the
package's ``smoke()`` and ``bench.py``'s CPU baseline may use it; the CUDA
library never does.

Inputs are plain objects with the attributes of ``System``, ``Potential`` and
``Integrator`` in ``paper_2606_02455_b300.workloads`` (duck-typed: this module
imports nothing from the package).

Pins: every function here is pinned by ``tests/test_oracle_*.py`` against the
paper's closed forms, published known-answer vectors, finite differences or
brute force.  None is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblsd_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Sys(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("n_species", ctypes.c_int32), ("box", ctypes.c_double * 3),
                ("species", ctypes.c_void_p), ("species_mass", ctypes.c_void_p)]


class _Pot(ctypes.Structure):
    _fields_ = [("lj_eps", ctypes.c_void_p), ("lj_sigma", ctypes.c_void_p), ("lj_cutoff", ctypes.c_double),
                ("n_rbf", ctypes.c_int32), ("n_ang", ctypes.c_int32), ("n_layers", ctypes.c_int32),
                ("width", ctypes.c_int32), ("desc_cutoff", ctypes.c_double), ("head", ctypes.c_int32),
                ("head_scale", ctypes.c_double), ("weights", ctypes.c_void_p), ("k_harm", ctypes.c_double),
                ("q_ref", ctypes.c_void_p), ("shear", ctypes.c_double)]


class _Prm(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("gamma", ctypes.c_double), ("temperature", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("integrator", ctypes.c_int32)]


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, I32, I64, D, U64, U32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                         ctypes.c_uint64, ctypes.c_uint32)
            sigs = {
                "o_const_kappa": (D, []), "o_const_kb": (D, []),
                "o_input_dim": (I32, [I32, I32, I32]),
                "o_n_weights": (I64, [I32, I32, I32]),
                "o_philox4x32_10": (None, [P, P, P]),
                "o_normals": (None, [U64, U64, U32, U32, P]),
                "o_uniform": (D, [U64, U64]),
                "o_neighbors": (ctypes.c_int, [P, P, D, I32, P, P]),
                "o_fixpoint_export": (None, [P, P, P, P]),
                "o_energy_forces": (D, [P, P, P, P, P, P, P]),
                "o_coefficients": (None, [P, P, P, P, P, P]),
                "o_mb_momenta": (None, [P, P, P]),
                "o_transport": (ctypes.c_int, [I32, P, D, P, P, P, P, P]),
                "o_transport_terms": (ctypes.c_int, [I32, P, D, P, P, P, P, P, P, P]),
                "o_set_threads": (None, [I32]),
                "o_set_list_prefilter": (None, [I32]),
                "o_eval_range": (ctypes.c_int, [P, P, I32, P, I32, I32, P, P]),
                "o_get_threads": (ctypes.c_int, []),
                "o_lsd_window": (ctypes.c_int, [P, P, P, P, I64, I32, I32, P, P, P, P, P, P, P, P, P, P, P, P, P]),
                "o_lsd_run": (ctypes.c_int, [P, P, P, P, I64, I32, I32, P, P, P, P, P, P, P]),
                "o_plain_run": (ctypes.c_int, [P, P, P, I64, P, P, P, P, P, P]),
                "o_obabo_output": (None, [P, P, I64, P, P, P, P]),
                "o_obabo_enter": (ctypes.c_int, [P, P, P, I64, P, P]),
                "o_obabo_literal": (ctypes.c_int, [P, P, P, I64, P, P, P, P, P]),
                "o_force_match": (D, [P, P, I32, P, P, P]),
                "o_forces_subset": (ctypes.c_int, [P, P, P, I32, P, P]),
            }
            for name, (res, args) in sigs.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class _Keep:
    """Holds the numpy buffers behind the ctypes structures alive."""

    def __init__(self):
        self.items = []

    def arr(self, x, dtype):
        if x is None:
            return None
        a = np.ascontiguousarray(np.asarray(x, dtype=dtype))
        self.items.append(a)
        return a


def _csys(system, keep):
    s = _Sys()
    s.n_atoms = int(system.n_atoms)
    s.n_species = int(system.n_species)
    for a in range(3):
        s.box[a] = float(system.box[a])
    s.species = _ptr(keep.arr(system.species, np.int32))
    s.species_mass = _ptr(keep.arr(system.masses, np.float64))
    return s


def _cpot(pot, keep):
    p = _Pot()
    p.lj_eps = _ptr(keep.arr(getattr(pot, "lj_eps", None), np.float64))
    p.lj_sigma = _ptr(keep.arr(getattr(pot, "lj_sigma", None), np.float64))
    p.lj_cutoff = float(getattr(pot, "lj_cutoff", 0.0) or 0.0)
    p.n_rbf = int(getattr(pot, "n_rbf", 0) or 0)
    p.n_ang = int(getattr(pot, "n_ang", 0) or 0)
    p.n_layers = int(getattr(pot, "n_layers", 0) or 0)
    p.width = int(getattr(pot, "width", 0) or 0)
    p.desc_cutoff = float(getattr(pot, "desc_cutoff", 0.0) or 0.0)
    p.head = 1 if getattr(pot, "head", "tanh") == "linear" else 0
    p.head_scale = float(getattr(pot, "head_scale", 0.0) or 0.0)
    w = getattr(pot, "weights", None)
    p.weights = _ptr(keep.arr(w, np.float64)) if w is not None else None
    p.k_harm = float(getattr(pot, "k_harm", 0.0) or 0.0)
    p.q_ref = _ptr(keep.arr(getattr(pot, "q_ref", None), np.float64))
    p.shear = float(getattr(pot, "shear", 0.0) or 0.0)
    return p


SCHEMES = {"aboba": 0, "obabo": 1}


def _cprm(integ, seed):
    p = _Prm()
    p.dt = float(integ.dt)
    p.gamma = float(integ.gamma)
    p.temperature = float(integ.temperature)
    p.seed = int(seed)
    p.integrator = SCHEMES[getattr(integ, "scheme", "aboba")]
    return p


# ----------------------------------------------------------------------------------------------
# constants and random numbers
# ----------------------------------------------------------------------------------------------

def kappa() -> float:
    return _L().o_const_kappa()


def kboltz() -> float:
    return _L().o_const_kb()


def input_dim(n_species, n_rbf, n_ang) -> int:
    return int(_L().o_input_dim(n_species, n_rbf, n_ang))


def n_weights(d0, n_layers, width) -> int:
    return int(_L().o_n_weights(d0, n_layers, width))


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    _L().o_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def normals(seed, n, atom, stream=0):
    out = np.zeros(3, dtype=np.float64)
    _L().o_normals(int(seed), int(n), int(atom), int(stream), _ptr(out))
    return out


def uniform(seed, n):
    return float(_L().o_uniform(int(seed), int(n)))


def coefficients(system, integ):
    """(c1, aF, hm[S], sig[S]) of Eq. 4 as the oracle forms them."""
    keep = _Keep()
    s = _csys(system, keep)
    prm = _cprm(integ, 0)
    c1 = ctypes.c_double()
    aF = ctypes.c_double()
    hm = np.zeros(system.n_species)
    sg = np.zeros(system.n_species)
    _L().o_coefficients(ctypes.byref(s), ctypes.byref(prm), ctypes.byref(c1), ctypes.byref(aF), _ptr(hm), _ptr(sg))
    return c1.value, aF.value, hm, sg


def mb_momenta(system, integ, seed):
    keep = _Keep()
    s = _csys(system, keep)
    prm = _cprm(integ, seed)
    p = np.zeros((system.n_atoms, 3))
    _L().o_mb_momenta(ctypes.byref(s), ctypes.byref(prm), _ptr(p))
    return p


# ----------------------------------------------------------------------------------------------
# neighbours, energies and forces
# ----------------------------------------------------------------------------------------------

def fixpoint(system, q):
    keep = _Keep()
    s = _csys(system, keep)
    qq = keep.arr(q, np.float64)
    u = np.zeros((system.n_atoms, 3), dtype=np.uint32)
    m = np.zeros((system.n_atoms, 3), dtype=np.int64)
    _L().o_fixpoint_export(ctypes.byref(s), _ptr(qq), _ptr(u), _ptr(m))
    return u, m


def neighbors(system, q, rc, cap=1024):
    """Canonical neighbour lists: list of int32 arrays of packed keys (j << 5 | shift code)."""
    keep = _Keep()
    s = _csys(system, keep)
    qq = keep.arr(q, np.float64)
    keys = np.zeros((system.n_atoms, cap), dtype=np.int32)
    counts = np.zeros(system.n_atoms, dtype=np.int32)
    r = _L().o_neighbors(ctypes.byref(s), _ptr(qq), float(rc), int(cap), _ptr(keys), _ptr(counts))
    if r != 0:
        raise RuntimeError("oracle neighbour list exceeds capacity %d" % cap)
    return [keys[i, :counts[i]].copy() for i in range(system.n_atoms)]


def energy_forces(system, pot, q, want=("F",)):
    """Returns dict with E (total), and on request F [N,3], E_atom [N], X [N,d0], dEdX [N,d0]."""
    keep = _Keep()
    s = _csys(system, keep)
    p = _cpot(pot, keep)
    qq = keep.arr(q, np.float64)
    N = system.n_atoms
    out = {}
    F = np.zeros((N, 3)) if "F" in want else None
    Ea = np.zeros(N) if "E_atom" in want else None
    d0 = input_dim(system.n_species, p.n_rbf, p.n_ang) if p.n_layers > 0 else 0
    X = np.zeros((N, d0)) if "X" in want and d0 else None
    G = np.zeros((N, d0)) if "dEdX" in want and d0 else None
    E = _L().o_energy_forces(ctypes.byref(s), ctypes.byref(p), _ptr(qq), _ptr(F), _ptr(Ea), _ptr(X), _ptr(G))
    if np.isnan(E):
        raise RuntimeError("oracle neighbour list overflow")
    out["E"] = E
    for k, v in (("F", F), ("E_atom", Ea), ("X", X), ("dEdX", G)):
        if v is not None:
            out[k] = v
    return out


def energy(system, pot, q):
    return energy_forces(system, pot, q, want=())["E"]


def forces(system, pot, q):
    return energy_forces(system, pot, q, want=("F",))["F"]


# ----------------------------------------------------------------------------------------------
# transport, windows and trajectories
# ----------------------------------------------------------------------------------------------

def set_threads(n: int) -> None:
    """Threads of a window's verification loop (its K target evaluations, one per thread); 1 runs it serially.
    The results do not depend on the thread count."""
    _L().o_set_threads(int(n))


def set_list_prefilter(on: bool) -> None:
    """The conservative minimum-image pre-test of the neighbour lists (on by default; lists are the same either
    way)."""
    _L().o_set_list_prefilter(int(bool(on)))


def get_threads() -> int:
    return int(_L().o_get_threads())


def transport(sig, u, p_draft, mu_draft, mu_target):
    """reflectionVerify (Eq. 5) on flat vectors; returns (accept, p, log_ratio)."""
    sig = np.ascontiguousarray(sig, dtype=np.float64)
    pd = np.ascontiguousarray(p_draft, dtype=np.float64)
    md = np.ascontiguousarray(mu_draft, dtype=np.float64)
    mt = np.ascontiguousarray(mu_target, dtype=np.float64)
    out = np.zeros_like(pd)
    lr = ctypes.c_double()
    acc = _L().o_transport(int(pd.size), _ptr(sig), float(u), _ptr(pd), _ptr(md), _ptr(mt), _ptr(out),
                           ctypes.byref(lr))
    return bool(acc), out, lr.value


def transport_terms(sig, u, p_draft, mu_draft, mu_target):
    """reflectionVerify (Eq. 5) on flat vectors; returns (accept, p, log_ratio, z.delta, delta.delta)."""
    sig = np.ascontiguousarray(sig, dtype=np.float64)
    pd = np.ascontiguousarray(p_draft, dtype=np.float64)
    md = np.ascontiguousarray(mu_draft, dtype=np.float64)
    mt = np.ascontiguousarray(mu_target, dtype=np.float64)
    out = np.zeros_like(pd)
    lr, zd, dd = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    acc = _L().o_transport_terms(int(pd.size), _ptr(sig), float(u), _ptr(pd), _ptr(md), _ptr(mt), _ptr(out),
                                 ctypes.byref(lr), ctypes.byref(zd), ctypes.byref(dd))
    return bool(acc), out, lr.value, zd.value, dd.value


def lsd_window(system, draft, target, integ, seed, n0, K, q, p, ec_dF=None, max_commit=None):
    """One synchronous window (Alg. 1, L = K). Returns dict with the committed count, new state and window arrays."""
    keep = _Keep()
    s = _csys(system, keep)
    pd_ = _cpot(draft, keep)
    pt_ = _cpot(target, keep)
    prm = _cprm(integ, seed)
    N = system.n_atoms
    qq = np.array(q, dtype=np.float64).reshape(N, 3).copy()
    pp = np.array(p, dtype=np.float64).reshape(N, 3).copy()
    dF = None if ec_dF is None else np.array(ec_dF, dtype=np.float64).reshape(N, 3).copy()
    arrs = {k: np.zeros((K, N, 3)) for k in ("qmid", "pdraft", "mudraft", "Fdraft", "Ftarget")}
    logr, logu, dn = np.zeros(K), np.zeros(K), np.zeros(K)
    acc = np.zeros(K, dtype=np.int32)
    mc = K if max_commit is None else int(max_commit)
    pob = np.zeros((N, 3))
    nc = _L().o_lsd_window(ctypes.byref(s), ctypes.byref(pd_), ctypes.byref(pt_), ctypes.byref(prm), int(n0), int(K),
                           mc, _ptr(qq), _ptr(pp), _ptr(dF), _ptr(arrs["qmid"]), _ptr(arrs["pdraft"]),
                           _ptr(arrs["mudraft"]), _ptr(arrs["Fdraft"]), _ptr(arrs["Ftarget"]), _ptr(logr), _ptr(logu),
                           _ptr(dn), _ptr(acc), _ptr(pob))
    if nc < 0:
        raise RuntimeError("oracle window failed (%d)" % nc)
    out = dict(arrs)
    out.update(n_committed=nc, q=qq, p=pp, logr=logr, logu=logu, delta_norm=dn, accept=acc.astype(bool), ec_dF=dF,
               p_obabo=pob)
    return out


def lsd_run(system, draft, target, integ, seed, n_steps, K, q, p, step=0, use_ec=False, traj=False):
    keep = _Keep()
    s = _csys(system, keep)
    pd_ = _cpot(draft, keep)
    pt_ = _cpot(target, keep)
    prm = _cprm(integ, seed)
    N = system.n_atoms
    qq = np.array(q, dtype=np.float64).reshape(N, 3).copy()
    pp = np.array(p, dtype=np.float64).reshape(N, 3).copy()
    st = ctypes.c_int64(int(step))
    tq = np.zeros((n_steps, N, 3)) if traj else None
    tp = np.zeros((n_steps, N, 3)) if traj else None
    stats = np.zeros(6)
    pob = np.zeros((N, 3))
    r = _L().o_lsd_run(ctypes.byref(s), ctypes.byref(pd_), ctypes.byref(pt_), ctypes.byref(prm), int(n_steps), int(K),
                       int(bool(use_ec)), _ptr(qq), _ptr(pp), ctypes.byref(st), _ptr(tq), _ptr(tp), _ptr(stats),
                       _ptr(pob))
    if r != 0:
        raise RuntimeError("oracle LSD run failed (%d)" % r)
    keys = ("windows", "committed", "rejected", "pred_rejected", "sum_delta", "verified")
    return dict(q=qq, p=pp, step=st.value, traj_q=tq, traj_p=tp, stats=dict(zip(keys, stats.tolist())), p_obabo=pob)


def plain_run(system, target, integ, seed, n_steps, q, p, step=0, traj=False):
    keep = _Keep()
    s = _csys(system, keep)
    pt_ = _cpot(target, keep)
    prm = _cprm(integ, seed)
    N = system.n_atoms
    qq = np.array(q, dtype=np.float64).reshape(N, 3).copy()
    pp = np.array(p, dtype=np.float64).reshape(N, 3).copy()
    st = ctypes.c_int64(int(step))
    tq = np.zeros((n_steps, N, 3)) if traj else None
    tp = np.zeros((n_steps, N, 3)) if traj else None
    pob = np.zeros((N, 3))
    r = _L().o_plain_run(ctypes.byref(s), ctypes.byref(pt_), ctypes.byref(prm), int(n_steps), _ptr(qq), _ptr(pp),
                         ctypes.byref(st), _ptr(tq), _ptr(tp), _ptr(pob))
    if r != 0:
        raise RuntimeError("oracle plain run failed (%d)" % r)
    return dict(q=qq, p=pp, step=st.value, traj_q=tq, traj_p=tp, p_obabo=pob)


# ----------------------------------------------------------------------------------------------
# OBABO in the staggered frame (App. E)
# ----------------------------------------------------------------------------------------------

def obabo_output(system, integ, seed, n, p_prev, F, p_new):
    """The OBABO output momentum of staggered step n from the staggered momenta around it and its target force."""
    keep = _Keep()
    s = _csys(system, keep)
    prm = _cprm(integ, seed)
    out = np.zeros_like(np.asarray(p_new, np.float64))
    _L().o_obabo_output(ctypes.byref(s), ctypes.byref(prm), int(n), _ptr(keep.arr(p_prev, np.float64)),
                        _ptr(keep.arr(F, np.float64)), _ptr(keep.arr(p_new, np.float64)), _ptr(out))
    return out


def obabo_enter(system, target, integ, seed, n, q, p):
    """The staggered momentum OB(q, p) of an OBABO state at step index n."""
    keep = _Keep()
    s = _csys(system, keep)
    pt_ = _cpot(target, keep)
    prm = _cprm(integ, seed)
    pp = np.array(p, dtype=np.float64).copy()
    r = _L().o_obabo_enter(ctypes.byref(s), ctypes.byref(pt_), ctypes.byref(prm), int(n),
                           _ptr(keep.arr(q, np.float64)), _ptr(pp))
    if r != 0:
        raise RuntimeError("oracle OB step failed (%d)" % r)
    return pp


def obabo_literal(system, pot, integ, seed, n_steps, q, p, step=0, traj=False):
    """OBABO written out literally (O B A B O), for distribution tests of the staggered construction."""
    keep = _Keep()
    s = _csys(system, keep)
    pt_ = _cpot(pot, keep)
    prm = _cprm(integ, seed)
    N = system.n_atoms
    qq = np.array(q, dtype=np.float64).reshape(N, 3).copy()
    pp = np.array(p, dtype=np.float64).reshape(N, 3).copy()
    st = ctypes.c_int64(int(step))
    tq = np.zeros((n_steps, N, 3)) if traj else None
    tp = np.zeros((n_steps, N, 3)) if traj else None
    r = _L().o_obabo_literal(ctypes.byref(s), ctypes.byref(pt_), ctypes.byref(prm), int(n_steps), _ptr(qq), _ptr(pp),
                             ctypes.byref(st), _ptr(tq), _ptr(tp))
    if r != 0:
        raise RuntimeError("oracle literal OBABO failed (%d)" % r)
    return dict(q=qq, p=pp, step=st.value, traj_q=tq, traj_p=tp)


def force_match(system, draft, frames_q, frames_F, grad=True):
    """Force-matching loss of a linear-head draft and its exact gradient with respect to the packed weights."""
    keep = _Keep()
    s = _csys(system, keep)
    pd_ = _cpot(draft, keep)
    fq = keep.arr(frames_q, np.float64)
    fF = keep.arr(frames_F, np.float64)
    nf = fq.shape[0]
    g = np.zeros(len(draft.weights)) if grad else None
    loss = _L().o_force_match(ctypes.byref(s), ctypes.byref(pd_), int(nf), _ptr(fq), _ptr(fF), _ptr(g))
    return loss, g


def eval_range(system, pot, qs, i0, i1):
    """Centre-atom terms [i0, i1) of the energy and forces of configurations qs [C, N, 3] (run on set_threads()
    threads, one configuration each): (F [C, N, 3], E [C]).  Summed over a partition of the atoms it is
    energy_forces."""
    keep = _Keep()
    s = _csys(system, keep)
    p = _cpot(pot, keep)
    qq = keep.arr(qs, np.float64).reshape(-1, system.n_atoms, 3)
    C = qq.shape[0]
    F = np.zeros((C, system.n_atoms, 3))
    E = np.zeros(C)
    r = _L().o_eval_range(ctypes.byref(s), ctypes.byref(p), int(C), _ptr(qq), int(i0), int(i1), _ptr(F), _ptr(E))
    if r == -2:
        raise IndexError("atom range out of bounds")
    if r != 0:
        raise RuntimeError("oracle neighbour list overflow")
    return F, E


def forces_subset(system, pot, q, atoms):
    """Forces on the selected atoms only (for systems too large for a full oracle pass)."""
    keep = _Keep()
    s = _csys(system, keep)
    p = _cpot(pot, keep)
    qq = keep.arr(q, np.float64)
    sel = keep.arr(np.asarray(atoms), np.int32)
    out = np.zeros((sel.size, 3))
    r = _L().o_forces_subset(ctypes.byref(s), ctypes.byref(p), _ptr(qq), int(sel.size), _ptr(sel), _ptr(out))
    if r == -2:
        raise IndexError("atom index out of range")
    if r != 0:
        raise RuntimeError("oracle neighbour list overflow")
    return out
