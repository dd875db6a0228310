"""Thin Python binding of liblsd.so (include/lsd.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts numpy
arrays / torch CUDA tensors to pointers and error codes to exceptions.  It
fails loudly if the library is missing: there is no CPU fallback.

``LSD`` wraps one ``lsd_handle``; ``TargetEnergy`` is a ``torch.autograd.Function``
whose forward returns the target potential energy of a batch of configurations
and whose backward is the library's hand-written force adjoint (F = -dE/dq).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblsd.so")

LSD_OK = 0
ERRORS = {-1: "LSD_EINVAL", -2: "LSD_ENOMEM", -3: "LSD_ECUDA", -4: "LSD_ETIMEOUT", -5: "LSD_ENONFINITE",
          -6: "LSD_ESTATE", -7: "LSD_EOVERFLOW", -8: "LSD_EUNSUPPORTED"}
POT_LJ, POT_LJ_MLP, POT_LEARNED = 0, 1, 2
HEAD_TANH, HEAD_LINEAR = 0, 1
PRECISION = {"fp32": 0, "bf16": 1, "fp8": 2, "fp32-cuda-cores": 3, "fp32-tf32": 4}

# every symbol declared in include/lsd.h
SYMBOLS = ["lsd_init", "lsd_draft_window", "lsd_verify_window", "lsd_step", "lsd_plain_step", "lsd_enqueue_windows",
           "lsd_enqueue_plain", "lsd_get_state",
           "lsd_set_state", "lsd_get_stats", "lsd_set_stream", "lsd_set_draft_weights", "lsd_get_draft_weights",
           "lsd_set_error_correction", "lsd_set_integrator", "lsd_set_pipelining", "lsd_set_frame_capture", "lsd_frame_count", "lsd_train_draft",
           "lsd_force_match_dev", "lsd_target_forces_dev", "lsd_draft_forces_dev", "lsd_neighbors",
           "lsd_descriptors", "lsd_get_window", "lsd_profile_window", "lsd_checkpoint", "lsd_restore", "lsd_query",
           "lsd_target_mlp_static_dev", "lsd_destroy",
           "lsd_strerror", "lsd_launch_counts", "lsd_window_host", "lsd_transport_window", "lsd_get_frames",
           "lsd_set_max_displacement", "lsd_set_plain_fused", "lsd_set_grid_draft", "lsd_set_angular_moments", "lsd_get_angular_moments", "lsd_set_online_training", "lsd_online_status",
           "lsd_set_window_stages", "lsd_stage_launch_counts", "lsd_set_list_reuse",
           "lsd_set_list_skin", "lsd_get_list_skin"]


class LSDError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = "%s (%d): %s" % (ERRORS.get(code, "?"), code, _lib().lsd_strerror(code).decode())
        super().__init__(msg + ((" in " + what) if what else ""))


class lsd_system(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("n_species", ctypes.c_int32), ("pos", ctypes.c_void_p),
                ("mom", ctypes.c_void_p), ("species", ctypes.c_void_p), ("species_mass", ctypes.c_void_p),
                ("box", ctypes.c_double * 3), ("seed", ctypes.c_uint64)]


class lsd_potential(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("precision", ctypes.c_int32), ("lj_eps", ctypes.c_void_p),
                ("lj_sigma", ctypes.c_void_p), ("lj_cutoff", ctypes.c_double), ("n_rbf", ctypes.c_int32),
                ("n_ang", ctypes.c_int32), ("n_layers", ctypes.c_int32), ("width", ctypes.c_int32),
                ("desc_cutoff", ctypes.c_double), ("head", ctypes.c_int32), ("head_scale", ctypes.c_double),
                ("weights", ctypes.c_void_p), ("n_weights", ctypes.c_size_t)]


class lsd_stats(ctypes.Structure):
    _fields_ = [("windows", ctypes.c_int64), ("committed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("verified", ctypes.c_int64), ("sum_delta", ctypes.c_double), ("sum_pred_reject", ctypes.c_double),
                ("step", ctypes.c_int64), ("stages", ctypes.c_int64), ("list_builds", ctypes.c_int64)]


_L = None


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("liblsd.so not built (%s); run `python -m paper_2606_02455_b300.build`" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        P, I32, I64, D, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        sig = {
            "lsd_init": [P, P, P, D, D, D, I32, P],
            "lsd_draft_window": [P],
            "lsd_verify_window": [P, P, P],
            "lsd_step": [P, I64, P],
            "lsd_plain_step": [P, I64],
            "lsd_enqueue_windows": [P, I32],
            "lsd_enqueue_plain": [P, I32],
            "lsd_get_state": [P, P, P, P],
            "lsd_set_state": [P, P, P, I64],
            "lsd_get_stats": [P, P],
            "lsd_set_stream": [P, P],
            "lsd_set_draft_weights": [P, P, SZ],
            "lsd_get_draft_weights": [P, P, SZ],
            "lsd_set_error_correction": [P, I32],
            "lsd_set_integrator": [P, I32],
            "lsd_set_pipelining": [P, I32],
            "lsd_set_frame_capture": [P, I64],
            "lsd_frame_count": [P, P],
            "lsd_train_draft": [P, I32, ctypes.c_float, I32, P],
            "lsd_force_match_dev": [P, P, P, I32, P, P],
            "lsd_target_forces_dev": [P, P, I32, P, P],
            "lsd_draft_forces_dev": [P, P, I32, P, P],
            "lsd_neighbors": [P, I32, I32, P, P, P, P],
            "lsd_descriptors": [P, I32, P, P],
            "lsd_get_window": [P, P, P, P, P, P, P, P, P],
            "lsd_checkpoint": [P, P, P],
            "lsd_restore": [P, P, SZ],
            "lsd_query": [P, P, P, P, P],
            "lsd_launch_counts": [P, P, P, P],
            "lsd_window_host": [P, P, P, ctypes.c_int64, P, P, P, P],
            "lsd_target_mlp_static_dev": [P, P, I32, P, P],
            "lsd_profile_window": [P, P, I32],
            "lsd_transport_window": [P, P, P, P, P, I32, P, P],
            "lsd_get_frames": [P, I64, I64, P, P],
            "lsd_set_max_displacement": [P, D],
            "lsd_set_plain_fused": [P, I32],
            "lsd_set_grid_draft": [P, I32],
            "lsd_set_angular_moments": [P, I32],
            "lsd_get_angular_moments": [P, ctypes.POINTER(ctypes.c_int32)],
            "lsd_set_online_training": [P, I64, I32, ctypes.c_float, I32],
            "lsd_online_status": [P, P, P],
            "lsd_set_window_stages": [P, I32],
            "lsd_stage_launch_counts": [P, P, P],
            "lsd_set_list_reuse": [P, I32],
            "lsd_set_list_skin": [P, D],
            "lsd_get_list_skin": [P, P],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.lsd_destroy.argtypes = [P]
        lib.lsd_destroy.restype = None
        lib.lsd_strerror.argtypes = [ctypes.c_int]
        lib.lsd_strerror.restype = ctypes.c_char_p
        _L = lib
    return _L


def load():
    """Loads the library (raises if it is missing)."""
    return _lib()


def _check(code, what=""):
    if code != LSD_OK:
        raise LSDError(code, what)


def _p(a):
    return None if a is None else a.ctypes.data


def _tp(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _cpot(pot, keep):
    cp = lsd_potential()
    mlp = (getattr(pot, "n_layers", 0) or 0) > 0
    if not mlp:
        cp.kind = POT_LJ
    else:
        cp.kind = POT_LEARNED if pot.head == "linear" else POT_LJ_MLP
    cp.precision = PRECISION[getattr(pot, "precision", "fp32")]
    if pot.lj_eps is not None:
        e = np.ascontiguousarray(pot.lj_eps, dtype=np.float64)
        s = np.ascontiguousarray(pot.lj_sigma, dtype=np.float64)
        keep += [e, s]
        cp.lj_eps, cp.lj_sigma = _p(e), _p(s)
    cp.lj_cutoff = float(pot.lj_cutoff or 0.0)
    cp.n_rbf, cp.n_ang, cp.n_layers, cp.width = int(pot.n_rbf), int(pot.n_ang), int(pot.n_layers), int(pot.width)
    cp.desc_cutoff = float(pot.desc_cutoff or 0.0)
    cp.head = HEAD_LINEAR if pot.head == "linear" else HEAD_TANH
    cp.head_scale = float(pot.head_scale)
    if mlp:
        w = np.ascontiguousarray(pot.weights, dtype=np.float32)
        keep.append(w)
        cp.weights, cp.n_weights = _p(w), w.size
    return cp


def _torch():
    import torch
    return torch


class LSD:
    """One simulation handle: system, draft and target potentials, ABOBA parameters and window length K."""

    def __init__(self, system, draft, target, integ, K=None, momenta="given"):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("liblsd needs a CUDA device")
        torch.cuda.init()
        lib = _lib()
        keep = []
        pos = np.ascontiguousarray(system.positions, dtype=np.float64)
        mom = np.ascontiguousarray(system.momenta, dtype=np.float64) if momenta == "given" else None
        spc = np.ascontiguousarray(system.species, dtype=np.int32)
        mas = np.ascontiguousarray(system.masses, dtype=np.float64)
        keep += [pos, spc, mas] + ([mom] if mom is not None else [])
        cs = lsd_system()
        cs.n_atoms, cs.n_species = pos.shape[0], mas.size
        cs.pos, cs.mom, cs.species, cs.species_mass = _p(pos), _p(mom), _p(spc), _p(mas)
        for a in range(3):
            cs.box[a] = float(system.box[a])
        cs.seed = int(system.seed)
        cd = _cpot(draft, keep)
        ct = _cpot(target, keep)
        self.K = int(K if K is not None else integ.K)
        self.N = pos.shape[0]
        self.h = ctypes.c_void_p()
        _check(lib.lsd_init(ctypes.byref(cs), ctypes.byref(cd), ctypes.byref(ct), float(integ.gamma),
                            float(integ.dt), float(integ.temperature), self.K, ctypes.byref(self.h)), "lsd_init")
        self.dt = float(integ.dt)
        self.n_draft_weights = 0 if draft.weights is None or not draft.n_layers else int(np.asarray(draft.weights).size)
        self._target = target
        if getattr(integ, "scheme", "aboba") != "aboba":
            self.set_integrator(integ.scheme)

    # -- lifecycle ---------------------------------------------------------------------------------------
    def close(self):
        if self.h:
            _lib().lsd_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the method -------------------------------------------------------------------------------------
    def draft_window(self):
        _check(_lib().lsd_draft_window(self.h), "lsd_draft_window")

    def verify_window(self):
        nc, fr = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib().lsd_verify_window(self.h, ctypes.byref(nc), ctypes.byref(fr)), "lsd_verify_window")
        return nc.value, fr.value

    def transport_window(self, q_mid, p_draft, F_draft, F_target):
        """reflectionVerify and commit on a given window (lsd_transport_window): [k, N, 3] arrays, float64 for
        q_mid and p_draft, float32 forces.  Returns (committed count, first rejected step or -1)."""
        k = int(np.asarray(q_mid).shape[0])
        arrs = [np.ascontiguousarray(q_mid, dtype=np.float64), np.ascontiguousarray(p_draft, dtype=np.float64),
                np.ascontiguousarray(F_draft, dtype=np.float32), np.ascontiguousarray(F_target, dtype=np.float32)]
        for a in arrs:
            assert a.shape == (k, self.N, 3)
        nc, fr = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib().lsd_transport_window(self.h, *[_p(a) for a in arrs], k, ctypes.byref(nc), ctypes.byref(fr)),
               "lsd_transport_window")
        return nc.value, fr.value

    def step(self, n_steps):
        st = lsd_stats()
        _check(_lib().lsd_step(self.h, int(n_steps), ctypes.byref(st)), "lsd_step")
        return _stats_dict(st)

    def plain_step(self, n_steps):
        _check(_lib().lsd_plain_step(self.h, int(n_steps)), "lsd_plain_step")

    def enqueue_windows(self, n=1):
        """Enqueue n window graphs on the handle's stream without waiting."""
        _check(_lib().lsd_enqueue_windows(self.h, int(n)), "lsd_enqueue_windows")

    def enqueue_plain(self, n=1):
        """Enqueue n plain target steps on the handle's stream without waiting."""
        _check(_lib().lsd_enqueue_plain(self.h, int(n)), "lsd_enqueue_plain")

    def stats(self):
        st = lsd_stats()
        _check(_lib().lsd_get_stats(self.h, ctypes.byref(st)), "lsd_get_stats")
        return _stats_dict(st)

    def get_state(self, pos=None, mom=None):
        pos = np.zeros((self.N, 3)) if pos is None else pos
        mom = np.zeros((self.N, 3)) if mom is None else mom
        step = ctypes.c_int64()
        _check(_lib().lsd_get_state(self.h, _p(pos), _p(mom), ctypes.byref(step)), "lsd_get_state")
        return pos, mom, step.value

    def set_state(self, pos, mom, step):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        mom = np.ascontiguousarray(mom, dtype=np.float64)
        _check(_lib().lsd_set_state(self.h, _p(pos), _p(mom), int(step)), "lsd_set_state")

    def window_host(self, pos, mom, step, pos_out=None, mom_out=None):
        """One window from a host state (lsd_window_host): numpy float64 [N, 3] arrays (pinned memory makes the
        copies asynchronous); pos_out / mom_out default to pos / mom.  Returns (new step, committed count)."""
        pos_out = pos if pos_out is None else pos_out
        mom_out = mom if mom_out is None else mom_out
        for a in (pos, mom, pos_out, mom_out):
            assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"] and a.shape == (self.N, 3)
        st = ctypes.c_int64()
        nc = ctypes.c_int32()
        _check(_lib().lsd_window_host(self.h, _p(pos), _p(mom), int(step), _p(pos_out), _p(mom_out),
                                      ctypes.byref(st), ctypes.byref(nc)), "lsd_window_host")
        return st.value, nc.value

    def set_stream(self, stream=None):
        ptr = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        _check(_lib().lsd_set_stream(self.h, ptr), "lsd_set_stream")

    def set_pipelining(self, on=True):
        """Overlap the draft of window w+1 with the verification of window w (lsd_set_pipelining)."""
        _check(_lib().lsd_set_pipelining(self.h, int(bool(on))), "lsd_set_pipelining")

    def set_window_stages(self, steps_per_stage):
        """Verify each window in stages of this many steps, stopping at the first rejection (0: one pass)."""
        _check(_lib().lsd_set_window_stages(self.h, int(steps_per_stage)), "lsd_set_window_stages")

    def set_list_reuse(self, on=True):
        """Keep the Verlet lists of unpipelined windows while the committed state stays within half the
        displacement bound of their base (lsd_set_list_reuse)."""
        _check(_lib().lsd_set_list_reuse(self.h, int(bool(on))), "lsd_set_list_reuse")

    def set_list_skin(self, skin):
        """The Verlet lists' skin in Angstrom, at most the planned one (lsd_set_list_skin)."""
        _check(_lib().lsd_set_list_skin(self.h, ctypes.c_double(skin)), "lsd_set_list_skin")

    def list_skin(self):
        v = ctypes.c_double()
        _check(_lib().lsd_get_list_skin(self.h, ctypes.byref(v)), "lsd_get_list_skin")
        return v.value

    SCHEMES = {"aboba": 0, "obabo": 1}

    def set_integrator(self, scheme):
        """"aboba" (Eq. 2) or "obabo" (the staggered frame of App. E; entering it evaluates the target once)."""
        _check(_lib().lsd_set_integrator(self.h, self.SCHEMES[scheme]), "lsd_set_integrator")

    def set_plain_fused(self, on=True):
        """Plain target steps in one fused cooperative launch per call (on) or one graph of kernels per step (off)."""
        _check(_lib().lsd_set_plain_fused(self.h, int(bool(on))), "lsd_set_plain_fused")

    def set_angular_moments(self, on=True):
        """The target's angular descriptors and adjoint through Cartesian moments (O(n)) or the pair sums (O(n^2))."""
        _check(_lib().lsd_set_angular_moments(self.h, int(bool(on))), "lsd_set_angular_moments")

    def angular_moments(self):
        """Whether the target's angular block runs by moments."""
        v = ctypes.c_int32()
        _check(_lib().lsd_get_angular_moments(self.h, ctypes.byref(v)), "lsd_get_angular_moments")
        return bool(v.value)

    def set_grid_draft(self, on=True):
        """Drafts in the grid form (one CTA per SM, grid-wide barriers; large systems) or in one cluster (off)."""
        _check(_lib().lsd_set_grid_draft(self.h, int(bool(on))), "lsd_set_grid_draft")

    def set_max_displacement(self, d_max):
        """End windows early once an atom moves d_max Angstrom from its lists' base (0 restores the default)."""
        _check(_lib().lsd_set_max_displacement(self.h, float(d_max)), "lsd_set_max_displacement")

    def set_error_correction(self, on=True):
        _check(_lib().lsd_set_error_correction(self.h, int(bool(on))), "lsd_set_error_correction")

    # -- learned draft ----------------------------------------------------------------------------------
    def set_draft_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(_lib().lsd_set_draft_weights(self.h, _p(w), w.size), "lsd_set_draft_weights")

    def get_draft_weights(self):
        w = np.zeros(self.n_draft_weights, dtype=np.float32)
        _check(_lib().lsd_get_draft_weights(self.h, _p(w), w.size), "lsd_get_draft_weights")
        return w

    def set_frame_capture(self, capacity):
        _check(_lib().lsd_set_frame_capture(self.h, int(capacity)), "lsd_set_frame_capture")

    def frame_count(self):
        n = ctypes.c_int64()
        _check(_lib().lsd_frame_count(self.h, ctypes.byref(n)), "lsd_frame_count")
        return n.value

    def get_frames(self, first, count):
        """Captured frames first .. first+count-1 (lsd_get_frames): q_mid [count, N, 3] float64, F_target float32."""
        q = np.zeros((count, self.N, 3))
        F = np.zeros((count, self.N, 3), np.float32)
        _check(_lib().lsd_get_frames(self.h, int(first), int(count), _p(q), _p(F)), "lsd_get_frames")
        return q, F

    def set_online_training(self, every_accepted, n_iters=100, lr=3e-3, frames_per_iter=0):
        """Retrain the learned draft during step() every `every_accepted` accepted steps (0: off)."""
        _check(_lib().lsd_set_online_training(self.h, int(every_accepted), int(n_iters), float(lr),
                                              int(frames_per_iter)), "lsd_set_online_training")

    def online_status(self):
        n, l = ctypes.c_int64(), ctypes.c_float()
        _check(_lib().lsd_online_status(self.h, ctypes.byref(n), ctypes.byref(l)), "lsd_online_status")
        return n.value, l.value

    def train_draft(self, n_iters, lr, frames_per_iter=0):
        loss = ctypes.c_float()
        _check(_lib().lsd_train_draft(self.h, int(n_iters), float(lr), int(frames_per_iter), ctypes.byref(loss)),
               "lsd_train_draft")
        return loss.value

    def force_match(self, frames_q, frames_F, want_grad=True):
        """Loss and gradient of the learned draft on frames (torch CUDA tensors [F,N,3]: float64 q, float32 F)."""
        torch = _torch()
        fq = frames_q.contiguous()
        fF = frames_F.contiguous()
        assert fq.is_cuda and fq.dtype == torch.float64 and fF.dtype == torch.float32
        g = torch.zeros(self.n_draft_weights, dtype=torch.float32, device=fq.device) if want_grad else None
        loss = ctypes.c_float()
        _check(_lib().lsd_force_match_dev(self.h, _tp(fq), _tp(fF), fq.shape[0], ctypes.byref(loss), _tp(g)),
               "lsd_force_match_dev")
        return loss.value, g

    # -- batched force evaluations ------------------------------------------------------------------------
    def _forces(self, fn, q, energies):
        torch = _torch()
        q = q.contiguous()
        assert q.is_cuda and q.dtype == torch.float64 and q.shape[-2:] == (self.N, 3)
        q3 = q.reshape(-1, self.N, 3)
        C = q3.shape[0]
        F = torch.empty((C, self.N, 3), dtype=torch.float32, device=q.device)
        E = torch.empty((C, self.N), dtype=torch.float32, device=q.device) if energies else None
        torch.cuda.current_stream().synchronize()
        _check(fn(self.h, _tp(q3), C, _tp(F), _tp(E)), "forces")
        return (F, E) if energies else F

    def target_forces(self, q, energies=False):
        return self._forces(_lib().lsd_target_forces_dev, q, energies)

    def draft_forces(self, q, energies=False):
        return self._forces(_lib().lsd_draft_forces_dev, q, energies)

    # -- inspection (parity tests) -------------------------------------------------------------------------
    def launch_counts(self):
        """Kernels of this library per window, per pipelined round and per plain step."""
        w, r, p = (ctypes.c_int32() for _ in range(3))
        _check(_lib().lsd_launch_counts(self.h, ctypes.byref(w), ctypes.byref(r), ctypes.byref(p)),
               "lsd_launch_counts")
        return dict(window=w.value, round=r.value, plain=p.value)

    def stage_launch_counts(self):
        """Kernels of a staged window's first stage and of each later stage (lsd_stage_launch_counts)."""
        f, l = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib().lsd_stage_launch_counts(self.h, ctypes.byref(f), ctypes.byref(l)), "lsd_stage_launch_counts")
        return dict(first=f.value, later=l.value)

    def query(self):
        K, N, d, cap = (ctypes.c_int32() for _ in range(4))
        _check(_lib().lsd_query(self.h, ctypes.byref(K), ctypes.byref(N), ctypes.byref(d), ctypes.byref(cap)))
        return dict(K=K.value, n_atoms=N.value, d_in=d.value, nb_cap=cap.value)

    def neighbors(self, config=0, cap=None):
        cap = cap or self.query()["nb_cap"]
        dk = np.zeros((self.N, cap), np.int32)
        dc = np.zeros(self.N, np.int32)
        lk = np.zeros((self.N, cap), np.int32)
        lc = np.zeros(self.N, np.int32)
        _check(_lib().lsd_neighbors(self.h, int(config), int(cap), _p(dk), _p(dc), _p(lk), _p(lc)), "lsd_neighbors")
        return [dk[i, :dc[i]].copy() for i in range(self.N)], [lk[i, :lc[i]].copy() for i in range(self.N)]

    def descriptors(self, n_configs):
        d = self.query()["d_in"]
        X = np.zeros((n_configs, self.N, d), np.float32)
        G = np.zeros((n_configs, self.N, d), np.float32)
        _check(_lib().lsd_descriptors(self.h, int(n_configs), _p(X), _p(G)), "lsd_descriptors")
        return X, G

    def get_window(self):
        K, N = self.K, self.N
        out = dict(q_mid=np.zeros((K, N, 3)), p_draft=np.zeros((K, N, 3)), F_draft=np.zeros((K, N, 3), np.float32),
                   F_target=np.zeros((K, N, 3), np.float32), log_ratio=np.zeros(K), log_u=np.zeros(K),
                   delta_norm=np.zeros(K), accept=np.zeros(K, np.int32))
        _check(_lib().lsd_get_window(self.h, *[_p(out[k]) for k in ("q_mid", "p_draft", "F_draft", "F_target",
                                                                    "log_ratio", "log_u", "delta_norm", "accept")]),
               "lsd_get_window")
        out["accept"] = out["accept"].astype(bool)
        return out

    PHASES = ("draft", "neighbors", "descriptors", "mlp", "pair_grad", "force_gather", "transport_reduce",
              "transport_commit", "verlet_lists")

    def profile_window(self):
        """One window with CUDA events between its kernels: {phase: milliseconds}."""
        ms = np.zeros(len(self.PHASES))
        _check(_lib().lsd_profile_window(self.h, _p(ms), len(self.PHASES)), "lsd_profile_window")
        return dict(zip(self.PHASES, ms.tolist()))

    def checkpoint(self):
        n = ctypes.c_size_t()
        _check(_lib().lsd_checkpoint(self.h, None, ctypes.byref(n)), "lsd_checkpoint")
        buf = ctypes.create_string_buffer(n.value)
        _check(_lib().lsd_checkpoint(self.h, buf, ctypes.byref(n)), "lsd_checkpoint")
        return buf.raw[:n.value]

    def restore(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(_lib().lsd_restore(self.h, buf, len(blob)), "lsd_restore")


def _stats_dict(st):
    return dict(windows=st.windows, committed=st.committed, rejected=st.rejected, verified=st.verified,
                sum_delta=st.sum_delta, pred_rejected=st.sum_pred_reject, step=st.step, stages=st.stages,
                list_builds=st.list_builds)


def _make_target_energy():
    torch = _torch()

    class TargetEnergy(torch.autograd.Function):
        """E(q) = sum of per-atom target energies of each configuration; backward by the force adjoint."""

        @staticmethod
        def forward(ctx, q, handle):
            F, E = handle.target_forces(q.detach(), energies=True)
            ctx.save_for_backward(F)
            return E.sum(dim=1).to(q.dtype)

        @staticmethod
        def backward(ctx, gE):
            (F,) = ctx.saved_tensors
            return -(F.to(gE.dtype) * gE[:, None, None]), None

    return TargetEnergy


_TE = None


def target_energy(q, handle):
    """torch.autograd entry point: energies of configurations q [C,N,3] (float64, CUDA)."""
    global _TE
    if _TE is None:
        _TE = _make_target_energy()
    return _TE.apply(q, handle)
