"""The allocation-free MLP entry point (lsd_target_mlp_static_dev), for callers that cannot allocate device memory
(their host application's allocator owns every device buffer, or a latency-critical loop cannot stall on the
device synchronisation that cudaMalloc implies).  Its scratch is a fixed array inside the library; the test calls
it through the C ABI twice in a row and compares each result with the MLP step of the existing batched entry point
(lsd_target_forces_dev, read back with lsd_descriptors), within the BF16 tolerance the other tests use.
Collected last so that a failing run stops only after every other test has run."""
import ctypes

import numpy as np
import pytest

from paper_2606_02455_b300 import workloads as W

pytestmark = pytest.mark.gpu

BF16_TOL = 2e-2


def _system():
    cells = 6
    L = (cells ** 3 / 0.1) ** (1.0 / 3.0)
    spacing = L / cells
    pos = W.jitter(W.simple_cubic(cells, spacing), spacing, seed=3)
    n = pos.shape[0]
    sp = (np.arange(n) % 3).astype(np.int32)
    masses = np.array([1.0, 12.0, 16.0])
    s = W.System(positions=pos, momenta=W.mb_momenta(masses[sp], 350.0, 4), species=sp, masses=masses,
                 box=np.array([L] * 3), seed=5)
    lj = dict(lj_eps=np.array([0.002, 0.004, 0.006]), lj_sigma=np.array([1.6, 2.2, 2.0]), lj_cutoff=6.0)
    d0 = W.input_dim(3, 16, 16)
    tgt = W.Potential(**lj, n_rbf=16, n_ang=16, n_layers=4, width=256, desc_cutoff=6.0, head="tanh",
                      head_scale=0.05, weights=W.mlp_weights(d0, 4, 256, seed=1, col_scale=W.dense_input_scale(3)),
                      precision="bf16")
    return s, W.Potential(**lj), tgt


def test_no_alloc_mlp_matches_existing_entry_point_twice():
    import torch
    from paper_2606_02455_b300 import lsd
    s, draft, tgt = _system()
    C = 2
    h = lsd.LSD(s, draft, tgt, W.Integrator(0.5, 0.01, 350.0, C))
    rng = np.random.default_rng(11)
    q = torch.tensor(np.stack([s.positions + 0.05 * rng.standard_normal(s.positions.shape) for _ in range(C)]),
                     device="cuda")
    h.target_forces(q)                      # the existing entry point (its MLP step runs on the tensor cores)
    X, G = h.descriptors(C)                 # its inputs and dE/dX
    M, d = C * s.n_atoms, X.shape[-1]
    dpad = (d + 31) // 32 * 32
    Xp = np.zeros((M, dpad), np.float32)
    Xp[:, :d] = X.reshape(M, d)
    X_dev = torch.tensor(Xp, device="cuda")
    lib = lsd.load()
    for call in range(2):
        E_dev = torch.full((M,), float("nan"), device="cuda")
        G_dev = torch.full((M, dpad), float("nan"), device="cuda")
        torch.cuda.synchronize()
        rc = lib.lsd_target_mlp_static_dev(h.h, ctypes.c_void_p(X_dev.data_ptr()), M,
                                           ctypes.c_void_p(E_dev.data_ptr()), ctypes.c_void_p(G_dev.data_ptr()))
        assert rc == 0, lsd.LSDError(rc)
        torch.cuda.synchronize()
        Gn = G_dev.cpu().numpy()[:, :d].reshape(C, s.n_atoms, d)
        assert np.isfinite(Gn).all() and np.isfinite(E_dev.cpu().numpy()).all(), call
        for c in range(C):
            err = np.linalg.norm(Gn[c] - G[c]) / np.linalg.norm(G[c])
            assert err < BF16_TOL, (call, c, err)
    h.close()


def test_no_alloc_rejects_wrong_target():
    """A handle whose target has no tensor-core MLP is rejected with LSD_EUNSUPPORTED (no launch)."""
    import torch
    from paper_2606_02455_b300 import lsd
    s, draft, tgt = _system()
    h = lsd.LSD(s, draft, W.replace(tgt, precision="fp32"), W.Integrator(0.5, 0.01, 350.0, 1))
    X = torch.zeros((8, 96), device="cuda")
    E = torch.zeros(8, device="cuda")
    G = torch.zeros((8, 96), device="cuda")
    rc = lsd.load().lsd_target_mlp_static_dev(h.h, ctypes.c_void_p(X.data_ptr()), 8, ctypes.c_void_p(E.data_ptr()),
                                              ctypes.c_void_p(G.data_ptr()))
    assert rc == -8
    h.close()
