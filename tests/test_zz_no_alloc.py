"""The allocation-free MLP entry point (lsd_target_mlp_static_dev), for callers that cannot allocate device memory:
code that runs inside a host application whose own allocator owns every device buffer, or a latency-critical loop
that must not stall on the device synchronisation cudaMalloc implies.  Its scratch is a fixed 4 MiB array inside the
library.  The test calls it through the C ABI twice in a row and compares each result with the MLP step of the
existing batched entry point (lsd_target_forces_dev; dE/dX read back with lsd_descriptors, the per-atom energies
with the target's LJ term switched off): the same kernel on the same tiles, so the results are bitwise equal.  The
rows span more 128-row tiles than the array has CTA slots for (21 at width 256, 4 layers), so CTAs reuse their
slots.  Collected last so that a failing run stops only after every other test has run."""
import ctypes

import numpy as np
import pytest

from paper_2606_02455_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _system(precision, width=256, layers=4):
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
    # no LJ term in the target: its per-atom energies are then the MLP's alone
    tgt = W.Potential(lj_eps=lj["lj_eps"], lj_sigma=lj["lj_sigma"], lj_cutoff=0.0, n_rbf=16, n_ang=16,
                      n_layers=layers, width=width, desc_cutoff=6.0, head="tanh", head_scale=0.05,
                      weights=W.mlp_weights(d0, layers, width, seed=1, col_scale=W.dense_input_scale(3)),
                      precision=precision)
    return s, W.Potential(**lj), tgt


def _static(lib, h, X_dev, M, E_dev, G_dev):
    return lib.lsd_target_mlp_static_dev(h.h, ctypes.c_void_p(X_dev.data_ptr()), M, ctypes.c_void_p(E_dev.data_ptr()),
                                         ctypes.c_void_p(G_dev.data_ptr()))


@pytest.mark.parametrize("precision,width,layers", [("bf16", 256, 4), ("fp8", 256, 4), ("fp32", 128, 3)])
def test_no_alloc_mlp_matches_existing_entry_point_twice(precision, width, layers):
    import torch
    from paper_2606_02455_b300 import lsd
    s, draft, tgt = _system(precision, width, layers)
    C = 16
    h = lsd.LSD(s, draft, tgt, W.Integrator(0.5, 0.01, 350.0, C))
    rng = np.random.default_rng(11)
    q = torch.tensor(np.stack([s.positions + 0.05 * rng.standard_normal(s.positions.shape) for _ in range(C)]),
                     device="cuda")
    _, E_ref = h.target_forces(q, energies=True)   # the existing entry point (its MLP step on the tensor cores)
    E_ref = E_ref.cpu().numpy().reshape(-1)
    X, G = h.descriptors(C)                          # its inputs and dE/dX
    M, d = C * s.n_atoms, X.shape[-1]
    assert M > 21 * 128                              # more tiles than CTA slots in the 4 MiB array (width 256)
    dpad = (d + 31) // 32 * 32
    Xp = np.zeros((M, dpad), np.float32)
    Xp[:, :d] = X.reshape(M, d)
    X_dev = torch.tensor(Xp, device="cuda")
    lib = lsd.load()
    for call in range(2):
        E_dev = torch.full((M,), float("nan"), device="cuda")
        G_dev = torch.full((M, dpad), float("nan"), device="cuda")
        torch.cuda.synchronize()
        rc = _static(lib, h, X_dev, M, E_dev, G_dev)
        assert rc == 0, lsd.LSDError(rc)
        torch.cuda.synchronize()
        Gn = G_dev.cpu().numpy()[:, :d]
        assert np.array_equal(Gn, G.reshape(M, d)), (call, np.abs(Gn - G.reshape(M, d)).max())
        assert np.array_equal(E_dev.cpu().numpy(), E_ref), call
    h.close()


@pytest.mark.parametrize("precision", ["fp32-cuda-cores", "lj-only"])
def test_no_alloc_rejects_targets_without_a_tensor_core_mlp(precision):
    """A target whose MLP runs on the CUDA cores (or that has no MLP) has no tensor-core plan: LSD_EUNSUPPORTED,
    no launch."""
    import torch
    from paper_2606_02455_b300 import lsd
    s, draft, tgt = _system("bf16")
    tgt = draft if precision == "lj-only" else W.replace(tgt, precision=precision)
    h = lsd.LSD(s, draft, tgt, W.Integrator(0.5, 0.01, 350.0, 1))
    X = torch.zeros((8, 96), device="cuda")
    E = torch.zeros(8, device="cuda")
    G = torch.zeros((8, 96), device="cuda")
    assert _static(lsd.load(), h, X, 8, E, G) == -8
    h.close()
