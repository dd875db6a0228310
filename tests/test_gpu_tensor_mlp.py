"""GPU parity of the tensor-core (tcgen05, BF16 operands, FP32 accumulation) MLP path against the FP64 oracle,
on the config-4 target architecture (67 -> 256 x4 -> 1, 3 species, 6 A cutoffs, rho = 0.1/A^3).
Tolerance: BF16 paths within 2e-2 relative per configuration (norm over atoms)."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W

pytestmark = pytest.mark.gpu

BF16_TOL = 2e-2


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _system(cells=8, precision="bf16", width=256, layers=4, seed=0):
    L = (cells ** 3 / 0.1) ** (1.0 / 3.0)
    spacing = L / cells
    pos = W.jitter(W.simple_cubic(cells, spacing), spacing, seed=seed)
    n = pos.shape[0]
    sp = (np.arange(n) % 3).astype(np.int32)
    masses = np.array([1.0, 12.0, 16.0])
    s = W.System(positions=pos, momenta=W.mb_momenta(masses[sp], 350.0, 4), species=sp, masses=masses,
                 box=np.array([L] * 3), seed=21)
    lj = dict(lj_eps=np.array([0.002, 0.004, 0.006]), lj_sigma=np.array([1.6, 2.2, 2.0]), lj_cutoff=6.0)
    d0 = W.input_dim(3, 16, 16)
    tgt = W.Potential(**lj, n_rbf=16, n_ang=16, n_layers=layers, width=width, desc_cutoff=6.0, head="tanh",
                      head_scale=0.05, weights=W.mlp_weights(d0, layers, width, seed=1,
                                                            col_scale=W.dense_input_scale(3)), precision=precision)
    return s, W.Potential(**lj), tgt


@pytest.mark.parametrize("width,layers", [(256, 4), (64, 2)])
def test_tensor_core_mlp_matches_oracle(width, layers):
    import torch
    from paper_2606_02455_b300 import lsd
    s, draft, tgt = _system(width=width, layers=layers)
    integ = W.Integrator(0.5, 0.01, 350.0, 4)
    h = lsd.LSD(s, draft, tgt, integ)
    rng = np.random.default_rng(5)
    qs = np.stack([s.positions + 0.05 * rng.standard_normal(s.positions.shape) for _ in range(4)])
    F, E = h.target_forces(torch.tensor(qs, device="cuda"), energies=True)
    F, E = F.cpu().numpy(), E.cpu().numpy()
    X, G = h.descriptors(4)
    for c in range(4):
        ref = O.energy_forces(s, tgt, qs[c], want=("F", "X", "dEdX", "E_atom"))
        assert _rel(X[c], ref["X"]) < 1e-5                       # descriptors stay FP32
        assert _rel(G[c], ref["dEdX"]) < BF16_TOL, _rel(G[c], ref["dEdX"])
        assert _rel(F[c], ref["F"]) < BF16_TOL, _rel(F[c], ref["F"])
        e_mlp_ref = ref["E_atom"] - O.energy_forces(s, draft, qs[c], want=("E_atom",))["E_atom"]
        e_mlp_gpu = E[c].astype(np.float64) - O.energy_forces(s, draft, qs[c], want=("E_atom",))["E_atom"]
        assert _rel(e_mlp_gpu, e_mlp_ref) < BF16_TOL
    h.close()


def test_tensor_core_bf16_against_fp32_cuda_core_path():
    """The same weights through the FP32 CUDA-core kernel and the BF16 tensor-core kernel agree to BF16 precision."""
    import torch
    from paper_2606_02455_b300 import lsd
    s, draft, tgt = _system(cells=6)
    integ = W.Integrator(0.5, 0.01, 350.0, 2)
    q = torch.tensor(np.stack([s.positions, s.positions + 0.03]), device="cuda")
    hb = lsd.LSD(s, draft, tgt, integ)
    hf = lsd.LSD(s, draft, W.replace(tgt, precision="fp32"), integ)
    Fb = hb.target_forces(q).cpu().numpy()
    Ff = hf.target_forces(q).cpu().numpy()
    _, Gb = hb.descriptors(2)
    _, Gf = hf.descriptors(2)
    for c in range(2):
        assert _rel(Gb[c], Gf[c].astype(np.float64)) < BF16_TOL
        assert _rel(Fb[c], Ff[c].astype(np.float64)) < BF16_TOL
    hb.close()
    hf.close()


def test_tensor_core_window_runs_and_commits():
    """A full window with the BF16 tensor-core target: it commits at least one step and its statistics are finite."""
    from paper_2606_02455_b300 import lsd
    s, draft, tgt = _system(cells=8)
    integ = W.Integrator(0.5, 0.01, 350.0, 8)
    h = lsd.LSD(s, draft, tgt, integ)
    st = h.step(32)
    assert st["committed"] == 32 and np.isfinite(st["sum_delta"])
    h.close()


@pytest.mark.parametrize("cfg", [1, 2])
@pytest.mark.parametrize("precision", ["fp32", "fp32-tf32"])
def test_fp32_tensor_core_mlp_matches_oracle(cfg, precision):
    """FP32 targets run their MLP on the tensor cores as three products per term, split in FP16 with exact
    power-of-two scales (fp32) or in TF32 (fp32-tf32): descriptors, dE/dX and forces on perturbed configurations
    stay within the FP32 bar (1e-5 relative) of the FP64 oracle, and agree with the plain FP32 CUDA-core kernel to
    the same bar."""
    import torch
    from paper_2606_02455_b300 import lsd
    w = W.CONFIGS[cfg]()
    s = w.system
    integ = W.replace(w.integ, K=4)
    rng = np.random.default_rng(cfg)
    qs = np.stack([s.positions + 0.05 * rng.standard_normal(s.positions.shape) for _ in range(4)])
    h = lsd.LSD(s, w.draft, W.replace(w.target, precision=precision), integ)
    hc = lsd.LSD(s, w.draft, W.replace(w.target, precision="fp32-cuda-cores"), integ)
    F = h.target_forces(torch.tensor(qs, device="cuda")).cpu().numpy()
    Fc = hc.target_forces(torch.tensor(qs, device="cuda")).cpu().numpy()
    X, G = h.descriptors(4)
    _, Gc = hc.descriptors(4)
    for c in range(4):
        ref = O.energy_forces(s, w.target, qs[c], want=("F", "X", "dEdX"))
        assert _rel(X[c], ref["X"]) < 1e-5
        assert _rel(G[c], ref["dEdX"]) < 1e-5, _rel(G[c], ref["dEdX"])
        assert _rel(F[c], ref["F"]) < 1e-5, _rel(F[c], ref["F"])
        assert _rel(G[c], Gc[c].astype(np.float64)) < 1e-5
        assert _rel(F[c], Fc[c].astype(np.float64)) < 1e-5
    h.close()
    hc.close()


# stated per-result bars of the FP8 path (3-bit mantissa through 4 + 4 GEMMs; measured on this system:
# dE/dX 8.8 %, forces 0.41 %, per-atom MLP energy 11.1 %)
FP8_TOL = {"dEdX": 0.15, "F": 0.02, "E": 0.2}


def test_fp8_tensor_core_mlp_against_oracle():
    """FP8 e4m3 target MLP (static per-tensor scales calibrated at init, FP32 accumulation) on the config-4
    architecture: its stated per-result error against FP64, which the FP8 path has no tighter bar for."""
    import torch
    from paper_2606_02455_b300 import lsd
    s, draft, tgt = _system(precision="fp8")
    integ = W.Integrator(0.5, 0.01, 350.0, 4)
    h = lsd.LSD(s, draft, tgt, integ)
    rng = np.random.default_rng(7)
    qs = np.stack([s.positions + 0.05 * rng.standard_normal(s.positions.shape) for _ in range(4)])
    F, E = h.target_forces(torch.tensor(qs, device="cuda"), energies=True)
    F, E = F.cpu().numpy(), E.cpu().numpy()
    X, G = h.descriptors(4)
    errs = []
    for c in range(4):
        ref = O.energy_forces(s, tgt, qs[c], want=("F", "X", "dEdX", "E_atom"))
        e_lj = O.energy_forces(s, draft, qs[c], want=("E_atom",))["E_atom"]
        e = (_rel(G[c], ref["dEdX"]), _rel(F[c], ref["F"]), _rel(E[c].astype(np.float64) - e_lj, ref["E_atom"] - e_lj))
        errs.append(e)
        assert _rel(X[c], ref["X"]) < 1e-5
        assert e[0] < FP8_TOL["dEdX"] and e[1] < FP8_TOL["F"] and e[2] < FP8_TOL["E"], e
    print("fp8 relative errors (dEdX, F, E_mlp):", errs)
    h.close()


def test_fp8_potential_is_one_function():
    """The FP8 scales are calibrated once: the same configuration gives bit-identical forces before and after a
    window of dynamics, and in a second evaluation."""
    import torch
    from paper_2606_02455_b300 import lsd
    s, draft, tgt = _system(cells=6, precision="fp8")
    h = lsd.LSD(s, draft, tgt, W.Integrator(0.5, 0.01, 350.0, 4))
    q = torch.tensor(s.positions[None] + 0.02, device="cuda")
    F0 = h.target_forces(q).cpu().numpy()
    h.step(8)
    F1 = h.target_forces(q).cpu().numpy()
    assert np.array_equal(F0, F1)
    h.close()


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp32-tf32", 1e-5), ("bf16", BF16_TOL)])
def test_persistent_tiles_match_single_tile_launches(precision, tol):
    """The grid is one CTA per SM looping over 128-row tiles: 40 configurations of 512 atoms are 160 tiles on 148
    SMs, so some CTAs run a second tile with their barrier phases carried over.  Those configurations agree with the
    same ones evaluated two at a time (8 tiles, one per CTA), and the FP32 form with the CUDA-core kernel."""
    import torch
    from paper_2606_02455_b300 import lsd
    s, draft, tgt = _system(cells=8, precision=precision)
    n = 40
    integ = W.Integrator(0.5, 0.01, 350.0, n)   # a batch holds up to K configurations
    h = lsd.LSD(s, draft, tgt, integ)
    rng = np.random.default_rng(11)
    qs = np.stack([s.positions + 0.05 * rng.standard_normal(s.positions.shape) for _ in range(n)])
    big = h.target_forces(torch.tensor(qs, device="cuda")).cpu().numpy()
    for c0 in (0, n - 2):
        small = h.target_forces(torch.tensor(qs[c0:c0 + 2], device="cuda")).cpu().numpy()
        for c in range(2):
            assert _rel(small[c], big[c0 + c].astype(np.float64)) < tol
    if precision.startswith("fp32"):
        hc = lsd.LSD(s, draft, W.replace(tgt, precision="fp32-cuda-cores"), integ)
        ref = hc.target_forces(torch.tensor(qs, device="cuda")).cpu().numpy()
        for c in range(n):
            assert _rel(big[c], ref[c].astype(np.float64)) < tol
        hc.close()
    h.close()


@pytest.mark.parametrize("precision", ["fp32", "fp32-tf32"])
def test_fp32_split_ragged_rows_match_oracle(precision):
    """216 atoms x 3 configurations = 648 rows: five full 128-row tiles and a ragged one of 8 rows, through the
    FP16 and TF32 splits of a 67 -> 128 x 3 -> 1 FP32 target: forces within the FP32 bar of the FP64 oracle."""
    import torch
    from paper_2606_02455_b300 import lsd
    s, draft, tgt = _system(cells=6, precision=precision, width=128, layers=3)
    integ = W.Integrator(0.5, 0.01, 350.0, 4)
    h = lsd.LSD(s, draft, tgt, integ)
    rng = np.random.default_rng(17)
    qs = np.stack([s.positions + 0.05 * rng.standard_normal(s.positions.shape) for _ in range(3)])
    F = h.target_forces(torch.tensor(qs, device="cuda")).cpu().numpy()
    _, G = h.descriptors(3)
    for c in range(3):
        ref = O.energy_forces(s, tgt, qs[c], want=("F", "dEdX"))
        assert _rel(G[c], ref["dEdX"]) < 1e-5, _rel(G[c], ref["dEdX"])
        assert _rel(F[c], ref["F"]) < 1e-5, _rel(F[c], ref["F"])
    h.close()
