"""Oracle pins for the synthetic potentials: forces are minus the energy gradient (finite differences),
closed forms for two- and three-atom geometries, periodic lattice sums, and extensivity under replication."""
import numpy as np
import pytest

import oracle.oracle as O
from paper_2606_02455_b300 import workloads as W


def _fd_forces(system, pot, q, h=1e-4):
    F = np.zeros_like(q)
    for i in range(q.shape[0]):
        for a in range(3):
            qp = q.copy(); qp[i, a] += h
            qm = q.copy(); qm[i, a] -= h
            F[i, a] = -(O.energy(system, pot, qp) - O.energy(system, pot, qm)) / (2 * h)
    return F


def _pot(system, n_rbf=16, n_ang=0, n_layers=2, width=16, head="tanh", rc=5.0, lj=True, seed=1, scale=1.0):
    ns = system.n_species
    d0 = W.input_dim(ns, n_rbf, n_ang)
    w = W.mlp_weights(d0, n_layers, width, seed) * scale if n_layers else None
    kw = dict(lj_eps=np.array([0.0104, 0.0067, 0.005][:ns]), lj_sigma=np.array([3.0, 2.8, 2.0][:ns]),
              lj_cutoff=4.9) if lj else {}
    return W.Potential(**kw, n_rbf=n_rbf, n_ang=n_ang, n_layers=n_layers, width=width, desc_cutoff=rc, head=head,
                       head_scale=0.05 if head == "tanh" else 1.0, weights=w)


CASES = [
    dict(n_rbf=16, n_ang=0, n_layers=2, head="tanh"),
    dict(n_rbf=8, n_ang=16, n_layers=1, head="linear"),
    dict(n_rbf=6, n_ang=16, n_layers=3, head="tanh", scale=3.0),
    dict(n_rbf=0, n_ang=0, n_layers=0, head="tanh"),   # pure LJ
]


@pytest.mark.parametrize("case", CASES)
def test_forces_are_minus_energy_gradient(case):
    """T1: analytic forces equal the central finite difference of the energy (h = 1e-4 A)."""
    s = W.small_system(n_cells=1, a=5.0, n_species=2, seed=3, L=10.0)
    pot = _pot(s, **case)
    q = s.positions + np.array([0.3, 0.1, -0.2])
    F = O.forces(s, pot, q)
    Ffd = _fd_forces(s, pot, q)
    err = np.linalg.norm(F - Ffd) / np.linalg.norm(Ffd)
    assert err < 1e-6, err


def test_forces_fd_with_multiple_images():
    """T1 with a cutoff larger than half the box (atoms see several images of the same neighbour)."""
    s = W.small_system(n_cells=1, a=5.0, n_species=1, seed=4, L=7.0)
    pot = W.Potential(lj_eps=np.array([0.0104]), lj_sigma=np.array([3.4]), lj_cutoff=6.5, n_rbf=8, n_ang=16,
                      n_layers=1, width=8, desc_cutoff=4.0, head="tanh", head_scale=0.05,
                      weights=W.mlp_weights(W.input_dim(1, 8, 16), 1, 8, 5))
    q = s.positions.copy()
    F = O.forces(s, pot, q)
    Ffd = _fd_forces(s, pot, q)
    assert np.linalg.norm(F - Ffd) / np.linalg.norm(Ffd) < 1e-6


def _lj(eps, sig, rc, r):
    return 4 * eps * ((sig / r) ** 12 - (sig / r) ** 6) - 4 * eps * ((sig / rc) ** 12 - (sig / rc) ** 6)


def test_two_atom_lj_closed_form():
    """Two atoms in a large box: E = U(r) - U(rc) and |F| = dU/dr along the bond."""
    r = 3.7
    s = W.System(positions=np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]]), momenta=np.zeros((2, 3)),
                 species=np.array([0, 1], dtype=np.int32), masses=np.array([12.0, 16.0]), box=np.array([30.0] * 3))
    pot = W.Potential(lj_eps=np.array([0.01, 0.004]), lj_sigma=np.array([3.0, 3.4]), lj_cutoff=8.0)
    eps, sig = np.sqrt(0.01 * 0.004), 0.5 * (3.0 + 3.4)
    res = O.energy_forces(s, pot, s.positions)
    assert res["E"] == pytest.approx(_lj(eps, sig, 8.0, r), rel=1e-13)
    dU = -24 * eps / r * (2 * (sig / r) ** 12 - (sig / r) ** 6)
    assert res["F"][0, 0] == pytest.approx(dU, rel=1e-12)      # atom 0 is pushed/pulled along +x by dU/dr
    assert res["F"][1, 0] == pytest.approx(-dU, rel=1e-12)
    assert np.allclose(res["F"][:, 1:], 0.0)


def test_bcc_lattice_sum_sees_every_image():
    """Two atoms at (0,0,0) and (L/2,L/2,L/2) of a periodic cubic box (a BCC cell), cutoff 0.98 L: each atom
    sees all 8 images of the other at distance L*sqrt(3)/2 (both images along every axis), none of its own
    (at distance L), so E = 8 U(L sqrt(3)/2) and F = 0."""
    L, rc = 6.0, 5.9
    s = W.System(positions=np.array([[0.2, 0.3, 0.4], [0.2 + L / 2, 0.3 + L / 2, 0.4 + L / 2]]),
                 momenta=np.zeros((2, 3)), species=np.array([0, 0], np.int32), masses=np.array([40.0]),
                 box=np.array([L] * 3))
    pot = W.Potential(lj_eps=np.array([0.0104]), lj_sigma=np.array([3.4]), lj_cutoff=rc)
    r = L * np.sqrt(3) / 2
    res = O.energy_forces(s, pot, s.positions)
    assert res["E"] == pytest.approx(8 * _lj(0.0104, 3.4, rc, r), rel=1e-12)
    assert np.allclose(res["F"], 0.0, atol=1e-14)
    nb = O.neighbors(s, s.positions, rc)
    assert len(nb[0]) == 8 and len(nb[1]) == 8
    # atom 1 sits at +L/2 of atom 0 on every axis: atom 0 sees atom 1 at shifts {0, -1} per axis, atom 1 sees
    # atom 0 at shifts {0, +1}; code = (sx+1) + 3(sy+1) + 9(sz+1)
    code = lambda sx, sy, sz: (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1)
    r01 = sorted(code(a, b, c) for a in (-1, 0) for b in (-1, 0) for c in (-1, 0))
    r10 = sorted(code(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1))
    assert sorted(int(k) & 31 for k in nb[0]) == r01 and all(int(k) >> 5 == 1 for k in nb[0])
    assert sorted(int(k) & 31 for k in nb[1]) == r10 and all(int(k) >> 5 == 0 for k in nb[1])


def test_simple_cubic_lattice_sees_eighteen_image_neighbours():
    """A simple cubic lattice of 2^3 atoms (spacing a) in a periodic box of side 2a, cutoff between sqrt(2) a and
    sqrt(3) a: every atom sees its 6 first and 12 second neighbours, which are images of only 6 distinct atoms (the
    two face neighbours along an axis are one atom at two shifts, each face-diagonal atom appears at four shifts).  The expected (atom, shift) set is the set
    of lattice points within the cutoff; E = 8/2 (6 U(a) + 12 U(sqrt2 a)); F = 0 by symmetry."""
    a, rc = 3.0, 4.6
    L = 2 * a
    g = np.array([[i, j, k] for i in range(2) for j in range(2) for k in range(2)], float)
    pos = g * a + 0.25
    s = W.System(positions=pos, momenta=np.zeros((8, 3)), species=np.zeros(8, np.int32), masses=np.array([40.0]),
                 box=np.array([L] * 3))
    pot = W.Potential(lj_eps=np.array([0.0104]), lj_sigma=np.array([3.4]), lj_cutoff=rc)
    nb = O.neighbors(s, pos, rc)
    code = lambda sh: (sh[0] + 1) + 3 * (sh[1] + 1) + 9 * (sh[2] + 1)
    for i in range(8):
        expect = sorted((j, code(sh)) for j in range(8) for sh in np.ndindex(3, 3, 3)
                        if 0 < np.linalg.norm(pos[j] + (np.array(sh) - 1) * L - pos[i]) < rc
                        for sh in [tuple(np.array(sh) - 1)])
        got = sorted((int(k) >> 5, int(k) & 31) for k in nb[i])
        assert len(got) == 18 and got == expect, i
        assert len({j for j, _ in got}) == 6
    res = O.energy_forces(s, pot, pos)
    assert res["E"] == pytest.approx(4 * (6 * _lj(0.0104, 3.4, rc, a) + 12 * _lj(0.0104, 3.4, rc, np.sqrt(2) * a)),
                                     rel=1e-12)
    assert np.allclose(res["F"], 0.0, atol=1e-13)


def test_radial_descriptor_two_atoms():
    """Two atoms of different species at distance r: atom 0's radial block for species 1 is
    exp(-(r-mu_k)^2/(2w^2)) * (cos(pi r/rc)+1)/2 with mu_k = k rc/(n-1), w = rc/(n-1); its species-0 block is 0."""
    r, rc, n = 2.3, 5.0, 8
    s = W.System(positions=np.array([[4.0, 4.0, 4.0], [4.0, 4.0 + r, 4.0]]), momenta=np.zeros((2, 3)),
                 species=np.array([0, 1], dtype=np.int32), masses=np.array([12.0, 16.0]), box=np.array([20.0] * 3))
    pot = W.Potential(n_rbf=n, n_ang=0, n_layers=1, width=4, desc_cutoff=rc, head="linear",
                      weights=W.mlp_weights(W.input_dim(2, n, 0), 1, 4, 0))
    X = O.energy_forces(s, pot, s.positions, want=("X",))["X"]
    w = rc / (n - 1)
    mu = np.arange(n) * w
    g = np.exp(-(r - mu) ** 2 / (2 * w * w)) * 0.5 * (np.cos(np.pi * r / rc) + 1)
    assert np.allclose(X[0, :n], 0.0)
    assert np.allclose(X[0, n:2 * n], g, rtol=1e-14, atol=0)
    assert np.array_equal(X[0, 2 * n:], [1.0, 0.0]) and np.array_equal(X[1, 2 * n:], [0.0, 1.0])


@pytest.mark.parametrize("cos_theta", [-1.0, 0.0, 1.0])
def test_angular_descriptor_special_angles(cos_theta):
    """Centre atom with two neighbours at r1, r2: the 16 terms 2^(1-zeta)(1+lambda c)^zeta e^{-eta(r1^2+r2^2)} fc fc
    reduce to 2*E for c=+-1 with matching lambda, 0 for the opposite lambda, and 2^(1-zeta)*E at c=0."""
    r1, r2, rc = 2.0, 2.5, 5.0
    u = np.array([1.0, 0.0, 0.0])
    v = np.array([cos_theta, np.sqrt(max(0.0, 1 - cos_theta ** 2)), 0.0])
    c0 = np.array([8.0, 8.0, 8.0])
    pos = np.array([c0, c0 + r1 * u, c0 + r2 * v])
    s = W.System(positions=pos, momenta=np.zeros((3, 3)), species=np.zeros(3, np.int32), masses=np.array([12.0]),
                 box=np.array([40.0] * 3))
    pot = W.Potential(n_rbf=2, n_ang=16, n_layers=1, width=4, desc_cutoff=rc, head="linear",
                      weights=W.mlp_weights(W.input_dim(1, 2, 16), 1, 4, 0))
    X = O.energy_forces(s, pot, pos, want=("X",))["X"]
    ang = X[0, 2:18]
    fc = lambda r: 0.5 * (np.cos(np.pi * r / rc) + 1)
    k = 0
    for zeta in (1, 2, 4, 8):
        for lam in (1, -1):
            for eta in (0.005, 0.05):
                E = np.exp(-eta * (r1 * r1 + r2 * r2)) * fc(r1) * fc(r2)
                if cos_theta == 0.0:
                    expect = 2.0 ** (1 - zeta) * E
                elif lam * cos_theta > 0:
                    expect = 2.0 * E
                else:
                    expect = 0.0
                assert ang[k] == pytest.approx(expect, rel=1e-12, abs=1e-15), (zeta, lam, eta)
                k += 1


def test_isolated_atom_mlp_head():
    """An atom with no neighbours has descriptor = one-hot of its species; its energy is
    0.05 tanh(MLP(onehot)), evaluated here with numpy matrix products of the same packed weights."""
    s = W.System(positions=np.array([[1.0, 1.0, 1.0], [10.0, 10.0, 10.0]]), momenta=np.zeros((2, 3)),
                 species=np.array([1, 0], np.int32), masses=np.array([12.0, 16.0]), box=np.array([20.0] * 3))
    d0 = W.input_dim(2, 4, 16)
    w = W.mlp_weights(d0, 2, 8, 9)
    w[8 * d0:8 * d0 + 8] = 0.3   # non-zero first bias
    pot = W.Potential(n_rbf=4, n_ang=16, n_layers=2, width=8, desc_cutoff=3.0, head="tanh", head_scale=0.05, weights=w)
    Ea = O.energy_forces(s, pot, s.positions, want=("E_atom",))["E_atom"]
    off = 0
    W1 = w[off:off + 8 * d0].reshape(8, d0); off += 8 * d0
    b1 = w[off:off + 8]; off += 8
    W2 = w[off:off + 64].reshape(8, 8); off += 64
    b2 = w[off:off + 8]; off += 8
    wo = w[off:off + 8]; bo = w[off + 8]
    silu = lambda z: z / (1 + np.exp(-z))
    for i, sp in enumerate([1, 0]):
        x = np.zeros(d0); x[d0 - 2 + sp] = 1.0
        y = wo @ silu(W2 @ silu(W1 @ x + b1) + b2) + bo
        assert Ea[i] == pytest.approx(0.05 * np.tanh(y), rel=1e-13)


def test_energy_is_extensive_under_replication():
    """A periodic system replicated 2x2x2 has 8x the energy and the same force on every copy of an atom
    (pins image handling of LJ, radial and angular terms together)."""
    s = W.small_system(n_cells=1, a=5.2, n_species=2, seed=8, L=5.2)
    pot = _pot(s, n_rbf=8, n_ang=16, n_layers=2, width=8, rc=2.5)
    pot.lj_cutoff = 4.5
    r1 = O.energy_forces(s, pot, s.positions)
    L = s.box[0]
    shifts = np.stack(np.meshgrid(*[np.arange(2)] * 3, indexing="ij"), -1).reshape(-1, 3) * L
    big_pos = np.concatenate([s.positions + sh for sh in shifts])
    big = W.System(positions=big_pos, momenta=np.zeros_like(big_pos), species=np.tile(s.species, 8),
                   masses=s.masses, box=s.box * 2)
    r8 = O.energy_forces(big, pot, big_pos)
    assert r8["E"] == pytest.approx(8 * r1["E"], rel=1e-11)
    assert np.allclose(r8["F"].reshape(8, -1, 3), r1["F"][None], rtol=1e-9, atol=1e-12)


def test_translation_invariance_and_unwrapped_positions():
    """Energy and forces do not change under a global translation or when atoms are shifted by whole boxes."""
    s = W.small_system(n_cells=1, a=5.0, n_species=2, seed=5, L=10.0)
    pot = _pot(s, n_rbf=8, n_ang=16, n_layers=1, width=8)
    r0 = O.energy_forces(s, pot, s.positions)
    q1 = s.positions + np.array([0.123, -7.5, 3.3])
    q1[0] += s.box * np.array([2, -1, 0])
    r1 = O.energy_forces(s, pot, q1)
    assert r1["E"] == pytest.approx(r0["E"], rel=1e-10)
    assert np.allclose(r1["F"], r0["F"], rtol=1e-8, atol=1e-12)


def test_neighbor_lists_symmetric_and_canonical():
    """Every member (i -> j, s) has its reverse (j -> i, -s); lists are sorted by (j, shift code)."""
    w = W.config2()
    lists = O.neighbors(w.system, w.system.positions, 5.0)
    pairs = set()
    for i, keys in enumerate(lists):
        assert np.all(np.diff(keys) > 0)
        for k in keys:
            pairs.add((i, int(k) >> 5, int(k) & 31))
    for (i, j, c) in pairs:
        assert (j, i, 26 - c) in pairs


@pytest.mark.parametrize("case", CASES[:3])
def test_forces_on_selected_atoms_equal_full_pass(case):
    """The atom-by-atom force routine used for large-system sampling equals the full evaluation."""
    s = W.small_system(n_cells=2, a=4.0, n_species=2, seed=6, L=8.0)
    pot = _pot(s, **case)
    q = s.positions + np.array([0.2, -0.1, 0.05])
    F = O.forces(s, pot, q)
    sel = [0, 3, 5, 7, 30]
    Fs = O.forces_subset(s, pot, q, sel)
    assert np.allclose(Fs, F[sel], rtol=1e-11, atol=1e-14)


def test_forces_on_selected_atoms_with_images():
    """Same with a cutoff larger than half the box (several images of one neighbour)."""
    s = W.small_system(n_cells=1, a=5.0, n_species=1, seed=4, L=7.0)
    pot = W.Potential(lj_eps=np.array([0.0104]), lj_sigma=np.array([3.4]), lj_cutoff=6.5, n_rbf=8, n_ang=16,
                      n_layers=1, width=8, desc_cutoff=4.0, head="tanh", head_scale=0.05,
                      weights=W.mlp_weights(W.input_dim(1, 8, 16), 1, 8, 5))
    F = O.forces(s, pot, s.positions)
    Fs = O.forces_subset(s, pot, s.positions, [0, 1, 2, 3])
    assert np.allclose(Fs, F, rtol=1e-11, atol=1e-14)


def test_centre_atom_ranges_partition_the_evaluation():
    """The centre-atom ranges of o_eval_range sum to the full energy and forces (every LJ pair and every e(x_i)
    term has exactly one centre atom), on several configurations at once and on several threads."""
    w = W.config2()
    s = w.system
    rng = np.random.default_rng(3)
    qs = np.stack([s.positions + 0.05 * rng.standard_normal(s.positions.shape) for _ in range(3)])
    cuts = [0, 37, 128, 200, 256]
    O.set_threads(3)
    try:
        parts = [O.eval_range(s, w.target, qs, a, b) for a, b in zip(cuts[:-1], cuts[1:])]
    finally:
        O.set_threads(1)
    for c in range(3):
        ref = O.energy_forces(s, w.target, qs[c], want=("F",))
        F = sum(p[0][c] for p in parts)
        E = sum(p[1][c] for p in parts)
        assert E == pytest.approx(ref["E"], rel=1e-12, abs=1e-12)
        assert np.allclose(F, ref["F"], rtol=1e-11, atol=1e-12)


def test_list_prefilter_changes_no_list():
    """The oracle's minimum-image pre-test only skips pairs the membership rule rejects: lists with and without
    it are identical, on the benchmark systems, on a box whose cutoff is 0.97 of its side (every image along every
    axis in play) and on pairs placed within 1e-6 of the cutoff."""
    rng = np.random.default_rng(8)
    cases = []
    w = W.config2()
    cases.append((w.system, w.system.positions + 0.1 * rng.standard_normal(w.system.positions.shape), 5.0))
    w = W.config1()
    cases.append((w.system, w.system.positions, 8.5))
    small = W.small_system(1, 5.0, 2)
    cases.append((small, small.positions, 0.97 * 5.0))
    rc = 4.0
    pos = np.array([[1.0, 1.0, 1.0], [1.0 + rc * (1 - 1e-6), 1.0, 1.0], [1.0, 1.0 + rc * (1 + 1e-6), 1.0],
                    [1.0, 1.0, 1.0 + rc]])
    tiny = W.System(positions=pos, momenta=np.zeros((4, 3)), species=np.zeros(4, np.int32), masses=np.array([1.0]),
                    box=np.array([12.0, 12.0, 12.0]))
    cases.append((tiny, pos, rc))
    for sysm, q, cut in cases:
        O.set_list_prefilter(True)
        a = O.neighbors(sysm, q, cut)
        O.set_list_prefilter(False)
        try:
            b = O.neighbors(sysm, q, cut)
        finally:
            O.set_list_prefilter(True)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
