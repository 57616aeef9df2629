"""One density per E sample (the discretisation of Sec. "FDTD implementation and design export":
N~ = sum_k prod_l (N_l + 1 - delta_kl) design variables for an N_x x N_y x N_z design region),
pinned on the oracle without the GPU:
* the design samples of each component are exactly the E_k nodes lying in the closed design
  region, counted from their Yee coordinates;
* with the extra face samples set to the background material, the per-sample problem is the
  per-voxel problem, and by the chain rule the voxel gradient is the sum of its three samples';
* the per-sample gradient, extra face samples included, matches central finite differences.
"""
import numpy as np
import pytest

import oracle
import synth
from synth import EPS0, base_desc, vacuum


def _oracle(desc, m1, m2, gamma=0.0, rho=None):
    o = oracle.Oracle(desc)
    o.set_materials(vacuum(), m1, m2, gamma)
    if rho is not None:
        o.set_density(rho)
    return o


def _damped_metal(seed):
    m = synth.drude_lorentz_metal(seed, 2)
    poles = []
    for comp in range(3):
        (a1, c1), (a2, c2) = m["poles"][comp]
        poles.append([(complex(-8e14, 0.0), 0.5 * c1), (complex(-1e15, a2.imag), c2)])
    m["poles"] = poles
    m["sigma"] = [-2 * EPS0 * poles[0][0][1].real] * 3
    return m


def _desc(layout, steps=3000, src_comp=2, lambdas=(600.0,)):
    d = base_desc(20, 20, 20, dx=20e-9, n_steps=steps, cpml=5, precision=64, design=(8, 7, 6),
                  gap=(2, 2, 2), src_kind=0, src_comp=src_comp, src_pos=(10, 10, 10), lambdas_nm=lambdas)
    d["density_layout"] = layout
    return d


def _sample_shapes(db):
    N = (db[1] - db[0], db[3] - db[2], db[5] - db[4])
    return [tuple(N[a] + (a != c) for a in (2, 1, 0)) for c in range(3)]   # (z, y, x)


def _sample_index(db, comp, i, j, k):
    """Position of design sample E_comp of voxel (i, j, k) in the concatenated density vector."""
    sh = _sample_shapes(db)
    off = sum(int(np.prod(s)) for s in sh[:comp])
    nz, ny, nx = sh[comp]
    return off + ((k - db[4]) * ny + (j - db[2])) * nx + (i - db[0])


def test_sample_sets_are_the_nodes_in_the_closed_region():
    d = _desc(1, steps=4)
    db, gb = d["design_box"], d["gap_box"]
    o = _oracle(d, vacuum(), synth.drude_lorentz_metal(1, 1))
    N = (db[1] - db[0], db[3] - db[2], db[5] - db[4])
    n_tilde = sum(np.prod([N[l] + 1 - (k == l) for l in range(3)]) for k in range(3))
    assert o.vshape == (n_tilde,)
    cls = o.get_index_map(0) & 3
    nz, ny, nx = o.n
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ijk = (I, J, K)
    gap = (I >= gb[0]) & (I < gb[1]) & (J >= gb[2]) & (J < gb[3]) & (K >= gb[4]) & (K < gb[5])
    for comp in range(3):
        # E_comp node: half-integer along comp, integer along the other axes
        inside = np.ones(o.n, bool)
        for a in range(3):
            x = ijk[a] + (0.5 if a == comp else 0.0)
            inside &= (x >= db[2 * a]) & (x <= db[2 * a + 1])
        assert inside.sum() == np.prod([N[l] + 1 - (comp == l) for l in range(3)])
        assert np.array_equal(cls[comp] == 1, inside & ~gap)
        assert np.array_equal(cls[comp] == 2, gap)
    wm = o.get_index_map(2)
    assert (wm >= 0).sum() == (N[0] + 1) * (N[1] + 1) * (N[2] + 1)


def test_reduces_to_per_voxel_layout():
    m2 = _damped_metal(7)
    d0, d1 = _desc(0, steps=1500), _desc(1, steps=1500)
    db = d0["design_box"]
    rho_v = synth.uniform_rho(synth.box_shape(db), 11, 0.2, 0.8)
    o0 = _oracle(d0, vacuum(), m2, rho=rho_v)
    o1 = _oracle(d1, vacuum(), m2)
    rho_s = np.zeros(o1.vshape)          # face samples outside the design box: rho = 0, vacuum = background
    for comp in range(3):
        for k in range(db[4], db[5]):
            for j in range(db[2], db[3]):
                for i in range(db[0], db[1]):
                    rho_s[_sample_index(db, comp, i, j, k)] = rho_v[k - db[4], j - db[2], i - db[0]]
    o1.set_density(rho_s)
    F0, g0 = o0.forward()
    F1, g1 = o1.forward()
    assert F1 == pytest.approx(F0, rel=1e-12)
    assert np.allclose(g1, g0, rtol=0, atol=1e-12 * np.abs(g0).max())
    o0.adjoint()
    o1.adjoint()
    G0, G1 = o0.gradient(), o1.gradient()
    Gsum = np.zeros_like(G0)
    for comp in range(3):
        for k in range(db[4], db[5]):
            for j in range(db[2], db[3]):
                for i in range(db[0], db[1]):
                    Gsum[k - db[4], j - db[2], i - db[0]] += G1[_sample_index(db, comp, i, j, k)]
    assert np.linalg.norm(Gsum - G0) <= 1e-10 * np.linalg.norm(G0)
    # the DFTs over the design box agree; the working box adds the +x/+y/+z face layer
    D0, D1 = o0.get_dft(False), o1.get_dft(False)
    assert D1.shape[2:] == tuple(s + 1 for s in D0.shape[2:])
    assert np.allclose(D1[:, :, :-1, :-1, :-1], D0, rtol=0, atol=1e-12 * np.abs(D0).max())


def test_per_sample_gradient_vs_finite_differences():
    d = _desc(1, steps=3000, src_comp=0, lambdas=(550.0, 650.0))
    db = d["design_box"]
    m1 = synth.lorentz_dielectric(5, 1, (1.5, 1.5, 2.0))
    o = _oracle(d, m1, _damped_metal(9), gamma=3e6)
    rho = synth.uniform_rho(o.vshape, 13, 0.2, 0.8)
    o.set_density(rho)
    o.forward()
    o.adjoint()
    g = o.gradient()
    scale = np.abs(g).max()
    picks = [(0, db[0] + 3, db[2] + 2, db[4] + 1),     # interior samples of each component
             (1, db[0] + 5, db[2] + 1, db[4] + 4),
             (2, db[0] + 1, db[2] + 5, db[4] + 2),
             (0, db[0] + 2, db[3], db[4] + 3),         # E_x on the +y face (outside the voxel box)
             (2, db[1], db[2] + 3, db[4] + 1)]         # E_z on the +x face
    h = 1e-4
    for comp, i, j, k in picks:
        q = _sample_index(db, comp, i, j, k)
        r = rho.copy()
        r[q] += h
        o.set_density(r)
        Fp, _ = o.forward()
        r[q] -= 2 * h
        o.set_density(r)
        Fm, _ = o.forward()
        fd = (Fp - Fm) / (2 * h)
        assert abs(g[q] - fd) <= 5e-5 * max(abs(fd), 1e-3 * scale), (comp, i, j, k, g[q], fd)
    # gap samples carry no gradient
    gb = d["gap_box"]
    assert g[_sample_index(db, 1, gb[0], gb[2], gb[4])] == 0.0


def test_paper_mode_refuses_per_sample_layout():
    d = _desc(1, steps=20)
    o = _oracle(d, vacuum(), _damped_metal(7), rho=np.full(_oracle(d, vacuum(), vacuum()).vshape, 0.5))
    with pytest.raises(oracle.OracleError):
        o.paper_objective()
