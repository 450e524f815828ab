"""The seeded input recipes produce what the workload descriptions state:
jitter bounds and planar boundaries, the strain of the sine states, the
distribution of the directions, the free-DoF count of the small cube, the
compressed state's volume ratio and symmetry, the uniaxial start, the tube's
radii and frames, and the size/degree draw of the 64-cube batch."""
import math

import numpy as np
import pytest

from paper_2408_12479_gb300 import inputs as I


def test_jitter_is_bounded_interior_only_and_uniform():
    n, jit = 8, 0.1
    V0 = I.box_vertices(n, n, n)
    V = I.box_vertices(n, n, n, jitter=jit, seed=4)
    d = V - V0
    h = 1.0 / n
    assert np.abs(d).max() <= jit * h
    on_face = ((np.isclose(V0, 0.0) | np.isclose(V0, 1.0)).any(axis=1))
    assert (d[on_face] == 0.0).all()  # the boundary stays planar
    interior = d[~on_face]
    assert interior.shape[0] == (n - 1) ** 3
    # U[-0.1h, 0.1h]: mean |d| = 0.05h, both signs equally often
    assert abs(np.abs(interior).mean() / (0.5 * jit * h) - 1.0) < 0.05
    assert abs((interior < 0).mean() - 0.5) < 0.05


def _max_gradient(f, m=24):
    """Largest |du_c/dX_d| of the field on an m^3 grid, by central differences."""
    t = (np.arange(m) + 0.5) / m
    Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    h = 1e-6
    g = 0.0
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        g = max(g, np.abs((f(P + e) - f(P - e)) / (2 * h)).max())
    return g


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sine_state_strain(seed):
    f = I.sine_field(seed, strain=0.05)
    assert f.grad_bound() == pytest.approx(0.05)
    k = f.k.reshape(-1, 3)
    assert ((k >= 0) & (k <= 2)).all() and k.any(axis=1).all()
    assert ((f.phi >= 0) & (f.phi < 2 * math.pi)).all()
    g = _max_gradient(f)
    # the bound holds, and it is not loose by more than the three terms' phase mismatch
    assert 0.01 < g <= 0.05 * (1 + 1e-6)


def test_directions_are_uniform_on_unit_interval():
    v = I.random_direction(200000, 7)
    assert v.min() >= -1.0 and v.max() <= 1.0
    assert abs(v.mean()) < 0.01 and abs(v.var() - 1.0 / 3.0) < 0.01
    assert np.array_equal(v, I.random_direction(200000, 7))  # seeded


def test_small_cube_free_dofs():
    m, f, seed = I.workload_small_cube()
    assert (m.box, m.p, m.n_dofs) == ((4, 4, 4), 2, 2187)
    assert m.n_dofs - int(m.dirichlet.sum()) == 1944  # "about 1.9k" with x = 0 clamped
    assert f.amp == 0.01


def test_compressed_cube_volume_ratio_and_symmetry():
    m, f, seed = I.workload_compressed_cube(n=4, p=2, J_target=0.9)
    assert (1.0 + f.s) ** 3 == pytest.approx(0.9, rel=1e-14)
    rng = np.random.Generator(np.random.PCG64(1))
    X = rng.uniform(0.0, 1.0, size=(500, 3))
    for c in range(3):
        Xc = X.copy()
        Xc[:, c] = 0.0
        assert np.abs(f(Xc)[:, c]).max() == 0.0  # compatible with the clamp of component c on X_c = 0
    mask = m.dirichlet.reshape(-1, 3).astype(bool)
    Nx = 4 * 2 + 1
    idx = np.arange(Nx ** 3)
    for c, L in enumerate((idx % Nx, (idx // Nx) % Nx, idx // Nx ** 2)):
        assert np.array_equal(mask[:, c], L == 0)


def test_uniaxial_start_carries_the_prescribed_values():
    m, u0 = I.workload_uniaxial(3, 2, 1.2)
    Nx = 7
    u = u0.reshape(-1, 3)
    mask = m.dirichlet.reshape(-1, 3).astype(bool)
    idx = np.arange(Nx ** 3)
    I_, J_, K_ = idx % Nx, (idx // Nx) % Nx, idx // Nx ** 2
    assert np.allclose(u[I_ == 0, 0], 0.0) and np.allclose(u[I_ == Nx - 1, 0], 0.2)
    # u_x on x = 0 and x = L; u_y on y = 0; u_z on z = 0; nothing else
    assert np.array_equal(mask[:, 0], (I_ == 0) | (I_ == Nx - 1))
    assert np.array_equal(mask[:, 1], J_ == 0) and np.array_equal(mask[:, 2], K_ == 0)
    assert (u[:, 1:] == 0.0).all()


def test_tube_geometry_and_frames():
    m = I.tube_mesh(3)
    x, y, z = m.geo_nodes.T
    r = np.hypot(x, y)
    assert r.min() == pytest.approx(1.0) and r.max() == pytest.approx(1.3)
    assert z.min() == 0.0 and z.max() == pytest.approx(10.0)
    assert m.n_elem == 16 * 8 * 64 and m.n_dofs == 3 * 48 * 25 * 193
    F = m.frames.reshape(-1, 3, 3)
    assert np.allclose(F @ F.transpose(0, 2, 1), np.eye(3))  # orthonormal frames
    assert np.allclose(np.linalg.det(F), 1.0)                # right-handed
    # E3 radial and E1 circumferential at each element's mid-angle
    c = m.geo_nodes[m.geo_conn].mean(axis=1)
    th = np.arctan2(c[:, 1], c[:, 0])
    assert np.allclose(F[:, 2, :2], np.stack([np.cos(th), np.sin(th)], axis=1), atol=1e-12)


def test_batch_draw(monkeypatch):
    drawn = []

    def stub(n, p, jitter=0.0, seed=0, lengths=(1.0, 1.0, 1.0), clamp=False, name=""):
        drawn.append((n, p, jitter))
        return (n, p)

    monkeypatch.setattr(I, "box_mesh", stub)
    batch = I.workload_batch()
    assert len(batch) == 64 and len(set(s for _, _, s in batch)) == 64
    ns = np.array([d[0] for d in drawn])
    ps = np.array([d[1] for d in drawn])
    assert ns.min() >= 8 and ns.max() <= 24 and set(ps) <= {2, 3, 4, 5}
    assert all(d[2] == 0.1 for d in drawn)
    assert len(set(ps)) == 4 and ns.max() - ns.min() >= 12  # the draw spans the ranges
    total = int((3 * (ns * ps + 1) ** 3).sum())
    assert abs(total - 66.8e6) < 0.05e6
