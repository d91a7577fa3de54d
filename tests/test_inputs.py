"""Seeded input generators: sizes, closedness and orientation."""
import numpy as np
import pytest

from paper_1212_3032_gb300 import inputs


def _edges_closed(tri):
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    fwd = {tuple(x) for x in e}
    # every directed edge must appear exactly once and its reverse once
    return len(fwd) == e.shape[0] and all((b, a) in fwd for a, b in fwd)


def _signed_volume(xyz, tri):
    p0, p1, p2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    return np.einsum("ij,ij->i", p0, np.cross(p1, p2)).sum() / 6.0


@pytest.mark.parametrize("n,count", [(1, 20), (4, 320), (16, 5120)])
def test_geodesic_sphere_counts(n, count):
    xyz, tri = inputs.geodesic_sphere(n)
    assert tri.shape == (count, 3)
    assert _edges_closed(tri)
    assert np.allclose(np.linalg.norm(xyz, axis=1), 1.0)
    assert _signed_volume(xyz, tri) > 0          # outward normals
    _, tri_in = inputs.geodesic_sphere(n, inward=True)
    assert _signed_volume(xyz, tri_in) < 0


def test_box_mesh():
    xyz, tri = inputs.box_mesh(1.0, 2.0, 3.0, h=0.5)
    assert _edges_closed(tri)
    assert _signed_volume(xyz, tri) == pytest.approx(6.0)


def test_cavity_problem_orientation():
    m = inputs.cavity_problem(4)
    assert m.ne == 320
    c = (m.xyz[m.tri[:, 0]] + m.xyz[m.tri[:, 1]] + m.xyz[m.tri[:, 2]]) / 3
    # traction -p n with n into the cavity: pushes the wall outward (along +c)
    assert np.all(np.einsum("ij,ij->i", m.pattern, c) > 0)
    assert np.all(m.bc_type == inputs.BC_TRACTION)


def test_heaviside_history():
    p = inputs.heaviside_history(8, 2.0)
    assert p[0] == 1.0 and np.all(p[1:] == 2.0)


def test_small_cube_with_cavities():
    m = inputs.cube_with_cavities(n_face=8, n_cav=2, cav_radius=0.1, cav_n=3, seed=1)
    assert m.ne == 6 * 2 * 64 + 2 * 20 * 9
    assert _edges_closed(m.tri)
    assert np.sum(m.bc_type == inputs.BC_DISPLACEMENT) == 128
    assert np.sum(m.pattern[:, 2] != 0) == 128


def test_batched_meshes_uneven():
    ms = inputs.batched_meshes(count=4, seed=3032, tri_min=200, tri_max=2000)
    sizes = [m.ne for m in ms]
    assert len(set(sizes)) == 4
    assert all(150 <= n <= 2600 for n in sizes)


def test_ball_with_void():
    m = inputs.ball_with_void(n_outer=6, n_inner=3)
    n_out = 20 * 36
    assert m.ne == n_out + 20 * 9
    assert _edges_closed(m.tri)
    p = m.xyz[m.tri]
    c = p.mean(axis=1)
    nrm = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    # outer normals away from the centre, void normals into the void
    assert np.all(np.einsum("ij,ij->i", nrm[:n_out], c[:n_out]) > 0)
    vc = np.array([0.35, 0.2, -0.1])
    assert np.all(np.einsum("ij,ij->i", nrm[n_out:], c[n_out:] - vc) < 0)
    # pressure on the outer surface only: t = -p n points inward there
    assert np.all(np.einsum("ij,ij->i", m.pattern[:n_out], c[:n_out]) < 0)
    assert np.all(m.pattern[n_out:] == 0) and np.all(m.bc_type == inputs.BC_TRACTION)
    # enclosed volume (divergence theorem) = ball minus void
    vol = np.sum(np.einsum("ij,ij->i", p[:, 0], np.cross(p[:, 1], p[:, 2]))) / 6
    assert abs(vol - 4 / 3 * np.pi * (1 - 0.3 ** 3)) < 0.1
    assert inputs.ball_with_void().ne == 20180


def test_rod_problem():
    m = inputs.rod_problem(h=0.25)
    assert m.ne == 2 * 32 + 4 * 96
    assert _edges_closed(m.tri)
    c = m.xyz[m.tri].mean(axis=1)
    fixed = np.abs(c[:, 0]) < 1e-9
    loaded = np.abs(c[:, 0] - 3.0) < 1e-9
    assert fixed.sum() == 32 and loaded.sum() == 32
    assert np.all(m.bc_type[fixed] == inputs.BC_DISPLACEMENT) and np.all(m.bc_type[~fixed] == inputs.BC_TRACTION)
    assert np.allclose(m.pattern[loaded], [-1.0, 0.0, 0.0])  # compressive traction on the end x = 3
    assert np.all(m.pattern[~loaded] == 0)
    assert inputs.rod_problem().ne == 12348
