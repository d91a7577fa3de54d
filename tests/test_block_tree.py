"""The block partition of the operator (host logic, no GPU): the cluster tree
and the near / admissible-far block lists that bem_mesh builds, through the
host-only entry point bem_block_tree.

* The blocks cover every (row element, column element) pair exactly once.
* Every far block satisfies the admissibility rule recomputed here from the
  centroids: min(diam) <= eta dist and dist^2 > 2.2 h_max^2, so no pair in it
  falls in the near-singular quadrature band.
* Near blocks are leaf pairs of at most leaf_size elements, and each leaf's
  diagonal block is among them; dense mode has no far blocks.
"""
import numpy as np
import pytest

from paper_1212_3032_gb300 import inputs


@pytest.fixture(scope="module")
def B():
    from paper_1212_3032_gb300 import binding, build
    build.build()
    return binding


def _geom(mesh):
    p = mesh.xyz[mesh.tri]
    c = p.mean(axis=1)
    e = np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 1], p[:, 0] - p[:, 2]], axis=1)
    return c, np.sqrt((e ** 2).sum(-1)).max(axis=1)


MESHES = {
    "sphere980": lambda: inputs.cavity_problem(7),
    "cube": lambda: inputs.cube_with_cavities(n_face=8, n_cav=2, cav_radius=0.12, cav_n=3, seed=5),
    "box": lambda: inputs.pressurised_surface(*inputs.box_mesh(1.0, 2.5, 1.5, 0.2)),
}


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("leaf", [16, 64])
def test_partition_and_admissibility(B, name, leaf):
    mesh = MESHES[name]()
    c, h = _geom(mesh)
    eta = 1.0
    perm, near, far = B.block_tree(c, h, leaf_size=leaf, eta_adm=eta)
    ne = mesh.ne
    assert np.array_equal(np.sort(perm), np.arange(ne))
    cover = np.zeros((ne, ne), dtype=np.int32)
    for r0, nr, c0, nc in np.concatenate([near, far]):
        cover[r0:r0 + nr, c0:c0 + nc] += 1
    assert np.all(cover == 1)
    ct, ht = c[perm], h[perm]  # tree order

    def box(b, n):
        return ct[b:b + n].min(axis=0), ct[b:b + n].max(axis=0)

    for r0, nr, c0, nc in far:
        (amin, amax), (bmin, bmax) = box(r0, nr), box(c0, nc)
        gap = np.maximum(0.0, np.maximum(amin - bmax, bmin - amax))
        d2 = float(gap @ gap)
        diam = min(np.linalg.norm(amax - amin), np.linalg.norm(bmax - bmin))
        hm = max(ht[r0:r0 + nr].max(), ht[c0:c0 + nc].max())
        assert d2 > 0 and diam <= eta * np.sqrt(d2) + 1e-12 and d2 > 2.2 * hm * hm
        # hence every element pair of the block is outside the near-singular band
        dd = ((ct[r0:r0 + nr, None, :] - ct[None, c0:c0 + nc, :]) ** 2).sum(-1)
        assert np.all(dd > 2.2 * ht[None, c0:c0 + nc] ** 2)
    assert np.all(near[:, 1] <= leaf) and np.all(near[:, 3] <= leaf)
    diag = near[(near[:, 0] == near[:, 2]) & (near[:, 1] == near[:, 3])]
    assert diag[:, 1].sum() == ne  # the leaves' diagonal blocks tile the diagonal


def test_dense_mode_has_no_far_blocks(B):
    mesh = inputs.cavity_problem(4)
    c, h = _geom(mesh)
    _, near, far = B.block_tree(c, h, leaf_size=32, dense=True)
    assert far.shape[0] == 0 and (near[:, 1] * near[:, 3]).sum() == mesh.ne ** 2


def test_invalid_arguments(B):
    with pytest.raises(B.BemError):
        B.block_tree(np.zeros((3, 3)), np.ones(3), leaf_size=0)
