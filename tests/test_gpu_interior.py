"""Interior displacement and strain (representation formula) on the GPU
against the oracle, through the C-ABI.

The rod (3 x 1 x 1, fixed end, step traction on the other end, nu = 0) is
swept on the GPU; the interior field at points inside it, near a face (the
subdivided 1,024-point band) and in the middle (regular bands), is compared
with ``oracle.bem.interior_field`` evaluated on the GPU's own boundary
solution (the kernel alone: FP32 kernel evaluation 2e-5, FP64 1e-8), and
with the oracle's whole chain (its own boundary solve: the sweep target 1e-4).
Strain: central differences with step h = 0.02 (FP32 rounding of the
displacement amplified by 1 / (2h)). Time histories: the IDFT of the oracle's
field spectra.
"""
import numpy as np
import pytest

from oracle import bem, kernels, sweep as osweep, transforms
from paper_1212_3032_gb300 import inputs

pytestmark = pytest.mark.gpu

MAT = kernels.Material(1.0, 0.0, 1.0)
PTS = np.array([[0.5, 0.05, -0.1], [1.5, 0.0, 0.0], [2.5, -0.2, 0.1],
                [1.2, 0.45, 0.1],          # 0.05 from the face y = 1/2: NEAR band
                [2.9, -0.3, 0.42]])        # near the loaded end and a side face
H_STRAIN = 0.02


@pytest.fixture(scope="module")
def B():
    from paper_1212_3032_gb300 import binding, build
    build.build()
    return binding


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def rod():
    return inputs.rod_problem(h=1 / 4)                  # 448 triangles


@pytest.mark.parametrize("prec,ktol,stol,ttol", [(0, 2e-5, 5e-4, 1e-4), (1, 1e-8, 1e-6, 1e-7)])
def test_interior_field_matches_oracle(B, rod, prec, ktol, stol, ttol):
    T, N = 6.0, 16
    eta = 5.0 / T
    load = inputs.heaviside_history(N)
    g = bem.geometry(rod.xyz, rod.tri)
    with B.Context(0) as ctx:
        ctx.set_material(MAT.E, MAT.nu, MAT.rho)
        ctx.set_window(eta, B.WIN_HANNING)
        o = B.default_opts(dense=0, leaf_size=16, precision=prec, tol=1e-9 if prec else 1e-7,
                           aca_tol=1e-9 if prec else 1e-6)
        ctx.mesh(rod.xyz, rod.tri, rod.bc_type, o)
        ctx.solve_sweep(T, N, load, rod.pattern, o)
        s_all = transforms.sampling_frequencies(T, N, eta)
        Pk = transforms.dft_mft(load, T, eta)
        spec = []
        for k in (1, 5, 8):
            a = ctx.get_frequency_solution(k)
            known = rod.pattern * Pk[k]
            ref = bem.interior_field(g, rod.bc_type, known, a, PTS, s_all[k], MAT)
            got = ctx.interior_field(k, PTS)
            for p in range(len(PTS)):
                assert _rel(got[p], ref[p]) <= ktol, (k, p)
            eps = ctx.interior_strain(k, PTS, H_STRAIN)
            eps_ref = bem.interior_strain(g, rod.bc_type, known, a, PTS, s_all[k], MAT, H_STRAIN)
            assert _rel(eps, eps_ref) <= stol, k
        # the time histories: every frequency's field, then the windowed IDFT
        for k in range(N // 2 + 1):
            a = ctx.get_frequency_solution(k)
            spec.append(bem.interior_field(g, rod.bc_type, rod.pattern * Pk[k], a, PTS, s_all[k], MAT).ravel())
        tr = ctx.interior_time_response(PTS, B.FIELD_DISPLACEMENT)
        tr_ref = transforms.idft_mft(np.array(spec), T, eta, B.WIN_HANNING, N).reshape(N, len(PTS), 3)
        assert _rel(tr, tr_ref) <= ttol
        # strain histories: the IDFT of the strain spectra
        st = ctx.interior_time_response(PTS[:2], B.FIELD_STRAIN, H_STRAIN)
        sspec = np.array([ctx.interior_strain(k, PTS[:2], H_STRAIN).ravel() for k in range(N // 2 + 1)])
        st_ref = transforms.idft_mft(sspec, T, eta, B.WIN_HANNING, N).reshape(N, 2, 6)
        assert _rel(st, st_ref) <= 1e-10


def test_interior_field_end_to_end(B, rod):
    """GPU sweep + GPU interior field against the oracle's direct solves and
    its interior field (mixed precision, the sweep's 1e-4 target)."""
    T, N = 6.0, 8
    eta = 5.0 / T
    load = inputs.heaviside_history(N)
    ref = osweep.solve_sweep(rod, MAT, T, N, eta, load)
    g = bem.geometry(rod.xyz, rod.tri)
    with B.Context(0) as ctx:
        ctx.set_material(MAT.E, MAT.nu, MAT.rho)
        ctx.set_window(eta, B.WIN_HANNING)
        o = B.default_opts(dense=1, precision=0, tol=1e-7)
        ctx.mesh(rod.xyz, rod.tri, rod.bc_type, o)
        ctx.solve_sweep(T, N, load, rod.pattern, o)
        for k in (2, 4):
            f_ref = bem.interior_field(g, rod.bc_type, rod.pattern * ref["Pk"][k], ref["a"][k], PTS, ref["s"][k], MAT)
            assert _rel(ctx.interior_field(k, PTS), f_ref) <= 1e-4, k


def test_interior_edge_cases(B, rod):
    with B.Context(0) as ctx:
        ctx.set_material(MAT.E, MAT.nu, MAT.rho)
        o = B.default_opts(dense=1)
        ctx.mesh(rod.xyz, rod.tri, rod.bc_type, o)
        with pytest.raises(B.BemError) as e:                 # no sweep solved yet
            ctx.interior_field(0, PTS)
        assert e.value.code == -7
        ctx.set_window(0.5, B.WIN_NONE)
        ctx.solve_sweep(4.0, 2, inputs.heaviside_history(2), rod.pattern, o)
        assert ctx.interior_field(1, np.zeros((0, 3))).shape == (0, 3)
        with pytest.raises(B.BemError):
            ctx.interior_field(2, PTS)                        # frequency index not solved
        with pytest.raises(B.BemError):
            ctx.interior_strain(1, PTS, 0.0)                 # difference step must be positive
