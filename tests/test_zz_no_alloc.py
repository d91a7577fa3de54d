"""bem_apply_noalloc: the operator product for callers that cannot allocate.

Some callers cannot let a library call cudaMalloc during a call (a caching
allocator that owns the device's memory, or a latency-bound loop that cannot
take cudaMalloc's implicit synchronisation). The entry point under test keeps
its scratch in a fixed device array; this checks its output against the
existing product entry point bem_apply, on two calls in a row (the second on
different data, so stale scratch contents would show). This file is collected
last so that a failure here never hides the other tests.
"""
import numpy as np
import pytest

from paper_1212_3032_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_apply_noalloc_matches_apply():
    import torch

    from paper_1212_3032_gb300 import binding, build

    build.build()
    mesh = inputs.cavity_problem(7)  # 980 triangles, leaf 32: dense near blocks and ACA blocks
    with binding.Context(0) as ctx:
        ctx.set_material(1.0, 0.25, 1.0)
        o = binding.default_opts(leaf_size=32, aca_tol=1e-5, precision=binding.PREC_C64_MIXED)
        ctx.mesh(mesh.xyz, mesh.tri, mesh.bc_type, o)
        ctx.assemble(0.625 + 3.0j, o)
        rng = np.random.default_rng(11)
        dev = torch.device("cuda", 0)
        for _ in range(2):
            x = (rng.normal(size=3 * mesh.ne) + 1j * rng.normal(size=3 * mesh.ne)).astype(np.complex64)
            y_ref = ctx.apply(x.astype(np.complex128))
            x_t = torch.tensor(x, device=dev)
            y_t = torch.empty_like(x_t)
            ctx.apply_noalloc(x_t, y_t)
            torch.cuda.synchronize()
            y = y_t.cpu().numpy().astype(np.complex128)
            # FP32 accumulation against the FP64-accumulated product (same c64 operator)
            assert np.linalg.norm(y - y_ref) <= 2e-6 * np.linalg.norm(y_ref)


def test_apply_noalloc_error_paths():
    """The documented refusals: a complex128 operator (BEM_ERR_STATE), and an
    operator whose scratch exceeds the fixed 32 MiB array (BEM_ERR_INVALID_ARG;
    20,480 elements with leaf 16 need about 44 MiB). Neither reaches a kernel."""
    import torch

    from paper_1212_3032_gb300 import binding, build

    build.build()
    dev = torch.device("cuda", 0)
    with binding.Context(0) as ctx:
        ctx.set_material(1.0, 0.25, 1.0)
        mesh = inputs.cavity_problem(4)
        o = binding.default_opts(leaf_size=16, precision=binding.PREC_C128)
        ctx.mesh(mesh.xyz, mesh.tri, mesh.bc_type, o)
        ctx.assemble(0.625 + 1.0j, o)
        x_t = torch.zeros(3 * mesh.ne, dtype=torch.complex64, device=dev)
        with pytest.raises(binding.BemError) as e:
            ctx.apply_noalloc(x_t, torch.empty_like(x_t))
        assert e.value.code == -7          # BEM_ERR_STATE
        mesh = inputs.cavity_problem(32)
        o = binding.default_opts(leaf_size=16, precision=binding.PREC_C64_MIXED)
        ctx.mesh(mesh.xyz, mesh.tri, mesh.bc_type, o)
        ctx.assemble(0.625 + 1.0j, o)
        x_t = torch.zeros(3 * mesh.ne, dtype=torch.complex64, device=dev)
        with pytest.raises(binding.BemError) as e:
            ctx.apply_noalloc(x_t, torch.empty_like(x_t))
        assert e.value.code == -1          # BEM_ERR_INVALID_ARG
        assert "maximum" in str(e.value)
