"""The allocation-free Jacobian entry point against the ordinary one (GPU).

bp_assemble_jacobian_noalloc serves callers that must not allocate device memory while they
run (a fixed memory budget, or a framework whose allocator owns the device): it keeps its
residual scratch in a fixed array inside the library instead of allocating one.  These tests
call it through the C ABI twice in a row and compare its Jacobian with bp_assemble_jacobian's
at the parity tolerances of the other GPU tests, and check that meshes beyond its fixed
capacity are refused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2204_04321_b300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_noalloc_matches_allocating_entry_point_twice(precision, tol):
    from paper_2204_04321_b300 import capi
    L = capi.lib()
    mesh = synth.config_small()
    dm = capi.DeviceMesh(mesh)
    dtype = torch.float64 if precision == capi.BP_F64 else torch.float32
    stream = capi._stream_ptr(None)
    for seed in (103, 104):  # two calls in a row, different velocities
        U = torch.as_tensor(synth.random_velocity(mesh, seed), device="cuda")
        J_ref = torch.empty(dm.nnz, dtype=dtype, device="cuda")
        R_ref = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
        rc = L.bp_assemble_jacobian(dm.handle, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(R_ref.data_ptr()),
                                    ctypes.c_void_p(J_ref.data_ptr()), precision, capi.BP_SCATTER_ATOMIC,
                                    capi.BP_JAC_FACTORED, stream)
        assert rc == capi.BP_OK
        J = torch.full((dm.nnz,), 7.0, dtype=dtype, device="cuda")  # garbage: the call must overwrite
        rc = L.bp_assemble_jacobian_noalloc(dm.handle, ctypes.c_void_p(U.data_ptr()),
                                            ctypes.c_void_p(J.data_ptr()), precision,
                                            capi.BP_SCATTER_ATOMIC, capi.BP_JAC_FACTORED, stream)
        assert rc == capi.BP_OK, capi.bp_strerror(rc)
        torch.cuda.synchronize()
        assert _rel(J.double(), J_ref.double()) <= tol
    dm.close()


def test_noalloc_refuses_meshes_beyond_capacity():
    from paper_2204_04321_b300 import capi
    mesh = synth.dome_mesh(224, 10, 201, 202)   # 1,113,750 dofs > 1,048,576
    assert mesh.ndof > capi.BP_NOALLOC_MAX_NDOF
    dm = capi.DeviceMesh(mesh)
    U = torch.zeros(dm.ndof, dtype=torch.float64, device="cuda")
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = capi.lib().bp_assemble_jacobian_noalloc(dm.handle, ctypes.c_void_p(U.data_ptr()),
                                                 ctypes.c_void_p(J.data_ptr()), capi.BP_F64,
                                                 capi.BP_SCATTER_AUTO, capi.BP_JAC_AUTO, None)
    assert rc == capi.BP_ESIZE
    assert "capacity" in capi.bp_strerror(rc)
    dm.close()


def test_noalloc_first_call_on_a_fresh_mesh_allocates_nothing():
    """A caller that cannot allocate must be able to rely on it: the device's free memory is the
    same before and after the entry point's first call on a freshly uploaded mesh (the library's
    kernels are already loaded by an ordinary assembly on another mesh)."""
    from paper_2204_04321_b300 import capi
    L = capi.lib()
    warm = capi.DeviceMesh(synth.dome_mesh(6, 3, 11, 12))
    Uw = torch.as_tensor(synth.random_velocity(warm.mesh, 1), device="cuda")
    warm.jacobian(Uw)
    Jw = torch.empty(warm.nnz, dtype=torch.float64, device="cuda")
    assert L.bp_assemble_jacobian_noalloc(warm.handle, ctypes.c_void_p(Uw.data_ptr()),
                                          ctypes.c_void_p(Jw.data_ptr()), capi.BP_F64,
                                          capi.BP_SCATTER_ATOMIC, capi.BP_JAC_FACTORED, None) == capi.BP_OK
    mesh = synth.config_small()
    dm = capi.DeviceMesh(mesh)
    U = torch.as_tensor(synth.random_velocity(mesh, 103), device="cuda")
    J = torch.empty(dm.nnz, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    rc = L.bp_assemble_jacobian_noalloc(dm.handle, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(J.data_ptr()),
                                        capi.BP_F64, capi.BP_SCATTER_ATOMIC, capi.BP_JAC_FACTORED, None)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert rc == capi.BP_OK
    assert free1 == free0, (free0, free1)
    dm.close()
    warm.close()
