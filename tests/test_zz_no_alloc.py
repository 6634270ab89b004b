"""nl_assemble_noalloc: assembly into the caller's device array with no device allocation by
the library (for callers that reserve their device memory up front and cannot call cudaMalloc
while assembling).  Its output must match nl_assemble on the same mesh and pairs, call after
call, within the parity tolerance of the precision (FP64 1e-12; FP32 2e-6: nl_assemble's
scatter sums an element's FP32 blocks in FP32 shared memory, the allocation-free variant adds
each block to the FP64 values directly): the file-scope scratch it shares across calls keeps
the previous call's contents, so each call has to start from a clean state.  This file is
collected last on purpose."""
import numpy as np
import pytest

from nl_inputs import WORKLOADS, structured_mesh, workload_mesh
from paper_2101_08825_gb300 import nl

pytestmark = pytest.mark.gpu

CASES = [
    ("c1_fp64", lambda: workload_mesh(WORKLOADS["c1_2d"]), 0.1, 0.01, 3, nl.NL_PREC_FP64, 0),
    ("c1_fp32", lambda: workload_mesh(WORKLOADS["c1_2d"]), 0.1, 0.01, 3, nl.NL_PREC_FP32, 0),
    ("gauss2d_fp64", lambda: structured_mesh(2, 8, 1 / 8, 0.0, 2, jitter=0.1, seed=5), 0.2, 0.01,
     3, nl.NL_PREC_FP64, 1),
    ("jit3d_fp64", lambda: structured_mesh(3, 3, 1 / 3, 0.0, 1, jitter=0.1, seed=7), 0.22, 0.02,
     2, nl.NL_PREC_FP64, 0),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_assemble_on_two_calls(case):
    import torch
    name, mk, delta, eps, L_max, prec, kernel = case
    mesh = mk()
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, delta, eps)
    A, st_ref = nl.nl_assemble(m, p, delta, eps, L_max, kernel=kernel, precision=prec)
    ref = A.export()
    nnz = p.info()[1]
    out = torch.full((nnz,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        st = nl.nl_assemble_noalloc(m, p, delta, eps, L_max, out.data_ptr(), kernel=kernel,
                                    precision=prec)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel < (1e-12 if prec == nl.NL_PREC_FP64 else 2e-6), (name, call, rel)
        assert st.n_point_pairs == st_ref.n_point_pairs and st.n_items == st_ref.n_items


def test_noalloc_rejects_meshes_beyond_its_scratch():
    import torch
    # 2D: at most (16 MiB - 256 B) / 72 B = 233,013 elements
    mesh = structured_mesh(2, 340, 1.0 / 340, 0.0, 1)
    assert mesh.n_elem > 233013
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, 1.5 / 340, 0.1 / 340)
    out = torch.zeros(p.info()[1], dtype=torch.float64, device="cuda")
    with pytest.raises(nl.NLError) as e:
        nl.nl_assemble_noalloc(m, p, 1.5 / 340, 0.1 / 340, 2, out.data_ptr())
    assert e.value.status == nl.NL_EINVAL and "scratch" in str(e.value)


def test_noalloc_makes_no_device_allocation():
    # Every device allocation of the library goes through its allocator hook (nl_set_allocator).
    # A hook that counts its calls and refuses to allocate is installed around one call of the
    # allocation-free entry point (the handles are created before and released after, with the
    # default allocator): it must not be called, and the result must still match.  The ordinary
    # entry point, under the same hook, asks for memory and fails with NL_ENOMEM.
    import ctypes
    import torch
    w = WORKLOADS["c1_2d"]
    mesh = workload_mesh(w)
    m = nl.mesh_from(mesh)
    p = nl.nl_pairs_build(m, w.delta, w.eps)
    A, _ = nl.nl_assemble(m, p, w.delta, w.eps, w.L_max)
    ref = A.export()
    out = torch.zeros(p.info()[1], dtype=torch.float64, device="cuda")
    calls = []
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    alloc_cb = ALLOC(lambda nbytes, stream, ctx: calls.append(int(nbytes)) or None)
    free_cb = FREE(lambda ptr, nbytes, stream, ctx: calls.append(-1))
    L = nl.lib()
    assert L.nl_set_allocator(ctypes.cast(alloc_cb, ctypes.c_void_p), ctypes.cast(free_cb, ctypes.c_void_p), None) == 0
    try:
        nl.nl_assemble_noalloc(m, p, w.delta, w.eps, w.L_max, out.data_ptr())
        torch.cuda.synchronize()
        assert calls == []
        with pytest.raises(nl.NLError) as e:
            nl.nl_assemble(m, p, w.delta, w.eps, w.L_max)
        assert e.value.status == nl.NL_ENOMEM and calls
    finally:
        assert L.nl_set_allocator(None, None, None) == 0
    got = out.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
