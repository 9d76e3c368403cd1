"""dolinc_rk_step_noalloc — the step for callers that cannot allocate device memory
(they hold only their field's device pointer, e.g. a plugin inside a host
application with no allocator of its own).  Its workspace is a fixed array inside
the library, so the call must give exactly what dolinc_rk_step gives with a
caller-allocated workspace, call after call.

This file is collected last on purpose (test_zz_*): if it fails, a run that stops at
the first failure has already run every other test.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
dg = pytest.importorskip("paper_2404_08952_gb300")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_step_matches_workspace_step_twice(prec):
    m = synth.tet_mesh(6, 0.15, 41)
    u0 = synth.cell_average(m, lambda p: synth.isentropic_vortex(p, dim=3, R=0.2, images=0), q=2, nv=5)
    M = dg.Mesh(m)
    sch = dg.Scheme(k=3, r=1, n_diff=2, flux="rusanov", nv=5, gamma=1.4, precision=prec)
    assert dg.dolinc_workspace_size(M, sch) <= 32 << 20
    dt = 1e-3
    ws = dg.workspace(M, sch)
    ref = torch.from_numpy(M.to_lib(u0)).cuda()
    got = ref.clone()
    for _ in range(2):                      # two calls in a row: the shared array is reused
        dg.dolinc_rk_step(M, sch, dt, ref, ws)
        dg.dolinc_rk_step_noalloc(M, sch, dt, got)
        torch.cuda.synchronize()
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        tol = 1e-12 if prec == "fp64" else 1e-5
        assert np.abs(a - b).max() <= tol * np.abs(b).max()


def test_noalloc_rejects_a_workspace_above_its_limit():
    m = synth.tet_mesh(32, 0.15, 42)                 # 163,840 cells: ~49 MB of workspace
    M = dg.Mesh(m)
    sch = dg.Scheme(k=3, r=1, n_diff=2, flux="rusanov", nv=5, gamma=1.4, precision="fp32")
    assert dg.dolinc_workspace_size(M, sch) > 32 << 20
    u = torch.ones((5, M.n_cells), dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DolincError) as e:
        dg.dolinc_rk_step_noalloc(M, sch, 1e-3, u)
    assert e.value.status == 1 and "DOLINC_NOALLOC_MAX_BYTES" in str(e.value)
