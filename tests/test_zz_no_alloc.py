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


def _dirty_the_array():
    """Run other meshes and schemes through the shared array first, so that the
    compared calls start from whatever those left behind (stale records, increment
    accumulators, face fluxes)."""
    for m, sch in ((synth.tri_mesh(23, 19, 0.2, 7),
                    dg.Scheme(k=4, r=1, n_diff=3, flux="upwind", nv=1, adv=(1.0, 0.4, 0.0), precision="fp32")),
                   (synth.tet_mesh(8, 0.15, 8),
                    dg.Scheme(k=5, r=2, n_diff=2, flux="rusanov", nv=5, gamma=1.4, precision="fp64"))):
        M = dg.Mesh(m)
        u = torch.rand((sch.nv, M.n_cells), dtype=torch.float64, device="cuda") + 1.0
        u[-1] += 2.0
        dg.dolinc_rk_step_noalloc(M, sch, 1e-3, u)
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_step_matches_workspace_step_twice(prec):
    """Same kernels, launch shapes and slot-ordered sums as dolinc_rk_step with the
    caller's own workspace: the states must be bitwise equal, call after call, even
    though the shared array holds another problem's leftovers."""
    _dirty_the_array()
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
        assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy())
    assert not np.array_equal(ref.cpu().numpy(), M.to_lib(u0))        # the steps did move the state


def test_noalloc_rejects_a_workspace_above_its_limit():
    m = synth.tet_mesh(32, 0.15, 42)                 # 163,840 cells: ~49 MB of workspace
    M = dg.Mesh(m)
    sch = dg.Scheme(k=3, r=1, n_diff=2, flux="rusanov", nv=5, gamma=1.4, precision="fp32")
    assert dg.dolinc_workspace_size(M, sch) > 32 << 20
    u = torch.ones((5, M.n_cells), dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DolincError) as e:
        dg.dolinc_rk_step_noalloc(M, sch, 1e-3, u)
    assert e.value.status == 1 and "DOLINC_NOALLOC_MAX_BYTES" in str(e.value)
