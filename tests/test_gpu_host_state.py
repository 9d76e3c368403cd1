"""dolinc_rk_step_host: the SSP-RK3 step (Sec 3) of a state held in host memory.

With pinned (mapped) host memory the step's kernels read and write the state in place;
with pageable memory the library copies it in and out.  Either way the arithmetic is
that of dolinc_rk_step, so the results must be bit-identical to the device step, and
the FP64 step must match the oracle's."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

dg = pytest.importorskip("paper_2404_08952_gb300")

from test_gpu_parity import euler_ok, field, mesh, rel  # noqa: E402


def _host(a, kind):
    t = torch.from_numpy(np.ascontiguousarray(a).copy())
    return t.pin_memory() if kind == "pinned" else t


@pytest.mark.parametrize("kind", ["pinned", "pageable"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_bf16"])
def test_host_step_is_the_device_step(prec, kind):
    """Three steps of 3D Euler with USR3 and differentials through order 2 (the order-2
    pass runs beside the stage on the side stream): bit-identical to dolinc_rk_step."""
    m, _ = mesh("tet")
    M = dg.Mesh(m)
    u = field(m, 5, seed=21)
    sch = dg.Scheme(k=3, r=1, n_diff=2, precision=prec, nv=5, **euler_ok(5))
    ws = dg.workspace(M, sch)
    dt = 2e-3
    x = torch.from_numpy(M.to_lib(u)).cuda()
    uh = _host(M.to_lib(u), kind)
    ud = torch.empty_like(uh, device="cuda")
    for _ in range(3):
        dg.dolinc_rk_step(M, sch, dt, x, ws)
        dg.dolinc_rk_step_host(M, sch, dt, uh, ud, ws)
    torch.cuda.synchronize()
    dg.dolinc_sync_status(M, ws)
    assert np.array_equal(uh.numpy(), x.cpu().numpy())


@pytest.mark.parametrize("name,nv", [("tri_bnd", 4), ("hexprism", 1)])
def test_host_step_matches_the_oracle(name, nv):
    """One FP64 step from host memory against the oracle's SSP-RK3 step (mixed
    hex/prism cells: CSR slot ranges; triangles with transmissive faces)."""
    m, O = mesh(name)
    M = dg.Mesh(m)
    u = field(m, nv, seed=22)
    kw = euler_ok(nv) if nv > 1 else dict(flux="upwind", adv=(1.0, 0.5, 0.3))
    sch = dg.Scheme(k=3, r=1, n_diff=1, precision="fp64", nv=nv, **kw)
    ws = dg.workspace(M, sch)
    dt = 2e-3
    uh = _host(M.to_lib(u), "pinned")
    ud = torch.empty_like(uh, device="cuda")
    dg.dolinc_rk_step_host(M, sch, dt, uh, ud, ws)
    torch.cuda.synchronize()
    want = O.rk3_step(u, oracle.Scheme(k=3, r=1, n_diff=1, nv=nv, **kw), dt)
    assert rel(M.from_lib(uh.numpy()), want) < 1e-12


def test_host_step_rejects_buffers_it_cannot_use():
    m, _ = mesh("tri")
    M = dg.Mesh(m)
    sch = dg.Scheme(k=3, r=1, n_diff=1, precision="fp32", nv=1, flux="upwind", adv=(1.0, 0.5, 0.0))
    ws = dg.workspace(M, sch)
    uh = torch.zeros(M.n_cells, dtype=torch.float64).pin_memory()
    with pytest.raises(dg.DolincError, match="device memory"):
        dg.dolinc_rk_step_host(M, sch, 1e-3, uh, torch.zeros_like(uh), ws)     # scratch on the host
    with pytest.raises(dg.DolincError, match="different buffers"):
        dg.dolinc_rk_step_host(M, sch, 1e-3, uh, uh, ws)
