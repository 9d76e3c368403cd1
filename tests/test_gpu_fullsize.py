"""Parity at the workloads' full sizes, in the launch configuration the benchmark
times (Morton renumbering, autotuned launch shape).

  adv2d_tri64    8192 triangles, 100 full SSP-RK3 steps, FP64, every cell.
  euler3d_tet64  1,310,720 tetrahedra, one full stage from the vortex, FP64 and FP32,
                 every cell (the oracle runs one stage in a few seconds).
  euler2d_riemann ~1.05M triangles, residual with the criterion-flagged ENO3 limiter,
                 FP64, every cell.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
dg = pytest.importorskip("paper_2404_08952_gb300")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_adv2d_tri64_full_run_fp64():
    w = synth.workload("adv2d_tri64")
    M = dg.Mesh(w["mesh"])
    sch = dg.Scheme(precision="fp64", **w["scheme"])
    ws = dg.workspace(M, sch)
    u = torch.from_numpy(M.to_lib(w["u0"])).cuda()
    dg.dolinc_autotune(M, sch, u, ws)
    for _ in range(w["steps"]):
        dg.dolinc_rk_step(M, sch, w["dt"], u, ws)
    dg.dolinc_sync_status(M, ws)
    got = M.from_lib(u.cpu().numpy())
    want = oracle.Oracle(w["mesh"]).run(w["u0"], oracle.Scheme(**w["scheme"]), w["dt"], w["steps"])
    assert rel(got, want) < 1e-10


@pytest.fixture(scope="module")
def tet64():
    w = synth.workload("euler3d_tet64", q=2)
    O = oracle.Oracle(w["mesh"])
    want = O.rk3_stage(w["u0"], w["u0"], oracle.Scheme(**w["scheme"]), w["dt"], 0)
    return w, want


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_euler3d_tet64_full_stage(tet64, prec):
    w, want = tet64
    M = dg.Mesh(w["mesh"])
    sch = dg.Scheme(precision=prec, **w["scheme"])
    ws = dg.workspace(M, sch)
    u = torch.from_numpy(M.to_lib(w["u0"])).cuda()
    dg.dolinc_autotune(M, sch, u, ws)
    out = torch.zeros_like(u)
    dg.dolinc_rk_stage(M, sch, w["dt"], 0, u, u, out, ws)
    dg.dolinc_sync_status(M, ws)
    got = M.from_lib(out.cpu().numpy())
    inc, inc_ref = got - w["u0"], want - w["u0"]
    if prec == "fp64":
        assert rel(got, want) < 1e-13 and rel(inc, inc_ref) < 1e-11
    else:
        # FP32 bulk: the stage increment (dt * residual) to 1e-5 of the flux scale
        assert rel(inc, inc_ref) < 2e-4
        assert rel(got, want) < 1e-6


def test_euler2d_riemann_full_residual_with_limiter():
    w = synth.workload("euler2d_riemann", q=2)
    O = oracle.Oracle(w["mesh"])
    osch = oracle.Scheme(**w["scheme"])
    flags = O.criterion(w["u0"], osch)
    M = dg.Mesh(w["mesh"])
    sch = dg.Scheme(precision="fp64", limiter="eno3_flagged", **w["scheme"])
    fl = torch.from_numpy(M.to_lib(flags)).cuda()
    dg.dolinc_set_flags(M, fl)
    ws = dg.workspace(M, sch)
    u = torch.from_numpy(M.to_lib(w["u0"])).cuda()
    # the GPU criterion agrees with the oracle's on the full mesh
    gfl = torch.zeros_like(fl)
    dg.dolinc_criterion(M, sch, u, gfl, ws)
    assert (M.from_lib(gfl.cpu().numpy()) == flags).mean() == 1.0
    R = torch.zeros_like(u)
    dg.dolinc_residual(M, sch, u, R, ws)
    got = M.from_lib(R.cpu().numpy())
    want = O.residual(w["u0"], oracle.Scheme(eno=2, troubled=flags, **w["scheme"]))
    assert rel(got, want) < 1e-11
    dg.dolinc_set_flags(M, None)
