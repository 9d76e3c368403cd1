"""Batched persistent stages: many meshes of uneven size advanced by one cooperative
launch per SSP-RK3 stage (optionally replayed from a CUDA graph) must give what the
per-mesh path and the oracle give; a grid-barrier wait that gives up is reported as
a device timeout without touching the state."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
dg = pytest.importorskip("paper_2404_08952_gb300")
pytestmark = pytest.mark.gpu


def _batch_case(kind):
    rng = np.random.default_rng(77)
    out = []
    if kind == "burgers2d":
        for i, (nx, ny) in enumerate([(8, 8), (11, 7), (20, 17), (5, 9), (31, 3)]):
            m = synth.tri_mesh(nx, ny, 0.2, 100 + i)
            u0 = synth.cell_average(m, synth.fourier_modes(200 + i), q=3)[None]
            out.append((m, u0, float(rng.uniform(2e-3, 6e-3))))
        sch = dict(k=3, r=1, n_diff=2, flux="burgers", nv=1)
    else:
        for i, n in enumerate([4, 6]):
            m = synth.tet_mesh(n, 0.15, 300 + i)
            u0 = synth.cell_average(m, lambda p: synth.isentropic_vortex(p, dim=3, R=0.2, images=0), q=2, nv=5)
            out.append((m, u0, 1e-3 * (i + 1)))
        sch = dict(k=4, r=1, n_diff=2, flux="rusanov", nv=5, gamma=1.4)
    return out, sch


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("kind", ["burgers2d", "euler3d"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("graph", [True, False])
def test_batch_matches_per_mesh_and_oracle(kind, prec, graph):
    cases, sch_kw = _batch_case(kind)
    meshes = [dg.Mesh(m) for m, _, _ in cases]
    bt = dg.Batch(meshes)
    sch = dg.Scheme(precision=prec, **sch_kw)
    ws = bt.workspace(sch)
    u = torch.from_numpy(bt.to_lib([u0 for _, u0, _ in cases])).cuda()
    dt = torch.tensor([d for _, _, d in cases], dtype=torch.float64, device="cuda")
    steps = 3
    for _ in range(steps):
        bt.rk_step(sch, dt, u, ws, use_graph=graph)
    dg.dolinc_sync_status(meshes[0], ws)
    got = bt.from_lib(u.cpu().numpy())
    for (m, u0, d), M, g in zip(cases, meshes, got):
        # per-mesh library path
        w = dg.workspace(M, sch)
        x = torch.from_numpy(M.to_lib(u0)).cuda()
        for _ in range(steps):
            dg.dolinc_rk_step(M, sch, d, x, w)
        ref = M.from_lib(x.cpu().numpy())
        tol = 1e-13 if prec == "fp64" else 1e-6
        assert rel(g - u0, ref - u0) < tol * 100 or rel(g, ref) < tol
        if prec == "fp64":
            want = oracle.Oracle(m).run(u0, oracle.Scheme(**sch_kw), d, steps)
            assert rel(g, want) < 1e-12


def test_batch_barrier_timeout_is_reported_and_leaves_state():
    cases, sch_kw = _batch_case("burgers2d")
    meshes = [dg.Mesh(m) for m, _, _ in cases]
    bt = dg.Batch(meshes)
    sch = dg.Scheme(precision="fp64", **sch_kw)
    ws = bt.workspace(sch)
    u0 = bt.to_lib([c[1] for c in cases])
    u = torch.from_numpy(u0).cuda()
    dt = torch.tensor([c[2] for c in cases], dtype=torch.float64, device="cuda")
    bt.set_spin_limit(0)                      # every grid-barrier wait gives up at once
    bt.rk_step(sch, dt, u, ws, use_graph=False)
    with pytest.raises(dg.DolincError) as e:
        dg.dolinc_sync_status(meshes[0], ws)
    assert e.value.status == 5
    np.testing.assert_array_equal(u.cpu().numpy(), u0)
    bt.set_spin_limit(1 << 23)                # recovered: the status read cleared the barrier words
    bt.rk_step(sch, dt, u, ws, use_graph=False)
    dg.dolinc_sync_status(meshes[0], ws)
    assert np.abs(u.cpu().numpy() - u0).max() > 0


def test_batch_autotune_keeps_results():
    cases, sch_kw = _batch_case("burgers2d")
    meshes = [dg.Mesh(m) for m, _, _ in cases]
    bt = dg.Batch(meshes)
    sch = dg.Scheme(precision="fp64", **sch_kw)
    ws = bt.workspace(sch)
    u0 = bt.to_lib([c[1] for c in cases])
    u = torch.from_numpy(u0).cuda()
    dt = torch.tensor([c[2] for c in cases], dtype=torch.float64, device="cuda")
    t = bt.autotune(sch, dt, u, ws)
    assert t["block"] in (64, 128, 256) and t["grid"] >= 1
    np.testing.assert_array_equal(u.cpu().numpy(), u0)     # autotune restores the field
    bt.rk_step(sch, dt, u, ws)
    dg.dolinc_sync_status(meshes[0], ws)
    got = bt.from_lib(u.cpu().numpy())
    for (m, u0m, d), g in zip(cases, got):
        want = oracle.Oracle(m).rk3_step(u0m, oracle.Scheme(**sch_kw), d)
        assert rel(g, want) < 1e-12
