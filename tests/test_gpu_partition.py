"""Partitioned meshes on the GPU: the parts of one mesh, each with its own cells and a
depth-1 ghost layer, stepped through dolinc_part_step_begin / _continue with the
halo exchanges done in-process (copies between the parts' workspaces on one stream;
no kernel waits for another part).  A part keeps the whole mesh's cell order, face
order and orientation and geometry, so its own cells must end bit-identical to the
whole mesh's step under the same launch shapes (Sec 2.6: coupled boundaries need
only the adjacent cells' data and differentials)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
dg = pytest.importorskip("paper_2404_08952_gb300")
pytestmark = pytest.mark.gpu

CASES = {
    "tet_euler": lambda: synth.workload("euler3d_tet64", size=8, q=1),
    "tri_riemann": lambda: synth.workload("euler2d_riemann", size=18, q=1),
    "hexprism_order5": lambda: synth.workload("adv3d_hexprism", order=5, size=8, q=1),
    "tri_adv": lambda: synth.workload("adv2d_tri64", size=20, q=1),
}
_cache = {}


def case(name):
    if name not in _cache:
        _cache[name] = CASES[name]()
    return _cache[name]


def exchange_in_process(parts, wss, hs):
    """Each part's receive buffer, peer by peer, from that peer's send buffer."""
    views = [h.views(ws, P.plan) for P, ws, h in zip(parts, wss, hs)]
    for p, vp in enumerate(views):
        for q, _, rcv in vp:
            snd = [s for (pp, s, _) in views[q] if pp == p][0]
            assert snd.numel() == rcv.numel()
            rcv.copy_(snd)


SHAPES = [(1, 128, -2, 128), (4, 128, 4, 64)]


@pytest.mark.parametrize("name,n_parts,prec", [("tet_euler", 2, "fp32"), ("tet_euler", 3, "fp64"),
                                               ("tet_euler", 1, "fp32"), ("tri_riemann", 2, "fp64"),
                                               ("tri_riemann", 4, "fp32"), ("hexprism_order5", 3, "fp32"),
                                               ("hexprism_order5", 2, "fp64"), ("tri_adv", 5, "fp32_bf16")])
@pytest.mark.parametrize("shape", SHAPES)
def test_parts_step_like_the_whole_mesh(name, n_parts, prec, shape):
    w = case(name)
    m = w["mesh"]
    sch = dg.Scheme(precision=prec, **w["scheme"])
    M = dg.Mesh(m)
    dg.dolinc_set_tuning(M, sch, *shape)
    ws = dg.workspace(M, sch)
    u = torch.from_numpy(M.to_lib(w["u0"])).cuda()
    for _ in range(2):
        dg.dolinc_rk_step(M, sch, w["dt"], u, ws)
    dg.dolinc_sync_status(M, ws)
    whole = M.from_lib(u.cpu().numpy())
    pc = dg.dolinc_partition(m, n_parts)
    parts = [dg.Mesh(m, part=(pc, n_parts, p)) for p in range(n_parts)]
    wss, us = [], []
    for P in parts:
        dg.dolinc_set_tuning(P, sch, *shape)
        wss.append(dg.workspace(P, sch))
        x = w["u0"][:, P.plan["local_cells"]].copy()
        x[:, P.plan["owned"] == 0] += 0.25               # ghost entries are not read: any finite value
        us.append(torch.from_numpy(x).cuda())
    assert sum(int(P.plan["owned"].sum()) for P in parts) == M.n_cells
    exchanges = 0
    for _ in range(2):
        hs = [dg.dolinc_part_step_begin(P, sch, w["dt"], x, ws) for P, x, ws in zip(parts, us, wss)]
        while hs[0].pending:
            assert all(h.pending and h.order == hs[0].order for h in hs)
            exchange_in_process(parts, wss, hs)
            exchanges += 1
            hs = [dg.dolinc_part_step_continue(P, sch, ws) for P, ws in zip(parts, wss)]
        assert not any(h.pending for h in hs)
    # per stage: orders 0 .. max(n_diff - 1, the stencil's order)
    ns = max(sch.r, sch.k - sch.r - 2, 1)
    assert exchanges == 2 * 3 * (max(sch.n_diff - 1, ns) + 1)
    for P, x, ws in zip(parts, us, wss):
        dg.dolinc_sync_status(P, ws)
        got = x.cpu().numpy()
        own = P.plan["owned"].astype(bool)
        assert np.array_equal(got[:, own], whole[:, P.plan["local_cells"][own]])


def test_part_step_errors():
    w = case("tet_euler")
    m = w["mesh"]
    sch = dg.Scheme(precision="fp32", **w["scheme"])
    M = dg.Mesh(m)
    ws = dg.workspace(M, sch)
    u = torch.from_numpy(M.to_lib(w["u0"])).cuda()
    with pytest.raises(dg.DolincError):                  # not a part mesh
        dg.dolinc_part_step_begin(M, sch, w["dt"], u, ws)
    pc = dg.dolinc_partition(m, 2)
    P = dg.Mesh(m, part=(pc, 2, 0))
    wp = dg.workspace(P, sch)
    with pytest.raises(dg.DolincError):                  # no step in progress
        dg.dolinc_part_step_continue(P, sch, wp)
    assert dg.dolinc_workspace_size(P, sch) > 0
