"""Degenerate sizes: meshes of 5 to 320 cells, mostly fewer than one block and fewer
faces than one flux block, so grids are one or two ragged blocks and the persistent
kernels get fewer tiles than CTAs.  Every launch shape must still give the oracle's
SSP-RK3 steps."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

dg = pytest.importorskip("paper_2404_08952_gb300")

from test_gpu_parity import euler_ok, field, rel  # noqa: E402

TINY = {
    "tri3": lambda: synth.tri_mesh(3, 3, 0.15, 31),                                   # 18 triangles
    "tet4": lambda: synth.tet_mesh(4, 0.1, 32),                                       # 320 tetrahedra
    "hexprism3": lambda: synth.hexprism_mesh(3, 0.1, 33),                             # 36 mixed cells
    "strip5": lambda: synth.strip_mesh(0.1 * 1.2 ** np.arange(5), height=0.1, boundary="transmissive"),  # 5 cells
}

# (diff lanes, diff block, stage lanes, stage block)
SHAPES = [(1, 64, 1, 64), (4, 128, 4, 128), (8, 256, 8, 256), (0, 64, 0, 64), (-1, 128, -1, 64),
          (-4, 256, -1, 128), (1, 64, -2, 64), (1, 32, -2, 256)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "d%d_%d_s%d_%d" % s)
@pytest.mark.parametrize("name,nv,prec", [("tri3", 1, "fp64"), ("tet4", 5, "fp64"), ("tet4", 5, "fp32"),
                                          ("hexprism3", 1, "fp64"), ("strip5", 1, "fp64")])
def test_tiny_meshes_every_launch_shape(name, nv, prec, shape):
    m = TINY[name]()
    O = oracle.Oracle(m)
    M = dg.Mesh(m)
    u = field(m, nv, seed=60)
    fx = euler_ok(nv) if nv > 1 else dict(flux="upwind", adv=(1.0, 0.5, 0.3))
    sch = dg.Scheme(k=3, r=1, n_diff=2, nv=nv, precision=prec, **fx)
    ws = dg.workspace(M, sch)
    dg.dolinc_set_tuning(M, sch, *shape)
    x = torch.from_numpy(M.to_lib(u)).cuda()
    dt = 1e-3
    for _ in range(2):
        dg.dolinc_rk_step(M, sch, dt, x, ws)
    dg.dolinc_sync_status(M, ws)
    got = M.from_lib(x.cpu().numpy())
    want = u
    osch = oracle.Scheme(k=3, r=1, n_diff=2, nv=nv, **fx)
    for _ in range(2):
        want = O.rk3_step(want, osch, dt)
    if prec == "fp64":
        assert rel(got, want) < 1e-12
    else:
        assert rel(got - u, want - u) < 1e-4


def test_misaligned_differential_buffer_is_rejected():
    """The differential records are read with 16- and 32-byte vector loads and written
    by bulk copies: a caller buffer that is not 256-byte aligned is refused on the
    host, before any launch."""
    m = TINY["tri3"]()
    M = dg.Mesh(m)
    sch = dg.Scheme(k=3, r=1, n_diff=2, nv=1, precision="fp32", flux="upwind", adv=(1.0, 0.5, 0.3))
    ws = dg.workspace(M, sch)
    _, _, _, tot = dg.dolinc_diff_layout(M, sch, 2)
    buf = torch.zeros(tot + 256, dtype=torch.uint8, device="cuda")
    u = torch.zeros(M.n_cells, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DolincError, match="256-byte aligned"):
        dg.dolinc_differentials(M, sch, u, 2, buf[16:], ws)
    dg.dolinc_differentials(M, sch, u, 2, buf[:tot], ws)
    torch.cuda.synchronize()
