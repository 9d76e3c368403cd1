"""The roofline's algorithmic bytes (bench.alg_bytes) per cell per stage, summed over
the differential passes and the stage, for the four mesh families.

basis "table": the scope table's own evaluation (geometry at FP64 widths, the stage
reading every computed order), N_d = 1..4, FP64 / FP32 bulk.
basis "stored" (what the roofline reports): geometry at the stored widths (FP32
tables below FP64) and the stage reading the orders its stencil needs (here N_s = 1,
USR3), worked by hand from the per-cell formula:
  Gp = 8 nfc + (nfc/2)(D s_g + s_g) + (s_g + 4),  Gr = Gp + (nfc/2) D s_g
  diff m = nv s_b (c_{m-1} + c_m) + Gp,  stage = nv s_b (c_0 + c_1) + Gr + nv (24 + s_b)
e.g. tetrahedra, Euler, FP32: Gp = 32 + 2 * 16 + 8 = 72, Gr = 96, diff1 = 20 * 4 + 72 =
152, diff2 = 20 * 9 + 72 = 252, stage = 80 + 96 + 140 = 316.
"""
from types import SimpleNamespace

import pytest

import bench

# (dim, nv, slots per cell) -> {N_d: (FP64, FP32)}
TABLE = {
    (2, 1, 3): {1: (248, 220), 2: (384, 324), 3: (544, 440), 4: (728, 568)},          # 2D triangles, scalar
    (3, 5, 4): {1: (744, 564), 2: (1452, 972), 3: (2600, 1600), 4: (4308, 2508)},     # tetrahedra, Euler
    (3, 1, 16 / 3): {1: (440, 404), 2: (700, 604), 3: (1048, 848), 4: (1508, 1148)},  # hex/prism, scalar
    (2, 4, 3): {1: (488, 376), 2: (816, 576), 3: (1240, 824), 4: (1760, 1120)},       # 2D triangles, Euler
}

# stored widths, USR3 (stage reads orders 0..1): (dim, nv, nfc) -> {N_d: (FP64, FP32)}
STORED = {
    (2, 1, 3): {1: (248, 164), 2: (360, 234), 3: (488, 312), 4: (632, 398)},
    (3, 5, 4): {1: (744, 468), 2: (1212, 720), 3: (1960, 1112), 4: (3068, 1684)},
    (3, 1, 16 / 3): {1: (440, 278.67), 2: (652, 408), 3: (920, 565.33), 4: (1260, 758.67)},
    (2, 4, 3): {1: (488, 320), 2: (720, 450), 3: (1016, 612), 4: (1376, 806)},
}


def _total(M, nd, prec, nv, basis):
    sch = SimpleNamespace(nv=nv, precision=prec, n_diff=nd, k=3, r=1, limiter="none")
    total = sum(bench.alg_bytes("diff%d" % m, M, sch, basis) for m in range(1, nd + 1))
    return (total + bench.alg_bytes("stage", M, sch, basis)) / M.n_cells


@pytest.mark.parametrize("family", list(TABLE), ids=lambda f: "dim%d_nv%d_nfc%.2f" % f)
def test_alg_bytes_match_the_scope_table(family):
    dim, nv, nfc = family
    n = 3000
    M = SimpleNamespace(n_cells=n, dim=dim, n_slots=int(round(n * nfc)), n_faces=0)
    for nd, want in TABLE[family].items():
        for prec, w in zip(("fp64", "fp32"), want):
            assert _total(M, nd, prec, nv, "table") == pytest.approx(w, abs=0.5)


@pytest.mark.parametrize("family", list(STORED), ids=lambda f: "dim%d_nv%d_nfc%.2f" % f)
def test_alg_bytes_at_stored_widths(family):
    dim, nv, nfc = family
    n = 3000
    M = SimpleNamespace(n_cells=n, dim=dim, n_slots=int(round(n * nfc)), n_faces=0)
    for nd, want in STORED[family].items():
        for prec, w in zip(("fp64", "fp32"), want):
            assert _total(M, nd, prec, nv, "stored") == pytest.approx(w, abs=0.5)


def test_stage_orders_follow_the_stencil_and_limiter():
    s = lambda **kw: SimpleNamespace(**dict(dict(k=3, r=1, n_diff=2, limiter="none"), **kw))
    assert bench.stage_orders(s()) == 1
    assert bench.stage_orders(s(k=5, r=2)) == 2
    assert bench.stage_orders(s(limiter="weno5_all")) == 2
    assert bench.stage_orders(s(k=2, r=1, n_diff=1)) == 1
    assert bench.stage_orders(s(k=9, r=4, n_diff=4)) == 4


@pytest.mark.parametrize("nfc,per_it", [(3, 208), (4, 232), (16 / 3, 264)])
def test_solve_bytes(nfc, per_it):
    """Semi-implicit solve, per cell: an iteration reads or writes 16 FP64 vectors
    (128 B) and the scaled rows twice, 2 (12 nfc + 4) B (triangles 128 + 80 = 208,
    tetrahedra 128 + 104 = 232, hex/prism 128 + 136 = 264); a solve adds 72 B of
    set-up and final update."""
    n = 3000
    M = SimpleNamespace(n_cells=n, n_slots=nfc * n)
    assert bench.solve_alg_bytes(M, 1, 0) / n == pytest.approx(per_it)
    assert bench.solve_alg_bytes(M, 0, 1) / n == pytest.approx(72)
    assert bench.solve_alg_bytes(M, 7, 2) / n == pytest.approx(7 * per_it + 144)
