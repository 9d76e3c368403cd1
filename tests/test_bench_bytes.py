"""The roofline's algorithmic bytes (bench.alg_bytes) reproduce the per-cell B_alg
table of the measurement plan: bytes per cell per stage summed over the differential
passes and the stage, for the four mesh families and N_d = 1..4, FP64 / FP32 bulk."""
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


@pytest.mark.parametrize("family", list(TABLE), ids=lambda f: "dim%d_nv%d_nfc%.2f" % f)
def test_alg_bytes_match_the_table(family):
    dim, nv, nfc = family
    n = 3000
    M = SimpleNamespace(n_cells=n, dim=dim, n_slots=int(round(n * nfc)), n_faces=0)
    for nd, want in TABLE[family].items():
        for prec, w in zip(("fp64", "fp32"), want):
            sch = SimpleNamespace(nv=nv, precision=prec, n_diff=nd)
            total = sum(bench.alg_bytes("diff%d" % m, M, sch) for m in range(1, nd + 1))
            total += bench.alg_bytes("stage", M, sch)
            assert total / n == pytest.approx(w, abs=0.5)
