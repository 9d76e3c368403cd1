"""The skewness correction on the GPU (dolinc_mesh_set_skew_correction) against the
oracle's corrected operators, element by element on the same seeded inputs, with the
tolerance rule of the other parity tests; exactness for linear fields at face
centroids on skewed simplices; launch shapes bit-identical; and the rejections."""
import numpy as np
import pytest

import oracle
import synth
from _tol import cell_tol, face_tol, increment_ok, wave_speed

torch = pytest.importorskip("torch")
dg = pytest.importorskip("paper_2404_08952_gb300")
pytestmark = pytest.mark.gpu

from test_gpu_parity import RES_CASES, euler_ok, field, poly_coeffs, rel, scheme_order, to_dev  # noqa: E402

MESHES = {
    "tri": lambda: synth.tri_mesh(21, 17, 0.2, 11),
    "tri_bnd": lambda: synth.tri_mesh(19, 13, 0.2, 12, boundary="transmissive"),
    "tet": lambda: synth.tet_mesh(6, 0.15, 13),
    "hexprism": lambda: synth.hexprism_mesh(7, 0.2, 14),
}
_cache = {}


def mesh(name):
    if name not in _cache:
        m = MESHES[name]()
        _cache[name] = (m, oracle.Oracle(m, skew=True))
    return _cache[name]


def skew_mesh(m):
    M = dg.Mesh(m)
    dg.dolinc_mesh_set_skew_correction(M, True)
    return M


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,nv", [("tri", 1), ("tri_bnd", 4), ("tet", 5), ("hexprism", 1)])
def test_differentials(prec, name, nv):
    m, O = mesh(name)
    M = skew_mesh(m)
    u = field(m, nv, seed=1)
    N = 4
    sch = dg.Scheme(k=3, r=1, n_diff=N, nv=nv, precision=prec, **(euler_ok(nv) if nv > 1 else {}))
    ws = dg.workspace(M, sch)
    _, _, _, tot = dg.dolinc_diff_layout(M, sch, N)
    diff = torch.zeros(tot, dtype=torch.uint8, device="cuda")
    dg.dolinc_differentials(M, sch, to_dev(M, u), N, diff, ws)
    torch.cuda.synchronize()
    got = dg.diff_to_numpy(M, sch, diff, N)
    T, _ = O.differentials(u, N)
    for mm in range(1, N + 1):
        want = poly_coeffs(T[mm], m["dim"])
        g = got[mm - 1][:, M.perm, :]
        tol = (1e-12 * 4 ** mm) if prec == "fp64" else 1e-5 * 8 ** (mm - 1)
        assert rel(g, want) < tol, (mm, rel(g, want))


@pytest.mark.parametrize("k,r,nd", [(2, 1, 1), (3, 1, 1), (4, 1, 1), (3, 1, 2), (5, 2, 2), (6, 2, 2)])
@pytest.mark.parametrize("name", list(MESHES))
def test_face_states_fp64(k, r, nd, name):
    m, O = mesh(name)
    M = skew_mesh(m)
    u = field(m, 1, seed=2)
    sch = dg.Scheme(k=k, r=r, n_diff=nd, precision="fp64")
    ws = dg.workspace(M, sch)
    L = torch.zeros((1, M.n_faces), dtype=torch.float64, device="cuda")
    R = torch.zeros_like(L)
    dg.dolinc_reconstruct_faces(M, sch, to_dev(M, u), L, R, ws)
    wl, wr, _, _ = O.face_values(u, oracle.Scheme(k=k, r=r, n_diff=nd))
    tol = face_tol(O, "fp64", scheme_order(k, r), np.abs(u).max())
    assert np.all(np.abs(L.cpu().numpy()[0] - wl[0]) <= tol)
    assert np.all(np.abs(R.cpu().numpy()[0] - wr[0]) <= tol)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", range(len(RES_CASES)))
def test_residual(prec, case):
    name, nv, fx, (k, r, nd) = RES_CASES[case]
    if name not in MESHES:
        pytest.skip("mesh without skewness (strip)")
    m, O = mesh(name)
    M = skew_mesh(m)
    u = field(m, nv, seed=4 + case)
    sch = dg.Scheme(k=k, r=r, n_diff=nd, nv=nv, precision=prec, **fx)
    ws = dg.workspace(M, sch)
    Rg = torch.zeros((nv, M.n_cells), dtype=torch.float64, device="cuda")
    dg.dolinc_residual(M, sch, to_dev(M, u), Rg, ws)
    got = M.from_lib(Rg.cpu().numpy())
    want = O.residual(u, oracle.Scheme(k=k, r=r, n_diff=nd, nv=nv, **fx))
    Ns = scheme_order(k, r)
    lam = wave_speed(u, fx, m["dim"])
    base = {"fp64": 1e-12, "fp32": 1e-5}[prec]
    for v in range(nv):
        ct = cell_tol(O, face_tol(O, prec, Ns, np.abs(u).max()), lam) * (2.0 if nv > 1 else 1.0)
        assert np.all(np.abs(got[v] - want[v]) <= base * np.abs(want[v]).max() + ct), (v, rel(got[v], want[v]))
    if (O.neigh >= 0).all() and prec == "fp64":          # still conservative
        tot = (got * O.V).sum(axis=1)
        assert np.all(np.abs(tot) < 1e-13 * (np.abs(got) * O.V).sum(axis=1) + 1e-300)


@pytest.mark.parametrize("name", ["tri_bnd", "tet"])
def test_linear_fields_exact_at_face_centroids(name):
    """The corrected GPU scheme reproduces a linear field at the face centroids (both
    orientations) on skewed simplices, away from periodic seams and boundaries."""
    m, O = mesh(name)
    M = skew_mesh(m)
    D = m["dim"]
    a = np.array([0.7, -1.3, 0.4])[:D]
    u = (1.0 + O.xc[:, :D] @ a)[None]
    from test_oracle_pins import _far_from_seams
    ok = _far_from_seams(O, 3)
    nb = O.neigh >= 0
    fok = nb & ok[O.owner] & ok[np.maximum(O.neigh, 0)]
    assert fok.sum() > 20
    exact = 1.0 + O.xf[:, :D] @ a
    for k, r, nd in ((3, 1, 1), (4, 1, 1), (5, 2, 2)):
        sch = dg.Scheme(k=k, r=r, n_diff=nd, precision="fp64")
        ws = dg.workspace(M, sch)
        L = torch.zeros((1, M.n_faces), dtype=torch.float64, device="cuda")
        R = torch.zeros_like(L)
        dg.dolinc_reconstruct_faces(M, sch, to_dev(M, u), L, R, ws)
        assert np.abs(L.cpu().numpy()[0][fok] - exact[fok]).max() < 1e-11
        assert np.abs(R.cpu().numpy()[0][fok] - exact[fok]).max() < 1e-11


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_launch_shapes_bit_identical_and_step_matches_oracle(prec):
    m, O = mesh("tet")
    M = skew_mesh(m)
    u = field(m, 5, seed=60)
    sch = dg.Scheme(k=3, r=1, n_diff=2, nv=5, precision=prec, **euler_ok(5))
    ws = dg.workspace(M, sch)
    out = {}
    # the shapes whose sums run in the same order (one lane per cell: gather,
    # pipelined gather; the stage cell-centric, face-centric pair, pipelined) are
    # bit-identical; 4 lanes per cell sum in another order and are checked against
    # the oracle only
    for shape in ((1, 128, 1, 128), (1, 64, -2, 128), (-1, 128, -1, 128), (4, 128, 4, 64)):
        dg.dolinc_set_tuning(M, sch, *shape)
        x = to_dev(M, u)
        dg.dolinc_rk_step(M, sch, 1e-3, x, ws)
        dg.dolinc_sync_status(M, ws)
        out[shape] = x.cpu().numpy()
    vals = list(out.values())
    for v in vals[1:3]:
        assert np.array_equal(v, vals[0])
    want = O.rk3_step(u, oracle.Scheme(k=3, r=1, n_diff=2, nv=5, **euler_ok(5)), 1e-3)
    for v in (vals[0], vals[3]):
        got = M.from_lib(v)
        if prec == "fp64":
            assert rel(got - u, want - u) < 1e-11
        else:
            ok, worst = increment_ok(O, got - u, want - u, u, 1e-3, "fp32", 1, euler_ok(5), 3)
            assert ok, worst


def test_turning_the_correction_off_restores_the_plain_scheme():
    m, _ = mesh("tri")
    u = field(m, 1, seed=7)
    sch = dg.Scheme(k=3, r=1, n_diff=2, precision="fp64", flux="upwind", adv=(1.0, 0.6, 0.0))
    plain = dg.Mesh(m)
    M = skew_mesh(m)
    dg.dolinc_mesh_set_skew_correction(M, False)
    res = []
    for X in (plain, M):
        ws = dg.workspace(X, sch)
        R = torch.zeros((1, X.n_cells), dtype=torch.float64, device="cuda")
        dg.dolinc_residual(X, sch, to_dev(X, u), R, ws)
        res.append(R.cpu().numpy())
    assert np.array_equal(res[0], res[1])


def test_rejections():
    m = synth.tri_mesh(9, 9, 0.2, 3, boundary="transmissive")
    m["boundary_kind"] = np.where(np.asarray(m["face_neighbour"]) < 0, 2, 0).astype(np.int32)
    M = dg.Mesh(m)
    with pytest.raises(dg.DolincError) as e:
        dg.dolinc_mesh_set_skew_correction(M, True)
    assert e.value.status == 3
    S = skew_mesh(synth.tri_mesh(10, 10, 0.2, 4))
    with pytest.raises(dg.DolincError) as e:
        dg.Batch([S])
    assert e.value.status == 3
