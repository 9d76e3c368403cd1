"""Dirichlet and Neumann boundary faces (Sec 2.6) on the GPU against the oracle: the
first differential pass takes the boundary face value, the boundary face state is
that value, and everything downstream (higher differentials, interior faces next to
the wall, residual, full steps, every stage launch shape) follows."""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_parity import TOL, field, rel, to_dev

torch = pytest.importorskip("torch")
dg = pytest.importorskip("paper_2404_08952_gb300")
pytestmark = pytest.mark.gpu


def wall_channel(growth=1.3, ny=10, h0=0.02):
    ys = np.concatenate([[0.0], np.cumsum(h0 * growth ** np.arange(ny))])
    return synth.hex_mesh(np.linspace(0.0, 1.0, 8), ys, np.linspace(0.0, 0.6, 5), periodic=(True, False, True))


def with_kinds(m, pattern):
    """Boundary kinds 2 / 3 / 1 assigned to the boundary faces in turn."""
    m = dict(m)
    bnd = np.asarray(m["face_neighbour"]) < 0
    kinds = np.zeros(bnd.shape[0], dtype=np.int32)
    idx = np.nonzero(bnd)[0]
    kinds[idx] = np.asarray(pattern)[np.arange(idx.shape[0]) % len(pattern)]
    m["boundary_kind"] = kinds
    return m


def bc_values(m, nv, seed):
    rng = np.random.default_rng(seed)
    nf = np.asarray(m["face_owner"]).shape[0]
    v = 0.3 * rng.normal(size=(nv, nf))
    if nv > 1:                                   # Euler: positive density and energy on the faces
        v[0] = 1.0 + 0.1 * np.abs(v[0])
        v[-1] = 2.5 + 0.1 * np.abs(v[-1])
    return v


CASES = {
    "wall_hex": lambda: with_kinds(wall_channel(), [2, 3]),
    "tri_mixed": lambda: with_kinds(synth.tri_mesh(19, 13, 0.2, 12, boundary="transmissive"), [2, 3, 1]),
    "strip_dir": lambda: with_kinds(synth.strip_mesh(0.05 * 1.2 ** np.arange(17), height=0.05,
                                                     boundary="transmissive"), [2]),
}
_cache = {}


def case(name):
    if name not in _cache:
        m = CASES[name]()
        _cache[name] = (m, oracle.Oracle(m))
    return _cache[name]


def schemes(m, nv, bval, prec, **kw):
    fx = dict(flux="rusanov", gamma=1.4) if nv > 1 else dict(flux="upwind", adv=(1.0, -0.6, 0.3))
    o = oracle.Scheme(nv=nv, bkind=m["boundary_kind"], bval=bval, **fx, **kw)
    g = dg.Scheme(nv=nv, precision=prec, **fx, **kw)
    return o, g


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,nv", [("wall_hex", 1), ("wall_hex", 5), ("tri_mixed", 4), ("strip_dir", 1)])
def test_differentials_with_boundary_values(prec, name, nv):
    m, O = case(name)
    M = dg.Mesh(m)
    u = field(m, nv, seed=61)
    bval = bc_values(m, nv, 62)
    N = 3
    osch, sch = schemes(m, nv, bval, prec, k=3, r=1, n_diff=N)
    dg.dolinc_set_boundary_values(M, bval)
    ws = dg.workspace(M, sch)
    _, _, _, tot = dg.dolinc_diff_layout(M, sch, N)
    diff = torch.zeros(tot, dtype=torch.uint8, device="cuda")
    dg.dolinc_differentials(M, sch, to_dev(M, u), N, diff, ws)
    torch.cuda.synchronize()
    got = dg.diff_to_numpy(M, sch, diff, N)
    T, _ = O.differentials(u, N, scheme=osch)
    from test_gpu_parity import poly_coeffs
    for mm in range(1, N + 1):
        want = poly_coeffs(T[mm], m["dim"])
        g = got[mm - 1][:, M.perm, :]
        tol = TOL[prec] * (4 ** mm if prec == "fp64" else 8 ** (mm - 1))
        assert rel(g, want) < tol, (mm, rel(g, want))
    # zero-gradient treatment would differ at the boundary cells
    T0, _ = O.differentials(u, N)
    assert rel(poly_coeffs(T0[1], m["dim"]), poly_coeffs(T[1], m["dim"])) > 100 * TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,nv", [("wall_hex", 1), ("wall_hex", 5), ("tri_mixed", 4), ("strip_dir", 1)])
def test_face_states_and_residual_with_boundary_values(prec, name, nv):
    m, O = case(name)
    M = dg.Mesh(m)
    u = field(m, nv, seed=63)
    bval = bc_values(m, nv, 64)
    osch, sch = schemes(m, nv, bval, prec, k=3, r=1, n_diff=2)
    dg.dolinc_set_boundary_values(M, bval)
    ws = dg.workspace(M, sch)
    nf = O.n_faces
    fL = torch.zeros((nv, nf), dtype=torch.float64, device="cuda")
    fR = torch.zeros_like(fL)
    dg.dolinc_reconstruct_faces(M, sch, to_dev(M, u), fL, fR, ws)
    L, Rr, _, _ = O.face_values(u, osch)
    bnd = O.neigh < 0
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert rel(fL.cpu().numpy()[:, bnd], L[:, bnd]) < tol
    assert rel(fL.cpu().numpy(), L) < (1e-11 if prec == "fp64" else 1e-4)
    R = torch.zeros((nv, M.n_cells), dtype=torch.float64, device="cuda")
    dg.dolinc_residual(M, sch, to_dev(M, u), R, ws)
    got = M.from_lib(R.cpu().numpy())
    want = O.residual(u, osch)
    assert rel(got, want) < (1e-11 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("lanes,block", [(1, 128), (4, 64), (0, 128), (-1, 64), (-2, 128)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_steps_with_boundary_values_in_every_launch_shape(lanes, block, prec):
    m, O = case("wall_hex")
    M = dg.Mesh(m)
    u = field(m, 5, seed=65)
    bval = bc_values(m, 5, 66)
    osch, sch = schemes(m, 5, bval, prec, k=3, r=1, n_diff=2)
    dg.dolinc_set_boundary_values(M, bval)
    ws = dg.workspace(M, sch)
    dg.dolinc_set_tuning(M, sch, 1, 64, lanes, block)
    x = to_dev(M, u)
    dt = 2e-4
    for _ in range(2):
        dg.dolinc_rk_step(M, sch, dt, x, ws)
    dg.dolinc_sync_status(M, ws)
    got = M.from_lib(x.cpu().numpy())
    want = O.run(u, osch, dt, 2)
    assert rel(got - u, want - u) < (1e-10 if prec == "fp64" else 1e-4)


def test_linear_field_gradient_exact_with_exact_wall_data():
    """The Sec 2.6 rule in action on the GPU: with exact Dirichlet data a linear
    field's first differential is exact in every cell of a stretched wall mesh."""
    m = with_kinds(wall_channel(1.5), [2])
    O = oracle.Oracle(m)
    a = np.array([0.0, 2.3, 0.0])
    u = (1.0 + O.xc @ a)[None]
    bval = (1.0 + O.xf @ a)[None]
    M = dg.Mesh(m)
    dg.dolinc_set_boundary_values(M, bval)
    sch = dg.Scheme(k=3, r=1, n_diff=1, nv=1, precision="fp64", flux="upwind", adv=(1.0, 0.0, 0.0))
    ws = dg.workspace(M, sch)
    _, _, _, tot = dg.dolinc_diff_layout(M, sch, 1)
    diff = torch.zeros(tot, dtype=torch.uint8, device="cuda")
    dg.dolinc_differentials(M, sch, to_dev(M, u), 1, diff, ws)
    torch.cuda.synchronize()
    g = dg.diff_to_numpy(M, sch, diff, 1)[0][0]
    assert np.abs(g - a[None, :]).max() < 1e-11


def test_boundary_values_are_required_and_checked():
    m, _ = case("wall_hex")
    M = dg.Mesh(m)
    sch = dg.Scheme(k=3, r=1, n_diff=2, nv=1, precision="fp64", flux="upwind", adv=(1.0, 0.0, 0.0))
    ws = dg.workspace(M, sch)
    R = torch.zeros((1, M.n_cells), dtype=torch.float64, device="cuda")
    u = torch.ones((1, M.n_cells), dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DolincError) as e:
        dg.dolinc_residual(M, sch, u, R, ws)
    assert e.value.status == 1
    dg.dolinc_set_boundary_values(M, np.zeros((2, O_faces(m))))
    with pytest.raises(dg.DolincError):
        dg.dolinc_residual(M, sch, u, R, ws)                  # values set for nv = 2, scheme has 1
    with pytest.raises(dg.DolincError):
        dg.dolinc_set_boundary_values(M, np.full((1, O_faces(m)), np.nan))
    dg.dolinc_set_boundary_values(M, np.zeros((1, O_faces(m))))
    dg.dolinc_residual(M, sch, u, R, ws)
    dg.dolinc_sync_status(M, ws)


def O_faces(m):
    return np.asarray(m["face_owner"]).shape[0]


def test_blasius_single_step_reconstruction():
    """The paper's boundary-layer case with this library's Blasius data: cell averages
    of the Blasius velocity on a wall mesh growing by 1.3, Dirichlet wall and top; the
    GPU's face values equal the oracle's, and CSR4 reconstructs the wall-parallel
    faces more accurately than USR3."""
    import bench
    from synth import fields
    m = bench.bl_mesh(1.3)
    O = oracle.Oracle(m)
    bnd = O.neigh < 0
    cap = bnd & ((np.abs(O.xf[:, 1]) < 1e-12) | (O.xf[:, 1] > 0.29))
    m["boundary_kind"] = np.where(cap, 2, np.where(bnd, 1, 0)).astype(np.int32)
    ex = fields.blasius(O.xf)
    u0 = synth.cell_average(m, fields.blasius, q=4, nv=2)
    rows = (~bnd) & (np.abs(O.S[:, 1]) > 0.5 * np.linalg.norm(O.S, axis=1))
    M = dg.Mesh(m)
    err = {}
    for k in (3, 4):
        bval = np.where(cap, np.where(np.abs(O.xf[:, 1]) < 1e-12, 0.0, ex[:, 0]), 0.0)[None]
        dg.dolinc_set_boundary_values(M, bval)
        sch = dg.Scheme(k=k, r=1, n_diff=1, nv=1, precision="fp64", flux="upwind", adv=(1.0, 0.0, 0.0))
        ws = dg.workspace(M, sch)
        fL = torch.zeros((1, O.n_faces), dtype=torch.float64, device="cuda")
        fR = torch.zeros_like(fL)
        dg.dolinc_reconstruct_faces(M, sch, to_dev(M, u0[:1]), fL, fR, ws)
        osch = oracle.Scheme(k=k, r=1, n_diff=1, flux="upwind", adv=(1.0, 0.0, 0.0), bkind=m["boundary_kind"],
                             bval=bval)
        OL, OR, _, _ = O.face_values(u0[:1], osch)
        assert rel(fL.cpu().numpy(), OL) < 1e-11 and rel(fR.cpu().numpy(), OR) < 1e-11
        e = fL.cpu().numpy()[0][rows] - ex[rows, 0]
        err[k] = np.sqrt(np.mean(e ** 2))
    assert err[4] < 0.7 * err[3] and err[3] < 5e-3
