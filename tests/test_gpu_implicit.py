"""The semi-implicit DOLINC step on the GPU (dolinc_implicit_*) against the oracle's
direct solve of the same equations (Sec 2.4: weight part implicit, c_r explicit):
the assembled rows entry by entry, one step and several outer iterations element by
element, theta = 0 against the explicit forward Euler step, the FP32-residual path
through the solve's defining equation, a full-size mesh through the same equation,
determinism, the bounded barrier's report, and the rejections."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
dg = pytest.importorskip("paper_2404_08952_gb300")
sp = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu

from test_gpu_parity import field, to_dev  # noqa: E402

MESHES = {
    "tri": (lambda: synth.tri_mesh(24, 20, 0.2, 3), (1.0, 0.6, 0.0)),
    "tri_bnd": (lambda: synth.tri_mesh(23, 17, 0.2, 5, boundary="transmissive"), (0.8, -0.5, 0.0)),
    "tet": (lambda: synth.tet_mesh(6, 0.15, 2), (0.7, -0.5, 0.4)),
    "hexprism": (lambda: synth.hexprism_mesh(7, 0.2, 4), (1.0, 1.0, 1.0)),
}
_cache = {}
LIMITER_ENO = {"none": 0, "weno5_all": 4}
# Courant numbers (|a| dt / h_min) of the tests: USR3's weight part is dissipative on
# every mesh, so its rows stay definite at any dt; CSR4's and USR5's are not on jittered
# meshes (their V/dt + theta K turns indefinite above Courant numbers of about 0.6 and
# 1.2 on the tetrahedra), so they are tested below that.
CFL = {(3, 1): 3.0, (4, 1): 0.4, (5, 2): 0.8}


def mesh(name, skew=False):
    key = (name, skew)
    if key not in _cache:
        m = MESHES[name][0]()
        _cache[key] = (m, oracle.Oracle(m, skew=skew))
    return _cache[key]


def schemes(k, r, adv, prec="fp64", limiter="none"):
    return (dg.Scheme(k=k, r=r, flux="upwind", nv=1, precision=prec, limiter=limiter, adv=adv),
            oracle.Scheme(k=k, r=r, flux="upwind", nv=1, adv=adv, eno=LIMITER_ENO[limiter]))


def cfl_dt(O, adv, cfl):
    h = (O.V.min()) ** (1.0 / O.dim)
    return cfl * h / np.linalg.norm(adv)


def lib_matrix(M, solver):
    ro, nb, off, dg_ = solver.rows()
    n = M.n_cells
    rows = np.repeat(np.arange(n), np.diff(ro))
    A = sp.csr_matrix((off, (rows, nb)), shape=(n, n)) + sp.diags(dg_)
    return A[M.perm, :][:, M.perm]          # caller order


def oracle_matrix(O, so, dt, theta):
    return (sp.diags(O.V / dt) + theta * O.implicit_operator(so)).tocsr()


@pytest.mark.parametrize("theta", [1.0, 0.5])
@pytest.mark.parametrize("k,r", [(3, 1), (4, 1), (5, 2)])
@pytest.mark.parametrize("name", ["tri", "tri_bnd", "tet", "hexprism"])
def test_rows_equal_the_oracle_matrix(name, k, r, theta):
    m, O = mesh(name)
    adv = MESHES[name][1]
    M = dg.Mesh(m)
    sd, so = schemes(k, r, adv)
    dt = cfl_dt(O, adv, CFL[(k, r)])
    S = dg.Implicit(M, sd, dt, theta)
    got = lib_matrix(M, S)
    want = oracle_matrix(O, so, dt, theta)
    d = abs(got - want)
    assert d.max() <= 1e-12 * abs(want).max(), d.max()


def _step_case(name, k, r, theta, n_outer, skew=False, limiter="none", cfl=None, tol=1e-13):
    m, O = mesh(name, skew)
    adv = MESHES[name][1]
    M = dg.Mesh(m)
    if skew:
        dg.dolinc_mesh_set_skew_correction(M, True)
    sd, so = schemes(k, r, adv, limiter=limiter)
    dt = cfl_dt(O, adv, CFL[(k, r)] if cfl is None else cfl)
    S = dg.Implicit(M, sd, dt, theta)
    S.set_solver(rel_tol=tol, max_iter=2000)
    ws = dg.workspace(M, sd)
    u = field(m, 1, seed=7)
    ud = to_dev(M, u)
    S.step(ud, ws, n_outer)
    info = S.info()
    got = M.from_lib(ud.cpu().numpy())
    want = O.semi_implicit_step(u, so, dt, theta, n_outer)
    return got, want, u, info


@pytest.mark.parametrize("theta", [1.0, 0.5])
@pytest.mark.parametrize("k,r", [(3, 1), (4, 1), (5, 2)])
@pytest.mark.parametrize("name", ["tri", "tri_bnd", "tet", "hexprism"])
def test_step_equals_the_oracle(name, k, r, theta):
    got, want, u, info = _step_case(name, k, r, theta, 1)
    assert info["converged"] and info["solves"] == 1 and info["rel_residual"] <= 1e-13, info
    # BiCGSTAB to 1e-13 on rows of condition number O(CFL): the step's increment to ~1e-11
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want - u).max(), np.abs(got - want).max()


@pytest.mark.parametrize("name", ["tri", "tet"])
def test_outer_iterations_equal_the_oracle(name):
    got, want, u, info = _step_case(name, 3, 1, 0.5, 4)
    assert info["solves"] == 4 and info["converged"], info
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want - u).max()


@pytest.mark.parametrize("name", ["tri", "tet", "hexprism"])
def test_skew_corrected_step_equals_the_oracle(name):
    got, want, u, info = _step_case(name, 3, 1, 1.0, 1, skew=True)
    assert info["converged"]
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want - u).max()


def test_weno5_limited_step_equals_the_oracle():
    got, want, u, info = _step_case("tri", 5, 2, 1.0, 2, limiter="weno5_all", cfl=3.0)
    assert info["converged"]
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want - u).max()


@pytest.mark.parametrize("name", ["tri_bnd", "tet"])
def test_theta_zero_is_forward_euler(name):
    """theta = 0: the rows are diagonal, one iteration gives delta = dt R exactly up to
    the rounding of V / (V/dt)."""
    m, O = mesh(name)
    adv = MESHES[name][1]
    M = dg.Mesh(m)
    sd, _ = schemes(3, 1, adv)
    dt = cfl_dt(O, adv, 0.3)
    S = dg.Implicit(M, sd, dt, 0.0)
    ws = dg.workspace(M, sd)
    u = to_dev(M, field(m, 1, seed=3))
    R = torch.zeros_like(u)
    dg.dolinc_residual(M, sd, u, R, ws)
    want = u + dt * R
    S.step(u, ws)
    info = S.info()
    assert info["iterations"] == 1 and info["converged"]
    assert (u - want).abs().max().item() <= 4e-16 * dt * R.abs().max().item() + 4e-16 * want.abs().max().item()


@pytest.mark.parametrize("prec,k,r", [("fp32", 3, 1), ("fp32_bf16", 5, 2)])
def test_fp32_residual_path_solves_its_equation(prec, k, r):
    """FP32 bulk residual R32 (the stage path's own, checked against the oracle by the
    stage parity tests): the step solves (V/dt + theta K) delta = V R32 with the
    oracle's K to the solver tolerance, and stays near the FP64 oracle step."""
    name = "tet"
    m, O = mesh(name)
    adv = MESHES[name][1]
    M = dg.Mesh(m)
    sd, so = schemes(k, r, adv, prec=prec)
    dt = cfl_dt(O, adv, CFL[(k, r)])
    S = dg.Implicit(M, sd, dt, 1.0)
    S.set_solver(rel_tol=1e-12)
    ws = dg.workspace(M, sd)
    u = field(m, 1, seed=5)
    ud = to_dev(M, u)
    R = torch.zeros_like(ud)
    dg.dolinc_residual(M, sd, ud, R, ws)
    S.step(ud, ws)
    assert S.info()["converged"]
    delta = M.from_lib(ud.cpu().numpy())[0] - u[0]
    R32 = M.from_lib(R.cpu().numpy())[0]
    A = oracle_matrix(O, so, dt, 1.0)
    b = O.V * R32
    assert np.abs(A @ delta - b).max() <= 1e-10 * np.abs(b).max()
    want = O.semi_implicit_step(u, so, dt, 1.0)[0] - u[0]
    assert np.abs(delta - want).max() <= 1e-3 * np.abs(want).max()


def test_full_size_hexprism_solves_its_equation():
    """The bench's mesh size (hexes and prisms, 140^3 lattice, 4.12M cells): the step's
    increment satisfies the oracle's equation (V/dt + theta K) delta = V R(u) with the
    oracle's K and FP64 residual, row by row."""
    m = synth.hexprism_mesh(140, 0.2, 31)
    O = oracle.Oracle(m, parallel=True)
    adv = (1.0, 1.0, 1.0)
    M = dg.Mesh(m, renumber="morton")
    sd, so = schemes(3, 1, adv)
    dt = cfl_dt(O, adv, 4.0)
    S = dg.Implicit(M, sd, dt, 1.0)
    S.set_solver(rel_tol=1e-12)
    ws = dg.workspace(M, sd)
    rng = np.random.default_rng(2)
    xc = O.xc
    u = (np.sin(2 * np.pi * xc[:, 0]) * np.cos(2 * np.pi * xc[:, 1]) + 0.3 * np.sin(2 * np.pi * xc[:, 2])
         + 1e-3 * rng.standard_normal(O.n_cells))[None, :]
    ud = to_dev(M, u)
    S.step(ud, ws)
    info = S.info()
    assert info["converged"], info
    delta = M.from_lib(ud.cpu().numpy())[0] - u[0]
    b = O.V * O.residual(u, so)[0]
    A = oracle_matrix(O, so, dt, 1.0)
    assert np.abs(A @ delta - b).max() <= 1e-9 * np.abs(b).max()


def test_steps_are_deterministic():
    m, O = mesh("tet")
    adv = MESHES["tet"][1]
    M = dg.Mesh(m)
    sd, _ = schemes(3, 1, adv)
    S = dg.Implicit(M, sd, cfl_dt(O, adv, 3.0), 1.0)
    ws = dg.workspace(M, sd)
    u0 = to_dev(M, field(m, 1, seed=8))
    a, b = u0.clone(), u0.clone()
    for _ in range(3):
        S.step(a, ws)
    for _ in range(3):
        S.step(b, ws)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_barrier_timeout_is_reported_then_recovers():
    """A grid-barrier wait that gives up (spin limit 0: every wait gives up at its first
    poll) ends the solve in every block and is reported; the next step with the normal
    limit runs."""
    m = synth.tri_mesh(160, 160, 0.2, 9)              # 51,200 cells: 200 blocks
    O = oracle.Oracle(m)
    adv = (1.0, 0.6, 0.0)
    M = dg.Mesh(m)
    sd, so = schemes(3, 1, adv)
    dt = cfl_dt(O, adv, 2.0)
    S = dg.Implicit(M, sd, dt, 1.0)
    ws = dg.workspace(M, sd)
    u = field(m, 1, seed=4)
    ud = to_dev(M, u)
    S.set_solver(spin_limit=0)
    S.step(ud, ws)
    with pytest.raises(dg.DolincError) as e:
        S.info()
    assert e.value.status == 5
    S.set_solver(rel_tol=1e-13)
    ud = to_dev(M, u)
    S.step(ud, ws)
    assert S.info()["converged"]
    want = O.semi_implicit_step(u, so, dt, 1.0)
    got = M.from_lib(ud.cpu().numpy())
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want - u).max()


def test_rejections():
    m, O = mesh("tri")
    M = dg.Mesh(m)
    sd, _ = schemes(3, 1, (1.0, 0.5, 0.0))
    with pytest.raises(dg.DolincError) as e:
        dg.Implicit(M, dg.Scheme(k=3, r=1, flux="rusanov", nv=4), 0.1)
    assert e.value.status == 3
    with pytest.raises(dg.DolincError) as e:
        dg.Implicit(M, dg.Scheme(k=3, r=1, flux="burgers", nv=1), 0.1)
    assert e.value.status == 3
    for dt, th in ((0.0, 1.0), (-1.0, 1.0), (0.1, 1.5), (0.1, -0.1), (float("inf"), 1.0)):
        with pytest.raises(dg.DolincError) as e:
            dg.Implicit(M, sd, dt, th)
        assert e.value.status == 1
    S = dg.Implicit(M, sd, 0.1)
    ws = dg.workspace(M, sd)
    u = to_dev(M, field(m, 1, seed=1))
    with pytest.raises(dg.DolincError) as e:
        S.step(u, ws, n_outer=0)
    assert e.value.status == 1
    with pytest.raises(dg.DolincError) as e:
        S.set_solver(max_iter=0)
    assert e.value.status == 1
    mb = synth.tri_mesh(9, 7, 0.1, 2, boundary="transmissive")
    bk = np.where(np.asarray(mb["face_neighbour"]) < 0, 2, 0).astype(np.int32)
    mb = dict(mb, boundary_kind=bk)
    Mb = dg.Mesh(mb)
    dg.dolinc_set_boundary_values(Mb, np.zeros((1, bk.shape[0])))
    with pytest.raises(dg.DolincError) as e:
        dg.Implicit(Mb, sd, 0.1)
    assert e.value.status == 3


@pytest.mark.parametrize("name", ["tet", "hexprism"])
def test_warm_started_steps_equal_the_oracle(name):
    """Warm start (the step's first solve from the last step's solution, 1, or from its
    linear extrapolation from the last two steps, 2): every step equals the oracle's
    step from the same state; the first step starts from 0 in every mode, and the
    second uses the one kept solution in modes 1 and 2 alike.  (Whether later steps
    need fewer iterations depends on how the increment moves between steps, so it is
    measured by the benchmark, not asserted here.)"""
    m, O = mesh(name)
    adv = MESHES[name][1]
    M = dg.Mesh(m)
    sd, so = schemes(3, 1, adv)
    dt = cfl_dt(O, adv, 3.0)
    ws = dg.workspace(M, sd)
    its, res = {}, {}
    for warm in (0, 1, 2):
        S = dg.Implicit(M, sd, dt, 1.0)
        S.set_solver(rel_tol=1e-13, warm_start=warm)
        u = field(m, 1, seed=6)
        ud = to_dev(M, u)
        its[warm], res[warm] = [], []
        for _ in range(4):
            S.step(ud, ws)
            info = S.info()
            assert info["converged"], info
            its[warm].append(info["iterations"])
            got = M.from_lib(ud.cpu().numpy())
            res[warm].append(got)
            want = O.semi_implicit_step(u, so, dt, 1.0)
            assert np.abs(got - want).max() <= 1e-10 * np.abs(want - u).max()
            u = got
    assert its[1][0] == its[0][0] == its[2][0]
    assert its[2][1] == its[1][1] and np.array_equal(res[2][1], res[1][1])
    with pytest.raises(dg.DolincError) as e:
        S.set_solver(warm_start=3)
    assert e.value.status == 1


@pytest.mark.parametrize("name,narrowest", [("tri", 4), ("tet", 4), ("hexprism", 6)])
def test_row_layouts_give_the_same_step(name, narrowest):
    """Rows in ELL form of every width that covers the mesh and per face slot: the same
    rows, the same step (the per-cell sums keep their order; the grid, and so the order
    of the dot products, may differ), each equal to the oracle's."""
    m, O = mesh(name)
    adv = MESHES[name][1]
    M = dg.Mesh(m)
    sd, so = schemes(3, 1, adv)
    dt = cfl_dt(O, adv, 3.0)
    S = dg.Implicit(M, sd, dt, 1.0)
    S.set_solver(rel_tol=1e-13)
    assert S.layout == 0
    ws = dg.workspace(M, sd)
    u = field(m, 1, seed=12)
    want = O.semi_implicit_step(u, so, dt, 1.0)
    ref = lib_matrix(M, S)
    got = {}
    for ell in [w for w in (4, 6, 8) if w >= narrowest] + [0]:
        S.set_layout(ell)
        assert S.layout == ell
        assert abs(lib_matrix(M, S) - ref).max() == 0.0
        ud = to_dev(M, u)
        S.step(ud, ws)
        assert S.info()["converged"]
        got[ell] = M.from_lib(ud.cpu().numpy())
        assert np.abs(got[ell] - want).max() <= 1e-10 * np.abs(want - u).max()
    for bad in (3, 5, 12) + ((4,) if narrowest > 4 else ()):
        with pytest.raises(dg.DolincError) as e:
            S.set_layout(bad)
        assert e.value.status == 1
