"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle, element
by element on the same seeded inputs.

Tolerances are derived from the arithmetic of the inversion.  A face value is
sum_m W0[m] phi_0^(m) + W1[m] phi_1^(m) over the scheme's DOLINC order Ns; phi^(m)
carries the rounding of m nested Gauss sums (about eps * 24^m of the field on these
meshes) and the weights W the rounding of the far-field recursion, which grows with
the face's growth-rate spread G = max(g, 1/g) like G^(Ns(Ns-1)) (checked against
50-digit arithmetic).  Per face:
  FP64       1e-12 * 4^Ns     * G^(Ns(Ns-1)) * max|u|
  FP32       1e-5  * 8^(Ns-1) * G^(Ns(Ns-1)) * max|u|      (Ns = 1: the stated 1e-5)
  FP32+BF16  3e-3 (8-bit mantissa on orders >= 2; coarse test meshes)
Residuals take the same per-face bound through |S_f| * (largest wave speed) / V_c
(for FP32 that is 1e-5 relative to the face-flux magnitudes, not to the residual,
which is their O(h) cancellation);
differentials of order m are compared with 1e-12 * 4^m (FP64) / 1e-5 * 8^(m-1) (FP32).
"""
import numpy as np
import pytest

import oracle
import synth
from _tol import cell_tol, face_tol, increment_ok, wave_speed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

dg = pytest.importorskip("paper_2404_08952_gb300")


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp32_bf16": 1e-5}

MESHES = {
    "tri": lambda: synth.tri_mesh(21, 17, 0.2, 11),                       # 714 cells, ragged tail
    "tri_bnd": lambda: synth.tri_mesh(19, 13, 0.2, 12, boundary="transmissive"),
    "tet": lambda: synth.tet_mesh(6, 0.15, 13),                           # 1080 cells
    "hexprism": lambda: synth.hexprism_mesh(7, 0.2, 14),
    "strip": lambda: synth.strip_mesh(0.05 * 1.1 ** np.arange(23), height=0.05, boundary="transmissive"),
}
_cache = {}


def mesh(name):
    if name not in _cache:
        m = MESHES[name]()
        _cache[name] = (m, oracle.Oracle(m))
    return _cache[name]


def field(m, nv, seed=0):
    """Smooth seeded data: a few random Fourier modes per variable (positive density
    and pressure for Euler)."""
    rng = np.random.default_rng(seed)
    dim = m["dim"]

    def f(p):
        out = []
        for v in range(nv):
            k = rng.integers(1, 3, size=(3, dim))
            ph = rng.uniform(0, 6.28, size=3)
            a = rng.uniform(-0.3, 0.3, size=3)
            out.append(sum(a[i] * np.sin(2 * np.pi * p @ k[i] + ph[i]) for i in range(3)))
        return np.stack(out, axis=1)
    u = synth.cell_average(m, f, q=3, nv=nv)
    if nv > 1:          # Euler: rho ~ 1, momentum ~ 0.3, E ~ 2.5
        u[0] += 1.0
        u[-1] += 2.5
    return u


def gpu_mesh(m, renumber="morton"):
    return dg.Mesh(m, renumber=renumber)


def to_dev(M, u):
    return torch.from_numpy(M.to_lib(np.ascontiguousarray(u))).cuda()


def euler_ok(nv):
    return dict(flux="rusanov", gamma=1.4)


def scheme_order(k, r):
    return max(r, k - r - 2, 1)


# ---------------------------------------------------------------------------- geometry

@pytest.mark.parametrize("name", list(MESHES))
def test_geometry(name):
    m, O = mesh(name)
    M = gpu_mesh(m)
    g = M.geometry()
    np.testing.assert_allclose(g["V"][M.perm], O.V, rtol=1e-12)
    np.testing.assert_allclose(g["xc"][M.perm], O.xc, atol=1e-13)
    np.testing.assert_allclose(g["S"], O.S, atol=1e-14)
    inner = O.neigh >= 0
    np.testing.assert_allclose(g["w"][inner], O.w[inner], atol=1e-13)
    np.testing.assert_allclose(g["d"][inner], O.d[inner], atol=1e-13)


# ---------------------------------------------------------------------------- differentials

def poly_coeffs(T, dim):
    """Full tensor [nv, nc, dim^m] -> polynomial coefficients [nv, nc, C_m]."""
    m = int(round(np.log(T.shape[2]) / np.log(dim))) if T.shape[2] > 1 else 0
    C = m + 1 if dim == 2 else (m + 1) * (m + 2) // 2
    out = np.zeros(T.shape[:2] + (C,))
    for a in range(dim ** m):
        digits, t = [], a
        for _ in range(m):
            digits.append(t % dim)
            t //= dim
        if dim == 2:
            q = digits.count(1)
        else:
            b, c = digits.count(1), digits.count(2)
            tt = b + c
            q = tt * (tt + 1) // 2 + c
        out[:, :, q] += T[:, :, a]
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,nv", [("tri", 1), ("tri", 4), ("tet", 1), ("tet", 5), ("hexprism", 1),
                                     ("tri_bnd", 4), ("strip", 1)])
def test_differentials(prec, name, nv):
    m, O = mesh(name)
    M = gpu_mesh(m)
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
        tol = TOL[prec] * (4 ** mm if prec == "fp64" else 8 ** (mm - 1))
        assert rel(g, want) < tol, (mm, rel(g, want))


# ---------------------------------------------------------------------------- face states

SCHEMES = [(2, 1, 1), (3, 1, 1), (4, 1, 1), (3, 1, 2), (5, 2, 2), (6, 2, 2), (4, 1, 3), (7, 3, 3), (9, 4, 4)]


@pytest.mark.parametrize("k,r,nd", SCHEMES)
@pytest.mark.parametrize("name", ["tri", "tet", "hexprism", "strip", "tri_bnd"])
def test_face_states_fp64(k, r, nd, name):
    m, O = mesh(name)
    M = gpu_mesh(m)
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
    if scheme_order(k, r) == 1:          # well-conditioned: the plain 1e-12 bar
        assert rel(L.cpu().numpy(), wl) < 1e-12 and rel(R.cpu().numpy(), wr) < 1e-12


@pytest.mark.parametrize("prec", ["fp32", "fp32_bf16"])
@pytest.mark.parametrize("k,r,nd", [(3, 1, 2), (4, 1, 3), (5, 2, 2)])
@pytest.mark.parametrize("name,nv", [("tri", 1), ("tet", 5), ("hexprism", 1)])
def test_face_states_reduced_precision(prec, k, r, nd, name, nv):
    m, O = mesh(name)
    M = gpu_mesh(m)
    u = field(m, nv, seed=3)
    sch = dg.Scheme(k=k, r=r, n_diff=nd, nv=nv, precision=prec, **(euler_ok(nv) if nv > 1 else {}))
    ws = dg.workspace(M, sch)
    L = torch.zeros((nv, M.n_faces), dtype=torch.float64, device="cuda")
    R = torch.zeros_like(L)
    dg.dolinc_reconstruct_faces(M, sch, to_dev(M, u), L, R, ws)
    wl, wr, _, _ = O.face_values(u, oracle.Scheme(k=k, r=r, n_diff=nd, nv=nv))
    for v in range(nv):
        tol = face_tol(O, prec, scheme_order(k, r), np.abs(u[v]).max())
        assert np.all(np.abs(L.cpu().numpy()[v] - wl[v]) <= tol)
        assert np.all(np.abs(R.cpu().numpy()[v] - wr[v]) <= tol)
    if prec == "fp32" and scheme_order(k, r) == 1:
        for v in range(nv):
            assert rel(L.cpu().numpy()[v], wl[v]) < 1e-5 and rel(R.cpu().numpy()[v], wr[v]) < 1e-5


# ---------------------------------------------------------------------------- residual / stages

RES_CASES = [
    ("tri", 1, dict(flux="upwind", adv=(1.0, 0.6, 0.0)), (3, 1, 2)),
    ("tri", 1, dict(flux="burgers"), (3, 1, 2)),
    ("tri_bnd", 4, euler_ok(4), (3, 1, 2)),
    ("tri", 4, euler_ok(4), (4, 1, 1)),
    ("tet", 1, dict(flux="upwind", adv=(-0.4, 1.0, 0.7)), (5, 2, 2)),
    ("tet", 5, euler_ok(5), (4, 1, 3)),
    ("tet", 5, euler_ok(5), (2, 1, 1)),
    ("hexprism", 1, dict(flux="upwind", adv=(1.0, 1.0, 1.0)), (5, 2, 4)),
    ("strip", 1, dict(flux="burgers"), (6, 2, 2)),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_bf16"])
@pytest.mark.parametrize("case", range(len(RES_CASES)))
def test_residual(prec, case):
    name, nv, fx, (k, r, nd) = RES_CASES[case]
    m, O = mesh(name)
    M = gpu_mesh(m)
    u = field(m, nv, seed=4 + case)
    sch = dg.Scheme(k=k, r=r, n_diff=nd, nv=nv, precision=prec, **fx)
    ws = dg.workspace(M, sch)
    Rg = torch.zeros((nv, M.n_cells), dtype=torch.float64, device="cuda")
    dg.dolinc_residual(M, sch, to_dev(M, u), Rg, ws)
    got = M.from_lib(Rg.cpu().numpy())
    want = O.residual(u, oracle.Scheme(k=k, r=r, n_diff=nd, nv=nv, **fx))
    Ns = scheme_order(k, r)
    lam = wave_speed(u, fx, m["dim"])
    base = {"fp64": 1e-12, "fp32": 1e-5, "fp32_bf16": 3e-3}[prec]
    for v in range(nv):
        ct = cell_tol(O, face_tol(O, prec, Ns, np.abs(u).max()), lam) * (2.0 if nv > 1 else 1.0)
        assert np.all(np.abs(got[v] - want[v]) <= base * np.abs(want[v]).max() + ct), (v, rel(got[v], want[v]))
    if Ns == 1 and prec == "fp64":
        for v in range(nv):
            assert rel(got[v], want[v]) < base, (v, rel(got[v], want[v]))
    # conservation: the face fluxes cancel pairwise on periodic meshes, on the GPU too
    if (O.neigh >= 0).all() and prec == "fp64":
        tot = (got * O.V).sum(axis=1)
        assert np.all(np.abs(tot) < 1e-13 * (np.abs(got) * O.V).sum(axis=1) + 1e-300)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("stage", [0, 1, 2])
def test_rk_stage(prec, stage):
    m, O = mesh("tet")
    M = gpu_mesh(m)
    u0 = field(m, 5, seed=20)
    us = u0 * 1.01 + 0.001
    sch = dg.Scheme(k=4, r=1, n_diff=3, precision=prec, nv=5, **euler_ok(5))
    ws = dg.workspace(M, sch)
    out = torch.zeros((5, M.n_cells), dtype=torch.float64, device="cuda")
    dt = 1e-3
    dg.dolinc_rk_stage(M, sch, dt, stage, to_dev(M, u0), to_dev(M, us), out, ws)
    got = M.from_lib(out.cpu().numpy())
    want = O.rk3_stage(u0, us, oracle.Scheme(k=4, r=1, n_diff=3, nv=5, **euler_ok(5)), dt, stage)
    # compare the increment over the FP64 affine part, the part the FP32 path computes
    base = np.array([0.0, 0.75, 1 / 3])[stage] * u0 + np.array([1.0, 0.25, 2 / 3])[stage] * us
    assert rel(got - base, want - base) < (1e-11 if prec == "fp64" else 1e-5)


def test_c1_workload_100_steps_fp64():
    """adv2d_tri64 at half resolution, 100 full SSP-RK3 steps through dolinc_rk_step."""
    w = synth.workload("adv2d_tri64", size=32)
    m = w["mesh"]
    O = oracle.Oracle(m)
    M = gpu_mesh(m)
    sch = dg.Scheme(precision="fp64", **w["scheme"])
    ws = dg.workspace(M, sch)
    u = to_dev(M, w["u0"])
    for _ in range(w["steps"]):
        dg.dolinc_rk_step(M, sch, w["dt"], u, ws)
    dg.dolinc_sync_status(M, ws)
    got = M.from_lib(u.cpu().numpy())
    want = O.run(w["u0"], oracle.Scheme(**w["scheme"]), w["dt"], w["steps"])
    assert rel(got, want) < 1e-10


@pytest.mark.parametrize("prec", ["fp32", "fp32_bf16"])
def test_c1_workload_100_steps_below_fp64(prec):
    """The same 100 steps in the increment form of the step (bulk precision below FP64,
    one FP64 add per step): each stage's increment carries the bulk precision's
    relative rounding (~1e-7 in FP32), which 300 stages accumulate to a few 1e-6 of the
    field.  USR3 reads orders <= 1, so BF16 storage of order 2 does not reach the faces."""
    w = synth.workload("adv2d_tri64", size=32)
    m = w["mesh"]
    O = oracle.Oracle(m)
    M = gpu_mesh(m)
    sch = dg.Scheme(precision=prec, **w["scheme"])
    ws = dg.workspace(M, sch)
    u = to_dev(M, w["u0"])
    for _ in range(w["steps"]):
        dg.dolinc_rk_step(M, sch, w["dt"], u, ws)
    dg.dolinc_sync_status(M, ws)
    got = M.from_lib(u.cpu().numpy())
    want = O.run(w["u0"], oracle.Scheme(**w["scheme"]), w["dt"], w["steps"])
    assert rel(got, want) < 2e-5


@pytest.mark.parametrize("renumber", ["none", "morton"])
def test_renumbering_does_not_change_results(renumber):
    m, O = mesh("tet")
    M = gpu_mesh(m, renumber=renumber)
    u = field(m, 5, seed=9)
    sch = dg.Scheme(k=3, r=1, n_diff=2, precision="fp64", nv=5, **euler_ok(5))
    ws = dg.workspace(M, sch)
    dt = 2e-3
    x = to_dev(M, u)
    dg.dolinc_rk_step(M, sch, dt, x, ws)
    want = O.rk3_step(u, oracle.Scheme(k=3, r=1, n_diff=2, nv=5, **euler_ok(5)), dt)
    assert rel(M.from_lib(x.cpu().numpy()), want) < 1e-12


# ---------------------------------------------------------------------------- ENO3 limiter

@pytest.mark.parametrize("mode", ["eno3_all", "eno3_flagged", "first_order_flagged", "weno5_all", "weno5_flagged"])
@pytest.mark.parametrize("name,nv", [("tri", 1), ("tri_bnd", 4), ("tet", 5)])
def test_eno3_limiter_fp64(mode, name, nv):
    m, O = mesh(name)
    M = gpu_mesh(m)
    u = field(m, nv, seed=30)
    rng = np.random.default_rng(31)
    flags = (rng.uniform(size=O.n_cells) < 0.3).astype(np.uint8)
    fx = euler_ok(nv) if nv > 1 else dict(flux="burgers")
    sch = dg.Scheme(k=3, r=1, n_diff=2, nv=nv, precision="fp64", limiter=mode, **fx)
    fl_dev = torch.from_numpy(M.to_lib(flags)).cuda()
    dg.dolinc_set_flags(M, fl_dev)
    ws = dg.workspace(M, sch)
    Rg = torch.zeros((nv, M.n_cells), dtype=torch.float64, device="cuda")
    dg.dolinc_residual(M, sch, to_dev(M, u), Rg, ws)
    got = M.from_lib(Rg.cpu().numpy())
    eno = {"eno3_all": 1, "eno3_flagged": 2, "first_order_flagged": 3, "weno5_all": 4, "weno5_flagged": 5}[mode]
    osch = oracle.Scheme(k=3, r=1, n_diff=2, nv=nv, eno=eno, troubled=flags if eno in (2, 3, 5) else None, **fx)
    want = O.residual(u, osch)
    # stencil choices are taken in FP64 on both sides; smooth random data has no ties.
    # WENO5 combines values built from second-order differentials (N_s = 2): the
    # FP64 bound 1e-12 * 4^N_s of the tolerance rule
    assert rel(got, want) < (1.6e-11 if eno in (4, 5) else 1e-12)
    dg.dolinc_set_flags(M, None)


@pytest.mark.parametrize("name,nv", [("tri", 1), ("tri_bnd", 4), ("tet", 5), ("strip", 1)])
def test_weno5_fp32_step(name, nv):
    """WENO5-DOLINC in the FP32 bulk path: one SSP-RK3 step against the oracle (the
    nonlinear weights are smooth functions of the data, so FP32 stays close)."""
    m, O = mesh(name)
    M = gpu_mesh(m)
    u = field(m, nv, seed=71)
    fx = euler_ok(nv) if nv > 1 else dict(flux="upwind", adv=(1.0, 0.5, 0.3))
    sch = dg.Scheme(k=3, r=1, n_diff=2, nv=nv, precision="fp32", limiter="weno5_all", **fx)
    ws = dg.workspace(M, sch)
    x = to_dev(M, u)
    dt = 1e-3
    dg.dolinc_rk_step(M, sch, dt, x, ws)
    dg.dolinc_sync_status(M, ws)
    got = M.from_lib(x.cpu().numpy())
    want = O.rk3_step(u, oracle.Scheme(k=3, r=1, n_diff=2, nv=nv, eno=4, **fx), dt)
    # WENO5 reads second-order differentials: the per-cell rule at N_s = 2
    ok, worst = increment_ok(O, got - u, want - u, u, dt, "fp32", 2, fx, m["dim"])
    assert ok, worst


def test_weno5_reproduces_the_papers_sine_errors():
    """Sec 3.2, Table orderHOScheme, WENO5 column: one period of sine advection on 20
    and 40 uniform cells through the GPU step, FP64, within 6% of the printed errors."""
    import os
    rows = [r.split() for r in open(os.path.join(os.path.dirname(__file__), "golden", "paper_l2_1d_sine.txt"))
            if r.strip() and not r.startswith("#")]
    for row in rows[1:3]:
        n, want = int(row[0]), float(row[4])
        m = synth.strip_mesh(np.full(n, 1.0 / n))
        M = gpu_mesh(m)
        u0 = synth.cell_average(m, lambda p: np.sin(2 * np.pi * p[:, 0]), q=6)[None]
        sch = dg.Scheme(k=3, r=1, n_diff=2, nv=1, precision="fp64", limiter="weno5_all", flux="upwind",
                        adv=(1.0, 0.0))
        ws = dg.workspace(M, sch)
        x = to_dev(M, u0)
        steps = int(np.ceil(1.0 / (0.05 / n)))
        for _ in range(steps):
            dg.dolinc_rk_step(M, sch, 1.0 / steps, x, ws)
        dg.dolinc_sync_status(M, ws)
        e = np.sqrt(np.mean((M.from_lib(x.cpu().numpy()) - u0) ** 2))
        assert abs(e / want - 1) < 0.06, (n, e, want)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,nv", [("tri_bnd", 4), ("tet", 5), ("hexprism", 1)])
def test_first_order_fallback_csr4_one_differential(prec, name, nv):
    """The first-order fallback needs no second-order differentials: CSR4 (n_diff = 1)
    with flagged faces, one full SSP-RK3 step against the oracle."""
    m, O = mesh(name)
    M = gpu_mesh(m)
    u = field(m, nv, seed=34)
    flags = (np.random.default_rng(35).uniform(size=O.n_cells) < 0.4).astype(np.uint8)
    fx = euler_ok(nv) if nv > 1 else dict(flux="upwind", adv=(1.0, 0.7, 0.4))
    sch = dg.Scheme(k=4, r=1, n_diff=1, nv=nv, precision=prec, limiter="first_order_flagged", **fx)
    dg.dolinc_set_flags(M, torch.from_numpy(M.to_lib(flags)).cuda())
    ws = dg.workspace(M, sch)
    x = to_dev(M, u)
    dt = 2e-3
    dg.dolinc_rk_step(M, sch, dt, x, ws)
    dg.dolinc_sync_status(M, ws)
    got = M.from_lib(x.cpu().numpy())
    want = O.rk3_step(u, oracle.Scheme(k=4, r=1, n_diff=1, nv=nv, eno=3, troubled=flags, **fx), dt)
    base = O.rk3_step(u, oracle.Scheme(k=4, r=1, n_diff=1, nv=nv, **fx), dt)
    if prec == "fp64":
        assert rel(got - u, want - u) < 1e-11
    else:
        ok, worst = increment_ok(O, got - u, want - u, u, dt, "fp32", 1, fx, m["dim"])
        assert ok, worst
    assert rel(base - u, want - u) > 1e-3          # the fallback changed the step
    dg.dolinc_set_flags(M, None)


# ---------------------------------------------------------------------------- launch shapes

@pytest.mark.parametrize("lanes,block", [(1, 64), (1, 256), (4, 128), (4, 32), (8, 256), (8, 96), (0, 64), (0, 128),
                                         (0, 256)])
@pytest.mark.parametrize("name,nv,prec", [("tet", 5, "fp32"), ("hexprism", 1, "fp64"), ("tri_bnd", 4, "fp64"),
                                          ("tet", 5, "fp32_bf16")])
def test_launch_shapes_give_the_same_stage(lanes, block, name, nv, prec):
    """Every lanes-per-cell / block shape the autotuner may pick computes the same stage."""
    m, O = mesh(name)
    M = gpu_mesh(m)
    u = field(m, nv, seed=50)
    fx = euler_ok(nv) if nv > 1 else dict(flux="upwind", adv=(1.0, 0.5, 0.3))
    sch = dg.Scheme(k=3, r=1, n_diff=3, nv=nv, precision=prec, **fx)
    ws = dg.workspace(M, sch)
    dg.dolinc_set_tuning(M, sch, lanes, block, lanes, block)
    x = to_dev(M, u)
    dt = 1e-3
    dg.dolinc_rk_step(M, sch, dt, x, ws)
    dg.dolinc_sync_status(M, ws)
    got = M.from_lib(x.cpu().numpy())
    want = O.rk3_step(u, oracle.Scheme(k=3, r=1, n_diff=3, nv=nv, **fx), dt)
    tol = {"fp64": 1e-12, "fp32": 1e-6, "fp32_bf16": 1e-5}[prec]
    assert rel(got - u, want - u) < tol * 10 or rel(got, want) < tol


@pytest.mark.parametrize("lanes,block", [(-1, 128), (-1, 256), (-4, 128), (-4, 256)])
@pytest.mark.parametrize("name,nv,prec", [("tet", 5, "fp32"), ("hexprism", 1, "fp64"), ("tri_bnd", 4, "fp64"),
                                          ("tet", 5, "fp32_bf16"), ("strip", 1, "fp32"), ("tri", 1, "fp64")])
def test_pipelined_differentials_are_bit_identical(lanes, block, name, nv, prec):
    """The persistent pipelined differential passes (bulk asynchronous copies of each
    tile into two shared-memory buffers) do the arithmetic of the gather kernel with
    the same lanes per cell in the same order: every order is bit-identical to it,
    and the step still matches the oracle."""
    m, O = mesh(name)
    M = gpu_mesh(m)
    u = field(m, nv, seed=52)
    fx = euler_ok(nv) if nv > 1 else dict(flux="upwind", adv=(1.0, 0.5, 0.3))
    N = 4 if prec != "fp32_bf16" else 3
    sch = dg.Scheme(k=3, r=1, n_diff=N, nv=nv, precision=prec, **fx)
    ws = dg.workspace(M, sch)
    _, _, _, tot = dg.dolinc_diff_layout(M, sch, N)
    out = {}
    for dl, db in ((-lanes, 128), (lanes, block)):
        dg.dolinc_set_tuning(M, sch, dl, db, 1, 128)
        diff = torch.zeros(tot, dtype=torch.uint8, device="cuda")
        dg.dolinc_differentials(M, sch, to_dev(M, u), N, diff, ws)
        dg.dolinc_sync_status(M, ws)
        out[dl] = diff.cpu().numpy()
    assert np.array_equal(out[-lanes], out[lanes])
    x = to_dev(M, u)
    dt = 1e-3
    dg.dolinc_rk_step(M, sch, dt, x, ws)
    dg.dolinc_sync_status(M, ws)
    got = M.from_lib(x.cpu().numpy())
    want = O.rk3_step(u, oracle.Scheme(k=3, r=1, n_diff=N, nv=nv, **fx), dt)
    tol = {"fp64": 1e-12, "fp32": 1e-6, "fp32_bf16": 1e-5}[prec]
    assert rel(got - u, want - u) < tol * 10 or rel(got, want) < tol


@pytest.mark.parametrize("lanes,block", [(-1, 64), (-1, 128), (-2, 64), (-2, 256)])
@pytest.mark.parametrize("name,nv,prec,limiter", [("tet", 5, "fp32", "none"), ("hexprism", 1, "fp64", "none"),
                                                  ("tri_bnd", 4, "fp64", "none"), ("tet", 5, "fp32_bf16", "none"),
                                                  ("strip", 1, "fp32", "none"), ("tri", 1, "fp64", "none"),
                                                  ("tri_bnd", 4, "fp64", "eno3_flagged"),
                                                  ("tet", 5, "fp32", "first_order_flagged")])
def test_face_centric_stages_are_bit_identical(lanes, block, name, nv, prec, limiter):
    """The persistent pipelined stage (lanes -1: each face once per tile that needs it)
    and the face-centric pair (lanes -2: each face once, then a slot-ordered gather)
    evaluate faces in the canonical orientation with the operands of the
    one-thread-per-cell kernel and sum each cell's fluxes in slot order: without a
    limiter the residual and the full step are bit-identical to that kernel's.  With
    the ENO3 limiter the compiler is free to fuse the stencil-choice arithmetic
    differently in the kernels, so agreement is to rounding (a few ulp).  The step
    matches the oracle."""
    m, O = mesh(name)
    M = gpu_mesh(m)
    u = field(m, nv, seed=53)
    fx = euler_ok(nv) if nv > 1 else dict(flux="upwind", adv=(1.0, 0.5, 0.3))
    sch = dg.Scheme(k=3, r=1, n_diff=2, nv=nv, precision=prec, limiter=limiter, **fx)
    flags = None
    if limiter != "none":
        flags = (np.random.default_rng(54).uniform(size=O.n_cells) < 0.3).astype(np.uint8)
        dg.dolinc_set_flags(M, torch.from_numpy(M.to_lib(flags)).cuda())
    ws = dg.workspace(M, sch)
    res, step = {}, {}
    for sl, sb in ((1, 128), (lanes, block)):
        dg.dolinc_set_tuning(M, sch, 1, 128, sl, sb)
        R = torch.zeros((nv, M.n_cells), dtype=torch.float64, device="cuda")
        dg.dolinc_residual(M, sch, to_dev(M, u), R, ws)
        x = to_dev(M, u)
        for _ in range(2):
            dg.dolinc_rk_step(M, sch, 1e-3, x, ws)
        dg.dolinc_sync_status(M, ws)
        res[sl], step[sl] = R.cpu().numpy(), x.cpu().numpy()
    if limiter == "none":
        assert np.array_equal(res[1], res[lanes])
        assert np.array_equal(step[1], step[lanes])
    else:
        ulp = 1e-14 if prec == "fp64" else 1e-6
        assert rel(res[lanes], res[1]) < ulp
        inc = step[1] - to_dev(M, u).cpu().numpy()
        assert np.abs(step[lanes] - step[1]).max() < 100 * ulp * np.abs(inc).max()
    got = M.from_lib(step[lanes])
    eno = {"none": 0, "eno3_flagged": 2, "first_order_flagged": 3}[limiter]
    want = O.run(u, oracle.Scheme(k=3, r=1, n_diff=2, nv=nv, eno=eno, troubled=flags, **fx), 1e-3, 2)
    tol = {"fp64": 1e-12, "fp32": 1e-6, "fp32_bf16": 1e-5}[prec]
    assert rel(got - u, want - u) < tol * 10 or rel(got, want) < tol
    dg.dolinc_set_flags(M, None)


def test_autotune_picks_a_valid_shape_and_keeps_parity(tmp_path):
    m, O = mesh("tet")
    M = gpu_mesh(m)
    u = field(m, 5, seed=51)
    sch = dg.Scheme(k=3, r=1, n_diff=2, nv=5, precision="fp64", **euler_ok(5))
    ws = dg.workspace(M, sch)
    x = to_dev(M, u)
    cache = str(tmp_path / "tune.txt")
    t = dg.dolinc_autotune(M, sch, x, ws, cache_path=cache)
    assert t["diff_lanes"] in (0, 1, 4, 8, -1, -4) and t["stage_lanes"] in (0, 1, 4, 8, -1, -2) and not t["from_cache"]
    t2 = dg.dolinc_autotune(M, sch, x, ws, cache_path=cache)
    assert t2["from_cache"] and t2["stage_lanes"] == t["stage_lanes"]
    dt = 1e-3
    dg.dolinc_rk_step(M, sch, dt, x, ws)
    dg.dolinc_sync_status(M, ws)
    want = O.rk3_step(u, oracle.Scheme(k=3, r=1, n_diff=2, nv=5, **euler_ok(5)), dt)
    assert rel(M.from_lib(x.cpu().numpy()), want) < 1e-12


@pytest.mark.parametrize("name,nv,prec", [("tet", 5, "fp32"), ("tet", 5, "fp64"), ("tet", 5, "fp32_bf16"),
                                          ("tri", 4, "fp32"), ("tri", 1, "fp32"), ("hexprism", 1, "fp64")])
@pytest.mark.parametrize("stage_shape", [(-2, 128), (1, 128)])
def test_paired_schedule_is_bit_identical(name, nv, prec, stage_shape):
    """Diff lanes 2 (the paired schedule: a stage's unread order-2 pass runs in one
    launch with the next stage's order-1 pass, order 1 double-buffered) gives the
    steps of lanes 1 bit for bit; where the records allow it (16-byte multiples) the
    paired launch runs twice per step."""
    m, O = mesh(name)
    M = gpu_mesh(m)
    u = field(m, nv, seed=61)
    fx = euler_ok(nv) if nv > 1 else dict(flux="upwind", adv=(1.0, 0.5, 0.3))
    sch = dg.Scheme(k=3, r=1, n_diff=2, nv=nv, precision=prec, **fx)
    ws = dg.workspace(M, sch)
    out = {}
    for lanes in (1, 2):
        dg.dolinc_set_tuning(M, sch, lanes, 64, *stage_shape)
        x = to_dev(M, u)
        dg.dolinc_profile_enable(M, True)
        for _ in range(2):
            dg.dolinc_rk_step(M, sch, 1e-3, x, ws)
        kms, kn = dg.profile_read(M)
        dg.dolinc_profile_enable(M, False)
        dg.dolinc_sync_status(M, ws)
        out[lanes] = (x.cpu().numpy(), kn[dg.KERNEL_KINDS.index("diff_pair")])
    assert np.array_equal(out[1][0], out[2][0])
    assert out[1][1] == 0
    records_ok = not (name == "tri" and nv == 1 and prec != "fp64")      # 8-byte order-1 records
    assert out[2][1] == (4 if records_ok else 0), out[2][1]
    want = O.run(u, oracle.Scheme(k=3, r=1, n_diff=2, nv=nv, **fx), 1e-3, 2)
    got = M.from_lib(out[2][0])
    tol = {"fp64": 1e-12, "fp32": 1e-6, "fp32_bf16": 1e-5}[prec]
    assert rel(got - u, want - u) < tol * 10 or rel(got, want) < tol


@pytest.mark.parametrize("name,nv,prec", [("tet", 5, "fp32"), ("tet", 5, "fp64"), ("tet", 5, "fp32_bf16"),
                                          ("tri", 1, "fp32"), ("tri_bnd", 4, "fp64"), ("hexprism", 1, "fp32")])
@pytest.mark.parametrize("shape", [(1, 64, -2, 128), (2, 64, -2, 128), (2, 128, 1, 128), (4, 128, 4, 64),
                                   (-1, 128, -1, 128), (0, 128, 0, 64)])
def test_several_steps_per_call_equal_single_steps(name, nv, prec, shape):
    """dolinc_rk_steps(n) keeps the state on the device (the last stage writes the next
    step's record, the paired schedule pairs across steps) and must give n calls of
    dolinc_rk_step bit for bit, for every launch shape."""
    m, O = mesh(name)
    M = gpu_mesh(m)
    u = field(m, nv, seed=62)
    fx = euler_ok(nv) if nv > 1 else dict(flux="upwind", adv=(1.0, 0.5, 0.3))
    sch = dg.Scheme(k=3, r=1, n_diff=2, nv=nv, precision=prec, **fx)
    ws = dg.workspace(M, sch)
    dg.dolinc_set_tuning(M, sch, *shape)
    a, b = to_dev(M, u), to_dev(M, u)
    for _ in range(3):
        dg.dolinc_rk_step(M, sch, 1e-3, a, ws)
    dg.dolinc_rk_steps(M, sch, 1e-3, 3, b, ws)
    dg.dolinc_sync_status(M, ws)
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
