"""Pins of the oracle's semi-implicit DOLINC step (Sec 2.4, Eq USR3 and Eq CSR4:
phi_f = w_s phi_up + (1 - w_s) phi_down + c_r; an implicit time integration takes the
weight part at the new level and keeps c_r explicit).

Each pin is fixed by something other than the oracle itself:
  - the weights w_s of USR3 and CSR4 against the paper's formulas in the inversion
    coefficients (Eq lCoeffDLC1, Eq rCoeffDLC1), with the stencil coefficients from a
    brute-force solve of the polynomial-exactness conditions on geometric cells;
  - one step on a uniform periodic strip against the closed-form Fourier
    amplification factor of the split scheme, both flow directions, theta = 1 and 1/2;
  - the split reassembled (K u + C(u)) against the explicit residual of the C oracle;
  - theta = 0 against the explicit forward Euler step; conservation on periodic
    meshes; the deferred-correction fixed point against the full theta scheme.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _brute_coeff(k, r, g):
    """Stencil coefficients of the face value at the right face of cell i (x = 0) from
    the averages of cells i-r .. i-r+k-1, cell i+q of width g^q: exact for polynomials
    of degree < k (a k x k solve, nothing shared with the oracle's formula)."""
    q = np.arange(-r, k - r)
    right = np.array([sum(g ** j for j in range(1, qq + 1)) if qq >= 0 else -sum(g ** j for j in range(qq + 1, 1))
                      for qq in q])
    left = right - g ** q.astype(float)
    A = np.array([[(right[j] ** (p + 1) - left[j] ** (p + 1)) / ((p + 1) * (right[j] - left[j])) for j in range(k)]
                  for p in range(k)])
    b = np.zeros(k)
    b[0] = 1.0
    return dict(zip(q.tolist(), np.linalg.solve(A, b)))


def _paper_ws(k, r, g):
    """w_s by the paper: USR3 w_s = c_{-1} a0^{-1} + c_0, CSR4 adds c_2 a0^{2}, with
    a0^{-1} = 1 - 1/g (Eq lCoeffDLC1) and a0^{2} = g (Eq rCoeffDLC1)."""
    c = _brute_coeff(k, r, g)
    if (k, r) == (3, 1):
        return c[-1] * (1.0 - 1.0 / g) + c[0]
    if (k, r) == (4, 1):
        return c[-1] * (1.0 - 1.0 / g) + c[0] + c[2] * g
    raise ValueError


def _xfaces(O):
    return np.nonzero((O.neigh >= 0) & (O.neigh != O.owner))[0]


@pytest.mark.parametrize("g", [0.9, 1.0, 1.15])
@pytest.mark.parametrize("k,r", [(3, 1), (4, 1)])
def test_weights_follow_the_inversion_coefficients(k, r, g):
    n = 30
    m = synth.strip_mesh(0.02 * g ** np.arange(n), height=0.02, boundary="transmissive")
    O = oracle.Oracle(m)
    s = oracle.Scheme(k=k, r=r, flux="upwind", nv=1, adv=(1.0, 0.0, 0.0))
    WL, WR = O.face_weights(s)
    wL, wR = _paper_ws(k, r, g), _paper_ws(k, r, 1.0 / g)
    checked = 0
    for f in _xfaces(O):
        i = O.owner[f]
        if i < 4 or i > n - 6:
            continue
        assert abs(WL[f, 0, 0] - wL) < 1e-12 and abs(WL[f, 1, 0] - (1.0 - wL)) < 1e-12
        assert abs(WR[f, 0, 0] - wR) < 1e-12 and abs(WR[f, 1, 0] - (1.0 - wR)) < 1e-12
        checked += 1
    assert checked > 10
    if g == 1.0:    # the paper's uniform values: USR3 5/6 (from -1/6, 5/6, 1/3), CSR4 1/2
        assert abs(wL - {(3, 1): 5.0 / 6.0, (4, 1): 0.5}[(k, r)]) < 1e-14


@pytest.mark.parametrize("theta", [1.0, 0.5])
@pytest.mark.parametrize("a", [0.8, -0.7])
@pytest.mark.parametrize("k,r", [(3, 1), (4, 1)])
def test_fourier_amplification_on_uniform_strip(k, r, a, theta):
    """Discrete data u_j = cos(kappa j + p) on n uniform periodic cells of width h.
    With nu = a dt / h, face symbol Phi (the k-cell stencil), weight symbol W and
    difference symbol (1 - e^{-i kappa}) per cell, one step multiplies the mode by
        G = (1 - nu (1 - e^{-ik}) [(1 - theta) W + Phi - W]) / (1 + theta nu (1 - e^{-ik}) W)."""
    n, h, dt = 24, 0.05, 0.11
    m = synth.strip_mesh(np.full(n, h), height=0.07)
    O = oracle.Oracle(m)
    s = oracle.Scheme(k=k, r=r, flux="upwind", nv=1, adv=(a, 0.0, 0.0))
    c = _brute_coeff(k, r, 1.0)
    w = _paper_ws(k, r, 1.0)
    nu = a * dt / h
    for mode, p in ((1, 0.3), (5, 1.1), (11, -0.4)):
        kap = 2 * np.pi * mode / n
        e = lambda t: np.exp(1j * kap * t)
        if a >= 0:      # face j+1/2 from cell j upwind
            Phi = sum(cq * e(q) for q, cq in c.items())
            W = w + (1 - w) * e(1)
        else:           # from cell j+1 upwind, the stencil mirrored
            Phi = sum(cq * e(1 - q) for q, cq in c.items())
            W = w * e(1) + (1 - w)
        dif = 1 - e(-1)
        G = (1 - nu * dif * ((1 - theta) * W + Phi - W)) / (1 + theta * nu * dif * W)
        j = np.arange(n)
        u = np.cos(kap * j + p)[None, :]
        want = np.real(G * np.exp(1j * (kap * j + p)))
        got = O.semi_implicit_step(u, s, dt, theta)[0]
        np.testing.assert_allclose(got, want, atol=1e-12)


def _meshes():
    return [("tri", synth.tri_mesh(12, 10, 0.2, 3), (1.0, 0.6, 0.0)),
            ("tet", synth.tet_mesh(4, 0.15, 2), (0.7, -0.5, 0.4))]


@pytest.mark.parametrize("skew", [False, True])
@pytest.mark.parametrize("k,r", [(3, 1), (4, 1), (5, 2)])
def test_split_reassembles_the_residual(k, r, skew):
    """K u + C(u) = -V R(u): the weight part and c_r summed are the explicit DOLINC
    residual of the C oracle (face order, signs and the owner/neighbour scatter)."""
    for name, m, adv in _meshes():
        O = oracle.Oracle(m, skew=skew)
        s = oracle.Scheme(k=k, r=r, flux="upwind", nv=1, adv=adv)
        u = np.random.default_rng(7).normal(size=(1, O.n_cells))
        lhs = O.implicit_operator(s) @ u[0] + O.explicit_correction(u, s)
        R = O.residual(u, s)[0]
        np.testing.assert_allclose(lhs, -O.V * R, atol=1e-12 * np.abs(O.V * R).max(), err_msg=name)


def test_theta_zero_is_forward_euler_and_steps_conserve():
    for name, m, adv in _meshes():
        O = oracle.Oracle(m)
        s = oracle.Scheme(k=3, r=1, flux="upwind", nv=1, adv=adv)
        u = np.random.default_rng(2).normal(size=(1, O.n_cells))
        dt = 0.02
        np.testing.assert_allclose(O.semi_implicit_step(u, s, dt, 0.0), u + dt * O.residual(u, s), atol=1e-13)
        for theta, big in ((1.0, 2.0), (0.5, 0.3)):
            u1 = O.semi_implicit_step(u, s, big, theta)
            assert abs((O.V * u1[0]).sum() - (O.V * u[0]).sum()) < 1e-12 * np.abs(O.V * u[0]).sum()
        assert np.allclose(O.semi_implicit_step(np.ones((1, O.n_cells)), s, 1.0, 1.0), 1.0, atol=1e-13)


def test_boundary_faces_and_rejections():
    """Zero-gradient boundary faces take a.S u_c in the matrix; Dirichlet faces and
    systems are refused."""
    m = synth.strip_mesh(np.full(16, 0.05), height=0.05, boundary="transmissive")
    O = oracle.Oracle(m)
    s = oracle.Scheme(k=3, r=1, flux="upwind", nv=1, adv=(1.0, 0.0, 0.0))
    u = np.random.default_rng(4).normal(size=(1, O.n_cells))
    lhs = O.implicit_operator(s) @ u[0] + O.explicit_correction(u, s)
    np.testing.assert_allclose(lhs, -O.V * O.residual(u, s)[0], atol=1e-12)
    bk = np.where(O.neigh < 0, 2, 0).astype(np.int32)
    sd = oracle.Scheme(k=3, r=1, flux="upwind", nv=1, bkind=bk, bval=np.zeros((1, O.n_faces)))
    with pytest.raises(ValueError):
        O.semi_implicit_step(u, sd, 0.1)
    with pytest.raises(ValueError):
        O.semi_implicit_step(np.ones((4, O.n_cells)), oracle.Scheme(k=3, r=1, flux="rusanov", nv=4), 0.1)


def test_outer_iterations_reach_the_full_theta_scheme():
    """The deferred-correction fixed point solves the theta scheme of the full DOLINC
    operator: V (u' - u)/dt = theta V R(u') + (1 - theta) V R(u)."""
    m = synth.tri_mesh(12, 10, 0.2, 3)
    O = oracle.Oracle(m)
    s = oracle.Scheme(k=3, r=1, flux="upwind", nv=1, adv=(1.0, 0.6, 0.0))
    u = np.random.default_rng(9).normal(size=(1, O.n_cells))
    dt, theta = 0.04, 0.5
    u1 = O.semi_implicit_step(u, s, dt, theta, n_outer=60)
    res = O.V * (u1[0] - u[0]) / dt - theta * O.V * O.residual(u1, s)[0] - (1 - theta) * O.V * O.residual(u, s)[0]
    assert np.abs(res).max() < 1e-10 * np.abs(O.V * O.residual(u, s)[0]).max()
    one = O.semi_implicit_step(u, s, dt, theta, n_outer=1)
    assert np.abs(one - u1).max() > 1e-6        # the semi-implicit step itself is not the fixed point


def test_usr3_weight_part_is_dissipative_and_csr4_is_not():
    """Sec 2.4 remarks that the DOLINC split helps the implicit matrix; measured: on
    jittered triangles and tetrahedra every eigenvalue of
    V^-1 K has a non-negative real part for USR3 (its w_s favours the upwind cell), so
    V/dt + theta K is definite at any dt; CSR4's central weights give eigenvalues with
    negative real parts, so its matrix turns indefinite above some Courant number."""
    import scipy.sparse as sp
    for name, m, adv in _meshes():
        O = oracle.Oracle(m)
        for (k, r), dissipative in (((3, 1), True), ((4, 1), False)):
            s = oracle.Scheme(k=k, r=r, flux="upwind", nv=1, adv=adv)
            K = (sp.diags(1.0 / O.V) @ O.implicit_operator(s)).toarray()
            ev = np.linalg.eigvals(K)
            scale = np.abs(ev).max()
            if dissipative:
                assert ev.real.min() >= -1e-10 * scale, (name, k, ev.real.min())
            else:
                assert ev.real.min() < -0.05 * scale, (name, k, ev.real.min())
