"""Per-face / per-cell tolerance rule shared by the GPU parity tests.

A face value is sum_m W0[m] phi_0^(m) + W1[m] phi_1^(m) over the scheme's DOLINC
order Ns; phi^(m) carries the rounding of m nested Gauss sums and the weights the
rounding of the far-field recursion, which grows with the face's growth-rate spread
G = max(g, 1/g) like G^(Ns(Ns-1)).  Per face:
  FP64       1e-12 * 4^Ns     * G^(Ns(Ns-1)) * max|u|
  FP32       1e-5  * 8^(Ns-1) * G^(Ns(Ns-1)) * max|u|      (Ns = 1: the stated 1e-5)
  FP32+BF16  3e-3 (8-bit mantissa on orders >= 2; coarse test meshes)
A residual takes the per-face bound through |S_f| * (largest wave speed) / V_c: for
FP32 that is 1e-5 relative to the face-flux magnitudes, not to the residual, which is
their O(h) cancellation.
"""
import numpy as np


def face_G(O):
    g = np.where(O.neigh >= 0, O.w / np.maximum(1 - O.w, 1e-300), 1.0)
    return np.maximum(g, 1.0 / g)


def face_tol(O, prec, Ns, scale):
    base = {"fp64": 1e-12 * 4.0 ** Ns, "fp32": 1e-5 * 8.0 ** (Ns - 1), "fp32_bf16": 3e-3}[prec]
    return base * face_G(O) ** (Ns * (Ns - 1)) * scale


def cell_tol(O, ftol, lam):
    """per-cell residual bound: (1/V_c) sum_f |S_f| lam tol_f"""
    a = np.linalg.norm(O.S, axis=1) * lam * ftol
    t = np.zeros(O.n_cells)
    np.add.at(t, O.owner, a)
    nb = O.neigh >= 0
    np.add.at(t, O.neigh[nb], a[nb])
    return t / O.V


def wave_speed(u, fx, dim):
    """Largest wave speed of the data: |a| (advection), |u| sqrt(dim) (Burgers along
    (1,..,1)), |v| + c (Euler, gamma = 1.4)."""
    if fx["flux"] == "upwind":
        return float(np.linalg.norm(fx["adv"]))
    if fx["flux"] == "burgers":
        return float(np.abs(u).max() * np.sqrt(dim))
    rho, E = u[0], u[-1]
    vel = u[1:-1] / rho
    p = 0.4 * (E - 0.5 * rho * (vel * vel).sum(0))
    return float((np.sqrt((vel * vel).sum(0)) + np.sqrt(1.4 * p / rho)).max())


def increment_ok(O, got_inc, want_inc, u, dt, prec, Ns, fx, dim, factor=2.0):
    """Every cell's step (or stage) increment within dt times the per-cell residual
    bound (the SSP-RK3 stage weights of a step sum to one); factor 2 covers the
    Euler flux's two states per face.  Returns (ok, worst ratio)."""
    lam = wave_speed(u, fx, dim)
    ratio = 0.0
    for v in range(u.shape[0]):
        bound = dt * factor * cell_tol(O, face_tol(O, prec, Ns, np.abs(u).max()), lam)
        ratio = max(ratio, float((np.abs(got_inc[v] - want_inc[v]) / bound).max()))
    return ratio <= 1.0, ratio
