"""Initial fields and their cell averages.

Cell averages are integrals over each cell divided by its measure.  A cell is
integrated as the union of simplices joining the mean of its nodes to each of
its outward half-faces (a 4-node face is first split into the four triangles
that join consecutive nodes to the mean of the face's nodes).  Each simplex uses
the Stroud conical-product rule: Gauss-Legendre points on the unit cube (square)
collapsed onto the simplex (Duffy map), exact for polynomials of total degree
2q-3 (3D) or 2q-2 (2D) with q points per direction.
"""
import numpy as np


def _simplices(mesh, apex, c0, lo, hi):
    """Signed simplices (apex first) of half-faces lo..hi, as (cell id - c0, vertices);
    apex is indexed by cell id - c0."""
    dim = mesh["dim"]
    nodes = mesh["nodes"]
    hc = mesh["_hf_cell"][lo:hi] - c0
    hf = mesh["_hf_nodes"][lo:hi]
    if dim == 2:
        verts = np.stack([apex[hc], nodes[hf[:, 0]], nodes[hf[:, 1]]], axis=1)
        return hc, verts
    nf = (hf >= 0).sum(axis=1)
    cells, verts = [], []
    tri = nf == 3
    if tri.any():
        v = np.stack([apex[hc[tri]], nodes[hf[tri, 0]], nodes[hf[tri, 1]], nodes[hf[tri, 2]]], axis=1)
        cells.append(hc[tri])
        verts.append(v)
    quad = nf == 4
    if quad.any():
        q = hf[quad]
        fc = nodes[q].mean(axis=1)
        for e in range(4):
            v = np.stack([apex[hc[quad]], fc, nodes[q[:, e]], nodes[q[:, (e + 1) % 4]]], axis=1)
            cells.append(hc[quad])
            verts.append(v)
    if not cells:
        return np.zeros(0, dtype=np.int64), np.zeros((0, dim + 1, dim))
    return np.concatenate(cells), np.concatenate(verts)


def _average_range(mesh, func, q, c0, c1, chunk):
    """Integrals and measures of cells c0..c1-1 (half-faces are sorted by cell)."""
    dim = mesh["dim"]
    nodes = mesh["nodes"]
    hcell = mesh["_hf_cell"]
    lo, hi = (int(x) for x in np.searchsorted(hcell, [c0, c1]))
    n = c1 - c0
    # apex: mean of the cell's half-face node occurrences (any interior point gives the
    # same signed integral; duplicates do not matter)
    cnt = np.zeros(n)
    apex = np.zeros((n, dim))
    for s in range(lo, hi, chunk):
        h = mesh["_hf_nodes"][s:min(s + chunk, hi)]
        c = hcell[s:min(s + chunk, hi)] - c0
        valid = h >= 0
        pts = (nodes[np.maximum(h, 0)] * valid[..., None]).sum(axis=1)
        cnt += np.bincount(c, weights=valid.sum(axis=1), minlength=n)
        for k in range(dim):
            apex[:, k] += np.bincount(c, weights=pts[:, k], minlength=n)
    apex /= cnt[:, None]
    ref, wt = _duffy_rule(dim, q)
    acc = None
    vol = np.zeros(n)
    for s in range(lo, hi, chunk):
        c, v = _simplices(mesh, apex, c0, s, min(s + chunk, hi))
        if c.shape[0] == 0:
            continue
        E = v[:, 1:, :] - v[:, :1, :]                         # edge vectors [n, dim, dim]
        det = np.linalg.det(np.transpose(E, (0, 2, 1)))       # signed measure * dim!
        pts = v[:, None, 0, :] + np.einsum("pk,nkd->npd", ref, E)
        val = np.asarray(func(pts.reshape(-1, dim)), dtype=np.float64)
        val = val.reshape(pts.shape[0], pts.shape[1], -1)
        contrib = np.einsum("npv,p,n->nv", val, wt, det)
        if acc is None:
            acc = np.zeros((n, val.shape[2]))
        for j in range(val.shape[2]):
            acc[:, j] += np.bincount(c, weights=contrib[:, j], minlength=n)
        vol += np.bincount(c, weights=det * wt.sum(), minlength=n)
    return acc, vol


_FORKED = {}


def _forked_range(r):
    a = _FORKED
    return _average_range(a["mesh"], a["func"], a["q"], r[0], r[1], a["chunk"])


def _duffy_rule(dim, q):
    x, w = np.polynomial.legendre.leggauss(q)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    if dim == 2:
        U, V = np.meshgrid(x, x, indexing="ij")
        WU, WV = np.meshgrid(w, w, indexing="ij")
        U, V, W = U.ravel(), V.ravel(), (WU * WV).ravel()
        bary = np.stack([U, (1 - U) * V], axis=1)            # reference triangle coords
        wt = W * (1 - U)                                      # Jacobian of the collapse
        return bary, wt                                       # sum(wt) = 1/2
    U, V, Z = np.meshgrid(x, x, x, indexing="ij")
    WU, WV, WZ = np.meshgrid(w, w, w, indexing="ij")
    U, V, Z = U.ravel(), V.ravel(), Z.ravel()
    W = (WU * WV * WZ).ravel()
    bary = np.stack([U, (1 - U) * V, (1 - U) * (1 - V) * Z], axis=1)
    wt = W * (1 - U) ** 2 * (1 - V)                           # sum(wt) = 1/6
    return bary, wt


def cell_average(mesh, func, q=4, nv=None, chunk=1 << 16, workers=1):
    """Cell averages of func over every cell.

    func maps points [P, dim] to values [P] or [P, nv].
    Returns [n_cells] or [nv, n_cells] (variables first, the library's layout).
    Half-faces are taken `chunk` at a time, so memory stays bounded on large meshes.
    workers > 1 splits the cells over forked processes: only for callers that have not
    initialised CUDA (a process forked after that can hang).
    """
    n_cells = mesh["cell_face_offsets"].shape[0] - 1
    if workers <= 1 or n_cells < 4 * workers:
        acc, vol = _average_range(mesh, func, q, 0, n_cells, chunk)
    else:
        import multiprocessing as mp
        cuts = np.linspace(0, n_cells, 4 * workers + 1).astype(np.int64)
        ranges = [(int(cuts[i]), int(cuts[i + 1])) for i in range(4 * workers)]
        _FORKED.update(mesh=mesh, func=func, q=q, chunk=chunk)
        try:
            with mp.get_context("fork").Pool(workers) as pool:
                parts = pool.map(_forked_range, ranges)
        finally:
            _FORKED.clear()
        acc = np.concatenate([p[0] for p in parts])
        vol = np.concatenate([p[1] for p in parts])
    avg = acc / vol[:, None]
    if avg.shape[1] == 1 and nv is None:
        return avg[:, 0]
    return np.ascontiguousarray(avg.T)


# ----------------------------------------------------------------------------------------
# initial fields

def sine2d(p):
    """u0 = sin(2 pi x) sin(2 pi y)."""
    return np.sin(2 * np.pi * p[:, 0]) * np.sin(2 * np.pi * p[:, 1])


def gaussian3d(p, sigma=0.1, centre=(0.5, 0.5, 0.5), images=1):
    """Gaussian pulse of width sigma on the unit periodic cube, periodised by
    summing the images within `images` periods in each direction.  The pulse is a
    product over the axes, so the sum over the (2 images + 1)^3 shifted copies is the
    product of the three one-axis image sums."""
    out = np.ones(p.shape[0])
    for k in range(3):
        s = np.zeros(p.shape[0])
        for a in range(-images, images + 1):
            d = p[:, k] - (centre[k] + a)
            s += np.exp(-0.5 * d * d / sigma ** 2)
        out *= s
    return out


def vortex_params(gamma=1.4, beta=5.0, R=0.1, centre=(0.5, 0.5), u_inf=(1.0, 1.0, 0.0)):
    return dict(gamma=gamma, beta=beta, R=R, centre=centre, u_inf=u_inf)


def isentropic_vortex(p, t=0.0, dim=3, gamma=1.4, beta=5.0, R=0.1, centre=(0.5, 0.5),
                      u_inf=(1.0, 1.0, 0.0), images=1):
    """Conserved variables of an isentropic vortex (axis z) convected by u_inf
    on the unit periodic box, at time t.

    Tangential speed v(r) = beta/(2 pi) (r/R) exp((1 - (r/R)^2)/2).  With
    T = p/rho and p = rho^gamma (isentropic, free stream rho = p = 1), radial
    equilibrium dp/dr = rho v^2/r gives dT/dr = (gamma-1)/gamma v^2/r, hence
    T(r) = 1 - (gamma-1)/(2 gamma) (beta/(2 pi))^2 exp(1 - (r/R)^2).
    The nearest periodic images of the perturbation are summed.
    """
    x = p[:, 0] - u_inf[0] * t
    y = p[:, 1] - u_inf[1] * t
    du = np.zeros(p.shape[0])
    dv = np.zeros(p.shape[0])
    dT = np.zeros(p.shape[0])
    amp = beta / (2 * np.pi)
    for a in range(-images, images + 1):
        for b in range(-images, images + 1):
            dx = np.mod(x - centre[0] + 0.5, 1.0) - 0.5 + a
            dy = np.mod(y - centre[1] + 0.5, 1.0) - 0.5 + b
            s2 = (dx * dx + dy * dy) / R ** 2
            e = np.exp(0.5 * (1.0 - s2))
            du += -amp * (dy / R) * e
            dv += amp * (dx / R) * e
            dT += -(gamma - 1) / (2 * gamma) * amp ** 2 * e * e
    T = 1.0 + dT
    rho = T ** (1.0 / (gamma - 1))
    pres = rho * T
    u = u_inf[0] + du
    v = u_inf[1] + dv
    if dim == 2:
        E = pres / (gamma - 1) + 0.5 * rho * (u * u + v * v)
        return np.stack([rho, rho * u, rho * v, E], axis=1)
    w = np.full_like(u, u_inf[2])
    E = pres / (gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E], axis=1)


def fourier_modes(seed, n_modes=4, kmax=4, dim=2):
    """Seeded sum of n_modes Fourier modes with integer wave vectors in [1,kmax]^dim,
    phases U(0, 2 pi) and amplitudes with sum |A_q| <= 1."""
    rng = np.random.default_rng(seed)
    k = rng.integers(1, kmax + 1, size=(n_modes, dim))
    th = rng.uniform(0, 2 * np.pi, size=n_modes)
    A = rng.uniform(-1, 1, size=n_modes)
    A = A / max(1.0, np.abs(A).sum())

    def f(p):
        ph = 2 * np.pi * (p @ k.T) + th
        return (A * np.sin(ph)).sum(axis=1)
    f.params = dict(k=k, theta=th, A=A)
    return f


def riemann_quadrants(seed, centre=(0.5, 0.5)):
    """Seeded four-quadrant Riemann data: rho, p in U[0.1, 2], u, v in U[-1, 1]
    per quadrant.  Returns a function giving primitive (rho, u, v, p)."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 2.0, size=4)
    u = rng.uniform(-1.0, 1.0, size=4)
    v = rng.uniform(-1.0, 1.0, size=4)
    pr = rng.uniform(0.1, 2.0, size=4)

    def f(p):
        q = (p[:, 0] >= centre[0]).astype(int) + 2 * (p[:, 1] >= centre[1]).astype(int)
        return np.stack([rho[q], u[q], v[q], pr[q]], axis=1)
    f.params = dict(rho=rho, u=u, v=v, p=pr)
    return f


def prim_to_cons(prim, gamma=1.4):
    """(rho, u, v[, w], p) -> (rho, rho u, rho v[, rho w], E), rows are points."""
    rho = prim[:, 0]
    vel = prim[:, 1:-1]
    p = prim[:, -1]
    E = p / (gamma - 1) + 0.5 * rho * (vel * vel).sum(axis=1)
    return np.concatenate([rho[:, None], rho[:, None] * vel, E[:, None]], axis=1)


# ----------------------------------------------------------------------------------------
# laminar flat-plate boundary layer (Blasius)

_BLASIUS = {}


def _blasius_table(eta_max=12.0, n=24000):
    """f(eta), f'(eta) of f''' + f f'' / 2 = 0, f(0) = f'(0) = 0, f'(inf) = 1, by
    classical RK4 on a uniform eta grid and bisection on f''(0)."""
    if "tab" in _BLASIUS:
        return _BLASIUS["tab"]
    h = eta_max / n

    def integrate(s, keep=False):
        y = np.array([0.0, 0.0, s])
        rhs = lambda y: np.array([y[1], y[2], -0.5 * y[0] * y[2]])
        out = [y.copy()] if keep else None
        for _ in range(n):
            k1 = rhs(y)
            k2 = rhs(y + 0.5 * h * k1)
            k3 = rhs(y + 0.5 * h * k2)
            k4 = rhs(y + h * k3)
            y = y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
            if keep:
                out.append(y.copy())
        return (np.array(out) if keep else y)

    lo, hi = 0.2, 0.5
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if integrate(mid)[1] > 1.0:
            hi = mid
        else:
            lo = mid
    s = 0.5 * (lo + hi)
    Y = integrate(s, keep=True)
    eta = np.linspace(0.0, eta_max, n + 1)
    _BLASIUS["tab"] = (eta, Y[:, 0], Y[:, 1], Y[:, 2], s)
    return _BLASIUS["tab"]


def _hermite(x, xt, y, dy):
    """Cubic Hermite interpolation on the uniform grid xt (values y, slopes dy)."""
    h = xt[1] - xt[0]
    i = np.clip(((x - xt[0]) / h).astype(np.int64), 0, xt.shape[0] - 2)
    t = (x - xt[i]) / h
    h00, h10 = 2 * t**3 - 3 * t**2 + 1, t**3 - 2 * t**2 + t
    h01, h11 = -2 * t**3 + 3 * t**2, t**3 - t**2
    return h00 * y[i] + h10 * h * dy[i] + h01 * y[i + 1] + h11 * h * dy[i + 1]


def blasius(p, nu=1e-3, U=1.0, x0=0.0):
    """Velocity (u, v) of the Blasius boundary layer over a plate along y = 0 starting
    at x = x0: u = U f'(eta), v = (1/2) sqrt(nu U / x) (eta f' - f),
    eta = y sqrt(U / (nu x)).  Rows are points; returns [P, 2]."""
    eta_t, f_t, fp_t, fpp_t, _ = _blasius_table()
    x = p[:, 0] - x0
    eta = p[:, 1] * np.sqrt(U / (nu * x))
    e = np.clip(eta, 0.0, eta_t[-1])
    f = _hermite(e, eta_t, f_t, fp_t) + np.where(eta > eta_t[-1], eta - eta_t[-1], 0.0)
    fp = np.where(eta > eta_t[-1], 1.0, _hermite(e, eta_t, fp_t, fpp_t))
    u = U * fp
    v = 0.5 * np.sqrt(nu * U / x) * (eta * fp - f)
    return np.stack([u, v], axis=1)
