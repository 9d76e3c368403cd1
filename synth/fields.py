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


def _simplices(mesh):
    """Signed simplices (apex first) of each cell, as (cell id, vertex coordinates)."""
    dim = mesh["dim"]
    nodes = mesh["nodes"]
    hc = mesh["_hf_cell"]
    hf = mesh["_hf_nodes"]
    n_cells = mesh["cell_face_offsets"].shape[0] - 1
    # apex: mean of each cell's distinct half-face nodes (duplicates don't matter for
    # correctness: any point gives the same signed integral)
    valid = hf >= 0
    pts = nodes[np.maximum(hf, 0)] * valid[..., None]
    cnt = np.zeros(n_cells)
    np.add.at(cnt, hc, valid.sum(axis=1))
    apex = np.zeros((n_cells, dim))
    np.add.at(apex, hc, pts.sum(axis=1))
    apex /= cnt[:, None]
    if dim == 2:
        a = nodes[hf[:, 0]]
        b = nodes[hf[:, 1]]
        verts = np.stack([apex[hc], a, b], axis=1)
        return hc, verts
    nf = valid.sum(axis=1)
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
    return np.concatenate(cells), np.concatenate(verts)


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


def cell_average(mesh, func, q=4, nv=None, chunk=1 << 18):
    """Cell averages of func over every cell.

    func maps points [P, dim] to values [P] or [P, nv].
    Returns [n_cells] or [nv, n_cells] (variables first, the library's layout).
    """
    dim = mesh["dim"]
    n_cells = mesh["cell_face_offsets"].shape[0] - 1
    cid, verts = _simplices(mesh)
    ref, wt = _duffy_rule(dim, q)
    acc = None
    vol = np.zeros(n_cells)
    for s in range(0, cid.shape[0], chunk):
        c = cid[s:s + chunk]
        v = verts[s:s + chunk]
        E = v[:, 1:, :] - v[:, :1, :]                         # edge vectors [n, dim, dim]
        det = np.linalg.det(np.transpose(E, (0, 2, 1)))       # signed measure * dim!
        pts = v[:, None, 0, :] + np.einsum("pk,nkd->npd", ref, E)
        val = np.asarray(func(pts.reshape(-1, dim)), dtype=np.float64)
        val = val.reshape(pts.shape[0], pts.shape[1], -1)
        contrib = np.einsum("npv,p,n->nv", val, wt, det)
        if acc is None:
            acc = np.zeros((n_cells, val.shape[2]))
        np.add.at(acc, c, contrib)
        np.add.at(vol, c, det * wt.sum())
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
    summing the images within `images` periods."""
    out = np.zeros(p.shape[0])
    rng = range(-images, images + 1)
    for a in rng:
        for b in rng:
            for c in rng:
                d = p - (np.asarray(centre) + np.array([a, b, c], dtype=np.float64))
                out += np.exp(-0.5 * np.einsum("ij,ij->i", d, d) / sigma ** 2)
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
