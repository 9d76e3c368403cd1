"""The five synthetic workloads (mesh + initial cell averages + scheme + time step).

  adv2d_tri64        64x64 split quads (8192 triangles), +-20% jitter, periodic;
                     u0 = sin(2 pi x) sin(2 pi y), a = (1, 1); USR3 with differentials
                     through order 2, upwind flux, SSP-RK3 at CFL 0.5, 100 steps, FP64.
  euler3d_tet64      64^3 hexes x 5 tetrahedra (1,310,720 cells), +-15% jitter, periodic;
                     isentropic vortex (gamma 1.4), Rusanov flux; scheme orders 2/3/4
                     = stencils (2,1)/(3,1)/(4,1) with differentials through order 1/2/3.
  adv3d_hexprism     N^3 hexes, the x < 1/2 half split into prisms (1.5 N^3 cells),
                     +-20% jitter, periodic; Gaussian pulse sigma 0.1, a = (1,1,1);
                     orders 2..5 = stencils (2,1)/(3,1)/(4,1)/(5,2), differentials
                     through order p-1.
  euler2d_riemann    ~724^2 split quads (~1.05M triangles), +-20% jitter, zero-gradient
                     boundaries; seeded four-quadrant Riemann data.
  burgers_batch      512 periodic jittered triangle meshes, log-uniform 2k..200k cells,
                     u0 = seeded sum of 4 Fourier modes; Burgers flux; USR3, order 2.

Seeds are 20240414 + the workload index (+ mesh index within the batch).
Time steps come from the lattice spacing h and the initial data's largest wave
speed (no mesh geometry): dt = CFL * h * c_cell / lambda_max with the stated
per-family factor c_cell.
"""
import numpy as np

from . import fields, meshes

SEED = 20240414
WORKLOADS = ("adv2d_tri64", "euler3d_tet64", "adv3d_hexprism", "euler2d_riemann", "burgers_batch")
STENCIL_OF_ORDER = {2: (2, 1), 3: (3, 1), 4: (4, 1), 5: (5, 2)}


def _lam_euler(prim_fn, dim, n=64):
    g = np.linspace(0, 1, n, endpoint=False) + 0.5 / n
    if dim == 2:
        X, Y = np.meshgrid(g, g, indexing="ij")
        p = np.stack([X.ravel(), Y.ravel()], axis=1)
    else:
        X, Y = np.meshgrid(g, g, indexing="ij")
        p = np.stack([X.ravel(), Y.ravel(), np.full(X.size, 0.5)], axis=1)
    U = prim_fn(p)
    rho = U[:, 0]
    vel = U[:, 1:dim + 1] / rho[:, None]
    E = U[:, -1]
    pr = 0.4 * (E - 0.5 * rho * (vel * vel).sum(1))
    c = np.sqrt(1.4 * pr / rho)
    return float((np.abs(vel).sum(1) + np.sqrt(dim) * c).max())


def workload(name, order=None, size=None, q=3, n_meshes=None, workers=1):
    """Returns dict(mesh, u0 [nv, n_cells] caller order, scheme kwargs, dt, steps, info).
    workers > 1 forks processes for the initial averages (only before CUDA is initialised)."""
    if name == "adv2d_tri64":
        n = size or 64
        m = meshes.tri_mesh(n, n, jitter=0.2, seed=SEED + 0)
        u0 = fields.cell_average(m, fields.sine2d, q=q, workers=workers)[None]
        h = 1.0 / n
        dt = 0.5 * h / 2.0                        # CFL 0.5 on |a|_1 = 2
        return dict(mesh=m, u0=u0, dt=dt, steps=100,
                    scheme=dict(k=3, r=1, n_diff=2, flux="upwind", nv=1, adv=(1.0, 1.0, 0.0)),
                    info=dict(cells=2 * n * n, h=h))
    if name == "euler3d_tet64":
        n = size or 64
        order = order or 3
        k, r = STENCIL_OF_ORDER[order]
        m = meshes.tet_mesh(n, jitter=0.15, seed=SEED + 1)
        vf = lambda p: fields.isentropic_vortex(p, dim=3, images=0)
        u0 = fields.cell_average(m, vf, q=q, workers=workers, nv=5)
        h = 1.0 / n
        lam = _lam_euler(vf, 3)
        dt = 0.3 * (h / 4.0) / lam               # tetrahedra of the 5-split: width ~ h/4
        return dict(mesh=m, u0=u0, dt=dt, steps=10,
                    scheme=dict(k=k, r=r, n_diff=order - 1, flux="rusanov", nv=5, gamma=1.4),
                    info=dict(cells=5 * n ** 3, h=h, order=order))
    if name == "adv3d_hexprism":
        n = size or 140
        order = order or 5
        k, r = STENCIL_OF_ORDER[order]
        m = meshes.hexprism_mesh(n, jitter=0.2, seed=SEED + 2)
        u0 = fields.cell_average(m, fields.gaussian3d, q=q, workers=workers)[None]
        h = 1.0 / n
        dt = 0.3 * (h / 2.0) / 3.0
        return dict(mesh=m, u0=u0, dt=dt, steps=10,
                    scheme=dict(k=k, r=r, n_diff=order - 1, flux="upwind", nv=1, adv=(1.0, 1.0, 1.0)),
                    info=dict(cells=int(m["cell_face_offsets"].shape[0] - 1), h=h, order=order))
    if name == "euler2d_riemann":
        n = size or 724
        m = meshes.tri_mesh(n, n, jitter=0.2, seed=SEED + 3, boundary="transmissive")
        rq = fields.riemann_quadrants(SEED + 3 + (order or 0))
        cons = lambda p: fields.prim_to_cons(rq(p))
        u0 = fields.cell_average(m, cons, q=q, workers=workers, nv=4)
        h = 1.0 / n
        lam = _lam_euler(cons, 2)
        dt = 0.3 * (h / 3.0) / lam
        return dict(mesh=m, u0=u0, dt=dt, steps=10,
                    scheme=dict(k=3, r=1, n_diff=2, flux="rusanov", nv=4, gamma=1.4),
                    info=dict(cells=2 * n * n, h=h, quadrants=rq.params))
    if name == "burgers_batch":
        rng = np.random.default_rng(SEED + 4)
        nm = n_meshes or 512
        cells = np.exp(rng.uniform(np.log(2000), np.log(200000), size=nm))
        out = []
        for i in range(nm):
            nn = max(4, int(round(np.sqrt(cells[i] / 2))))
            m = meshes.tri_mesh(nn, nn, jitter=0.2, seed=SEED + 4 + i)
            f = fields.fourier_modes(SEED + 4 + i)
            u0 = fields.cell_average(m, f, q=q, workers=workers)[None]
            h = 1.0 / nn
            dt = 0.3 * (h / 3.0) / 2.0
            out.append(dict(mesh=m, u0=u0, dt=dt))
        return dict(meshes=out, steps=10,
                    scheme=dict(k=3, r=1, n_diff=2, flux="burgers", nv=1),
                    info=dict(n_meshes=nm, cells=int(sum(2 * max(4, int(round(np.sqrt(c / 2)))) ** 2
                                                         for c in cells))))
    raise KeyError(name)
