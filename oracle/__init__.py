"""FP64 CPU oracle of the DOLINC stage (arXiv 2404.08952) — test infrastructure.

Only tests, the smoke check and the benchmark's CPU-baseline leg use this package.
It compiles `dolinc_oracle.c` with the host C compiler into `oracle/_build/` and
calls it through ctypes.  It imports nothing from the CUDA library's package.
"""
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = [os.path.join(_HERE, "dolinc_oracle.c"), os.path.join(_HERE, "indicator_oracle.c")]
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

FLUX = {"upwind": 0, "burgers": 1, "rusanov": 2}


def _compile(out, extra, force):
    srcs = [s for s in _SRC if os.path.exists(s)]
    stale = force or not os.path.exists(out) or any(os.path.getmtime(s) > os.path.getmtime(out) for s in srcs)
    if stale:
        tmp = out + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared"] + extra + ["-o", tmp] + srcs + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def build(force=False):
    """Compile the oracle shared library (plain C, -O2, no machine-specific flags) and
    its OpenMP build (the same source with -fopenmp: face fluxes on every thread)."""
    os.makedirs(_BUILD, exist_ok=True)
    try:
        _compile(_LIB_OMP, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError) as e:     # no OpenMP: the plain build still serves
        print("oracle: OpenMP build failed (%s)" % e)
    return _compile(_LIB, [], force)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


def lib_omp():
    """The OpenMP build (threads from OMP_NUM_THREADS, default all cores)."""
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            os.makedirs(_BUILD, exist_ok=True)
            _lib_omp = C.CDLL(_compile(_LIB_OMP, ["-fopenmp"], False))
            _declare(_lib_omp)
    return _lib_omp


def threads(parallel=True):
    """Threads the (OpenMP) oracle computes face fluxes on."""
    return int((lib_omp() if parallel else lib()).or_threads())


class _Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_nodes", C.c_long), ("n_cells", C.c_long), ("n_faces", C.c_long),
                ("nodes", C.c_void_p), ("face_node_off", C.c_void_p), ("face_nodes", C.c_void_p),
                ("owner", C.c_void_p), ("neigh", C.c_void_p), ("shift", C.c_void_p)]


class _Geom(C.Structure):
    _fields_ = [("V", C.c_void_p), ("xc", C.c_void_p), ("S", C.c_void_p), ("xf", C.c_void_p),
                ("w", C.c_void_p), ("d", C.c_void_p), ("Minv", C.c_void_p), ("sdelta", C.c_void_p)]


class _Scheme(C.Structure):
    _fields_ = [("nv", C.c_int), ("k", C.c_int), ("r", C.c_int), ("n_diff", C.c_int), ("flux", C.c_int),
                ("gamma", C.c_double), ("adv", C.c_double * 3), ("eno", C.c_int), ("troubled", C.c_void_p),
                ("bkind", C.c_void_p), ("bval", C.c_void_p)]


def _declare(L):
    P = C.c_void_p
    L.or_geometry.argtypes = [P, P]
    L.or_differentials.argtypes = [P, P, C.c_int, C.c_int, P, P]
    L.or_differentials_bc.argtypes = [P, P, C.c_int, C.c_int, P, P, P, P]
    L.or_gauss_pass.argtypes = [P, P, C.c_int, C.c_int, P, P, P, P]
    L.or_skew_geometry.argtypes = [P, P]
    L.or_coeff.argtypes = [C.c_int, C.c_int, C.c_double, P]
    L.or_phantoms.argtypes = [C.c_int, C.c_double, P, P, P]
    L.or_face_values.argtypes = [P, P, P, P, P, P, P, P]
    L.or_residual_T.argtypes = [P, P, P, P, P]
    L.or_residual.argtypes = [P, P, P, P, P]
    L.or_rk3_step.argtypes = [P, P, P, C.c_double, P]
    L.or_rk3_stage.argtypes = [P, P, P, C.c_double, C.c_int, P, P, P]
    L.or_face_weights.argtypes = [P, P, P, P, P]
    L.or_weno5_parts.argtypes = [C.c_double, P, P, P, P]
    L.or_num_flux.argtypes = [C.c_int, P, P, P, P, P]
    L.or_threads.argtypes = []
    L.or_criterion.argtypes = [P, P, P, P, C.c_double, C.c_double, P]
    L.or_indicator_features.argtypes = [P, P, P, P, C.c_double, P, P]


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def coeff(k, r, g):
    """Eq coeff weights c_rj (j = 0..k-1) on cells growing by g."""
    c = np.zeros(k)
    if lib().or_coeff(k, r, float(g), _ptr(c)) != 0:
        raise ValueError("bad stencil")
    return c


def phantoms(N, g, phi0, phi1):
    """phi_n^(0), n = -N..N+1, from the two face cells' differentials (Eq diffDLC)."""
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    phi1 = np.ascontiguousarray(phi1, dtype=np.float64)
    out = np.zeros(2 * N + 2)
    if lib().or_phantoms(N, float(g), _ptr(phi0), _ptr(phi1), _ptr(out)) != 0:
        raise ValueError("bad order")
    return out


def weno5_parts(g, ph):
    """WENO5-DOLINC pieces at growth rate g from the five values ph = phi_n, n = -2..2:
    (q, d, beta), each [3] over the candidates r = 0, 1, 2 (cells i-r .. i-r+2):
    candidate face values, linear weights, smoothness measures."""
    ph = np.ascontiguousarray(ph, dtype=np.float64)
    assert ph.shape == (5,)
    q, d, beta = np.zeros(3), np.zeros(3), np.zeros(3)
    if lib().or_weno5_parts(float(g), _ptr(ph), _ptr(q), _ptr(d), _ptr(beta)) != 0:
        raise ValueError("g must be positive")
    return q, d, beta


def num_flux(dim, scheme, UL, UR, S):
    """The oracle's numerical flux through the area vector S (owner -> neighbour) from
    the two reconstructed states (scheme gives flux, gamma, adv, nv)."""
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    UR = np.ascontiguousarray(UR, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    F = np.zeros(scheme.nv)
    s = scheme._c()
    if lib().or_num_flux(int(dim), C.byref(s), _ptr(UL), _ptr(UR), _ptr(S), _ptr(F)) != 0:
        raise ValueError("bad dimension or variable count")
    return F


class Scheme:
    """Scheme parameters.  Stencil (k, r): k cells starting at i-r.
    n_diff: differential orders computed (>= what the stencil needs)."""

    def __init__(self, k=3, r=1, n_diff=None, flux="upwind", nv=1, gamma=1.4, adv=(1.0, 1.0, 0.0), eno=0,
                 troubled=None, bkind=None, bval=None):
        """bkind [n_faces] int (0/1 zero-gradient, 2 Dirichlet, 3 Neumann) and bval
        [nv, n_faces] (face value, or outward normal gradient) describe the boundary
        faces (Sec 2.6); None: every boundary face zero-gradient."""
        need = max(r, k - r - 2)
        if eno in (1, 2, 4, 5):
            need = max(need, 2)
        self.k, self.r = k, r
        self.n_diff = need if n_diff is None else n_diff
        if self.n_diff < need:
            raise ValueError("stencil (k=%d, r=%d) needs differentials through order %d" % (k, r, need))
        self.flux, self.nv, self.gamma = flux, nv, gamma
        self.adv = tuple(float(a) for a in adv) + (0.0,) * (3 - len(adv))
        self.eno = eno
        self.troubled = None if troubled is None else np.ascontiguousarray(troubled, dtype=np.uint8)
        self.bkind = None if bkind is None else np.ascontiguousarray(bkind, dtype=np.int32)
        self.bval = None if bval is None else np.ascontiguousarray(np.atleast_2d(bval), dtype=np.float64)
        if (self.bkind is None) != (self.bval is None):
            raise ValueError("bkind and bval go together")

    def _c(self):
        s = _Scheme()
        s.nv, s.k, s.r, s.n_diff, s.flux = self.nv, self.k, self.r, self.n_diff, FLUX[self.flux]
        s.gamma = self.gamma
        for i in range(3):
            s.adv[i] = self.adv[i]
        s.eno = self.eno
        s.troubled = _ptr(self.troubled) if self.troubled is not None else None
        s.bkind = _ptr(self.bkind) if self.bkind is not None else None
        s.bval = _ptr(self.bval) if self.bval is not None else None
        return s


class Oracle:
    """Geometry plus the stage operators of one mesh (dict from `synth`).
    parallel=True uses the OpenMP build (same results, face fluxes on every thread).
    skew=True applies the skewness correction (or_skew_geometry) in every operator."""

    def __init__(self, mesh, parallel=False, skew=False):
        self._L = lib_omp() if parallel else lib()
        self.dim = int(mesh["dim"])
        self._keep = {}
        for key, dt in (("nodes", np.float64), ("face_node_offsets", np.int64), ("face_nodes", np.int64),
                        ("face_owner", np.int64), ("face_neighbour", np.int64),
                        ("face_periodic_shift", np.float64)):
            self._keep[key] = np.ascontiguousarray(mesh[key], dtype=dt)
        k = self._keep
        self.n_cells = int(mesh["cell_face_offsets"].shape[0] - 1)
        self.n_faces = int(k["face_owner"].shape[0])
        m = _Mesh()
        m.dim = self.dim
        m.n_nodes, m.n_cells, m.n_faces = k["nodes"].shape[0], self.n_cells, self.n_faces
        m.nodes, m.face_node_off, m.face_nodes = _ptr(k["nodes"]), _ptr(k["face_node_offsets"]), _ptr(k["face_nodes"])
        m.owner, m.neigh, m.shift = _ptr(k["face_owner"]), _ptr(k["face_neighbour"]), _ptr(k["face_periodic_shift"])
        self._m = m
        nc, nf = self.n_cells, self.n_faces
        self.V = np.zeros(nc)
        self.xc = np.zeros((nc, 3))
        self.S = np.zeros((nf, 3))
        self.xf = np.zeros((nf, 3))
        self.w = np.zeros(nf)
        self.d = np.zeros((nf, 3))
        g = _Geom()
        g.V, g.xc, g.S, g.xf, g.w, g.d = (_ptr(a) for a in (self.V, self.xc, self.S, self.xf, self.w, self.d))
        self._g = g
        if self._L.or_geometry(C.byref(m), C.byref(g)) != 0:
            raise MemoryError("oracle geometry")
        self.Minv = self.sdelta = None
        if skew:
            self._skew()
        self.owner = k["face_owner"]
        self.neigh = k["face_neighbour"]

    def _skew(self):
        self.Minv = np.zeros((self.n_cells, 3, 3))
        self.sdelta = np.zeros((self.n_faces, 3))
        self._g.Minv, self._g.sdelta = _ptr(self.Minv), _ptr(self.sdelta)
        if self._L.or_skew_geometry(C.byref(self._m), C.byref(self._g)) != 0:
            raise ValueError("singular skewness matrix")

    @classmethod
    def from_geometry(cls, dim, owner, neigh, shift, V, xc, S, xf, w, d, parallel=False):
        """An oracle over given topology and geometry (no geometry computed): faces
        owner -> neigh (-1 boundary) with periodic translations shift [n_faces][dim]
        (or None), and the per-cell / per-face arrays of another Oracle's geometry.
        Only the stage operators that take geometry from these arrays are meaningful."""
        self = cls.__new__(cls)
        self._L = lib_omp() if parallel else lib()
        self.dim = int(dim)
        nc, nf = int(np.asarray(V).shape[0]), int(np.asarray(owner).shape[0])
        self.n_cells, self.n_faces = nc, nf
        k = {"face_owner": np.ascontiguousarray(owner, dtype=np.int64),
             "face_neighbour": np.ascontiguousarray(neigh, dtype=np.int64),
             "face_periodic_shift": (np.ascontiguousarray(shift, dtype=np.float64) if shift is not None
                                     else np.zeros((nf, dim))),
             "nodes": np.zeros((1, dim)), "face_node_offsets": np.zeros(nf + 1, dtype=np.int64),
             "face_nodes": np.zeros(1, dtype=np.int64)}
        self._keep = k
        m = _Mesh()
        m.dim, m.n_nodes, m.n_cells, m.n_faces = self.dim, 1, nc, nf
        m.nodes, m.face_node_off, m.face_nodes = _ptr(k["nodes"]), _ptr(k["face_node_offsets"]), _ptr(k["face_nodes"])
        m.owner, m.neigh, m.shift = _ptr(k["face_owner"]), _ptr(k["face_neighbour"]), _ptr(k["face_periodic_shift"])
        self._m = m
        self.V, self.xc, self.S, self.xf, self.w, self.d = (np.ascontiguousarray(a, dtype=np.float64).copy()
                                                            for a in (V, xc, S, xf, w, d))
        g = _Geom()
        g.V, g.xc, g.S, g.xf, g.w, g.d = (_ptr(a) for a in (self.V, self.xc, self.S, self.xf, self.w, self.d))
        self._g = g
        self.Minv = self.sdelta = None
        self.owner, self.neigh = k["face_owner"], k["face_neighbour"]
        return self

    def gauss_pass(self, T_prev, m, scheme=None):
        """Order m (>= 1) full tensors [nv, n_cells, dim**m] from order m-1 [nv, n_cells, dim**(m-1)]
        (one pass of the differentials; scheme supplies the boundary conditions)."""
        T_prev = np.ascontiguousarray(T_prev, dtype=np.float64)
        nv = T_prev.shape[0]
        out = np.zeros((nv, self.n_cells, self.dim ** m))
        bk = _ptr(scheme.bkind) if scheme is not None and scheme.bkind is not None else None
        bv = _ptr(scheme.bval) if scheme is not None and scheme.bval is not None else None
        if self._L.or_gauss_pass(C.byref(self._m), C.byref(self._g), nv, int(m), _ptr(T_prev), _ptr(out), bk, bv):
            raise ValueError("bad order")
        return out

    def residual_T(self, T, scheme):
        """Residual from given differentials T (list over orders 0..n_diff of [nv, n_cells, dim**m])."""
        flat = np.ascontiguousarray(np.concatenate([np.asarray(t, dtype=np.float64).ravel() for t in T]))
        nv = scheme.nv
        R = np.zeros((nv, self.n_cells))
        s = scheme._c()
        if self._L.or_residual_T(C.byref(self._m), C.byref(self._g), C.byref(s), _ptr(flat), _ptr(R)) != 0:
            raise MemoryError
        return R

    # differentials: list of arrays, order m -> [nv, n_cells, dim**m]
    def differentials(self, u, N, nv=None, scheme=None):
        """scheme (optional) supplies the boundary conditions (Scheme bkind/bval)."""
        u = np.ascontiguousarray(np.atleast_2d(u), dtype=np.float64)
        nv = u.shape[0]
        D = self.dim
        sizes = [nv * self.n_cells * D ** m for m in range(N + 1)]
        T = np.zeros(sum(sizes))
        if scheme is not None and scheme.bkind is not None:
            self._L.or_differentials_bc(C.byref(self._m), C.byref(self._g), nv, N, _ptr(u), _ptr(scheme.bkind),
                                      _ptr(scheme.bval), _ptr(T))
        else:
            self._L.or_differentials(C.byref(self._m), C.byref(self._g), nv, N, _ptr(u), _ptr(T))
        out, o = [], 0
        for m in range(N + 1):
            out.append(T[o:o + sizes[m]].reshape(nv, self.n_cells, D ** m))
            o += sizes[m]
        return out, T

    def face_values(self, u, scheme):
        """(phiL, phiR, rL, rR): [nv, n_faces] owner-upwind / neighbour-upwind states
        and the ENO3 stencil offsets chosen (-1 on boundary faces)."""
        _, T = self.differentials(u, scheme.n_diff, scheme=scheme)
        nv = scheme.nv
        L = np.zeros((nv, self.n_faces))
        R = np.zeros((nv, self.n_faces))
        rL = np.zeros((nv, self.n_faces), dtype=np.int32)
        rR = np.zeros((nv, self.n_faces), dtype=np.int32)
        s = scheme._c()
        self._L.or_face_values(C.byref(self._m), C.byref(self._g), C.byref(s), _ptr(T), _ptr(L), _ptr(R),
                             _ptr(rL), _ptr(rR))
        return L, R, rL, rR

    def face_weights(self, scheme):
        """DOLINC representation weights per face: (WL, WR) each [n_faces, 2, n_diff+1]
        (upwind cell's W0[m], downwind cell's W1[m])."""
        nw = 2 * (scheme.n_diff + 1)
        WL = np.zeros((self.n_faces, nw))
        WR = np.zeros((self.n_faces, nw))
        s = scheme._c()
        self._L.or_face_weights(C.byref(self._m), C.byref(self._g), C.byref(s), _ptr(WL), _ptr(WR))
        return WL.reshape(self.n_faces, 2, -1), WR.reshape(self.n_faces, 2, -1)

    def criterion(self, u, scheme, kappa=4.0, eps=1e-3):
        """Troubled-cell flags [n_cells] (uint8) of the criterion in indicator_oracle.c."""
        _, T = self.differentials(u, scheme.n_diff, scheme=scheme)
        flags = np.zeros(self.n_cells, dtype=np.uint8)
        s = scheme._c()
        if self._L.or_criterion(C.byref(self._m), C.byref(self._g), C.byref(s), _ptr(T), float(kappa), float(eps),
                              _ptr(flags)) != 0:
            raise ValueError("criterion needs Euler with n_diff >= 2")
        return flags

    def features(self, u, scheme, tiny=1e-6):
        """(own [n_cells, 6], x [n_cells, 24]) network inputs of indicator_oracle.c."""
        _, T = self.differentials(u, scheme.n_diff, scheme=scheme)
        own = np.zeros((self.n_cells, 6))
        x = np.zeros((self.n_cells, 24))
        s = scheme._c()
        if self._L.or_indicator_features(C.byref(self._m), C.byref(self._g), C.byref(s), _ptr(T), float(tiny),
                                       _ptr(own), _ptr(x)) != 0:
            raise MemoryError
        return own, x

    def residual(self, u, scheme):
        u = np.ascontiguousarray(np.atleast_2d(u), dtype=np.float64)
        R = np.zeros_like(u)
        s = scheme._c()
        if self._L.or_residual(C.byref(self._m), C.byref(self._g), C.byref(s), _ptr(u), _ptr(R)) != 0:
            raise MemoryError
        return R

    def rk3_step(self, u, scheme, dt):
        u = np.array(np.atleast_2d(u), dtype=np.float64, order="C")
        s = scheme._c()
        if self._L.or_rk3_step(C.byref(self._m), C.byref(self._g), C.byref(s), float(dt), _ptr(u)) != 0:
            raise MemoryError
        return u

    def rk3_stage(self, u0, us, scheme, dt, stage):
        u0 = np.ascontiguousarray(np.atleast_2d(u0), dtype=np.float64)
        us = np.ascontiguousarray(np.atleast_2d(us), dtype=np.float64)
        out = np.zeros_like(us)
        s = scheme._c()
        if self._L.or_rk3_stage(C.byref(self._m), C.byref(self._g), C.byref(s), float(dt), int(stage),
                              _ptr(u0), _ptr(us), _ptr(out)) != 0:
            raise MemoryError
        return out

    def run(self, u, scheme, dt, steps):
        for _ in range(steps):
            u = self.rk3_step(u, scheme, dt)
        return u

    # ------------------------------------------------------------ semi-implicit step
    # Sec 2.4 (Eq USR3, Eq CSR4): a DOLINC face value splits into the weight part of the
    # two face cells and a remainder,  phi_f = w_s phi_up + (1 - w_s) phi_down + c_r,
    # w_s the weight of the upwind cell; under an implicit time integration the weight
    # part enters the matrix and c_r (the inverted far-field data) stays explicit, a
    # semi-implicit scheme.  Linear advection (flux "upwind", one variable) on meshes
    # whose boundary faces are zero-gradient.

    def _split_faces(self, scheme):
        if scheme.flux != "upwind" or scheme.nv != 1:
            raise ValueError("the semi-implicit step is for linear advection (flux 'upwind', nv = 1)")
        if scheme.bkind is not None and np.any(np.isin(scheme.bkind[self.neigh < 0], (2, 3))):
            raise ValueError("the semi-implicit step takes zero-gradient boundary faces only")
        D = self.dim
        an = self.S[:, :D] @ np.asarray(scheme.adv[:D], dtype=np.float64)     # a . S_f, owner -> neighbour
        WL, WR = self.face_weights(scheme)
        P, Q = self.owner, self.neigh
        bnd = Q < 0
        own_up = an >= 0.0
        # weights of the owner's and the neighbour's averages in the upwind face value
        cP = np.where(bnd, 1.0, np.where(own_up, WL[:, 0, 0], WR[:, 1, 0]))
        cQ = np.where(bnd, 0.0, np.where(own_up, WL[:, 1, 0], WR[:, 0, 0]))
        return an, P, np.where(bnd, P, Q), bnd, cP, cQ

    def implicit_operator(self, scheme):
        """K (scipy CSR, n_cells x n_cells): (K u)_c is the sum over the faces of c of
        the outward flux a.S (w_s u_up + (1 - w_s) u_down), the weight part of every
        face value (boundary faces: a.S u_c)."""
        import scipy.sparse as sp
        an, P, Q, bnd, cP, cQ = self._split_faces(scheme)
        it = ~bnd
        rows = np.concatenate([P, P, Q[it], Q[it]])
        cols = np.concatenate([P, Q, P[it], Q[it]])
        vals = np.concatenate([an * cP, an * cQ, -(an * cP)[it], -(an * cQ)[it]])
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n_cells, self.n_cells))

    def explicit_correction(self, u, scheme):
        """C(u) (n_cells): the sum over the faces of c of the outward a.S c_r, with
        c_r = phi_f - w_s u_up - (1 - w_s) u_down from the DOLINC face values of u."""
        u = np.ascontiguousarray(np.atleast_2d(u), dtype=np.float64)
        an, P, Q, bnd, cP, cQ = self._split_faces(scheme)
        phiL, phiR, _, _ = self.face_values(u, scheme)
        phi = np.where(an >= 0.0, phiL[0], phiR[0])
        Fc = an * (phi - cP * u[0, P] - cQ * u[0, Q])
        out = np.zeros(self.n_cells)
        np.add.at(out, P, Fc)
        np.add.at(out, Q[~bnd], -Fc[~bnd])
        return out

    def semi_implicit_step(self, u, scheme, dt, theta=1.0, n_outer=1):
        """One theta-scheme step with the weight part implicit and c_r explicit:
            V (u' - u) / dt = -theta K u' - (1 - theta) K u - C(u),
        solved directly (sparse LU).  n_outer > 1 repeats the solve with the c_r of the
        latest iterate taken at the new level,
            V (u^(k+1) - u) / dt = -theta K u^(k+1) - (1 - theta) (K u + C(u)) - theta C(u^(k)),
        whose fixed point is the theta scheme of the full DOLINC operator."""
        import scipy.sparse as sp
        import scipy.sparse.linalg as spl
        u = np.array(np.atleast_2d(u), dtype=np.float64)
        K = self.implicit_operator(scheme)
        A = (sp.diags(self.V / dt) + theta * K).tocsc()
        base = self.V / dt * u[0] - (1.0 - theta) * (K @ u[0] + self.explicit_correction(u, scheme))
        uk = u
        for _ in range(max(int(n_outer), 1)):
            rhs = base - theta * self.explicit_correction(uk, scheme)
            uk = spl.spsolve(A, rhs)[None, :]
        return uk
