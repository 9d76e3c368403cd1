"""Python binding of libdolinc (the GB300 DOLINC stage library, include/dolinc.h).

Argument marshalling only: every step of the stage runs in the library's CUDA
kernels.  Functions keep the C names (dolinc_mesh_create, dolinc_rk_step, ...);
device buffers are torch CUDA tensors, streams are torch CUDA streams.  If the
library is not built the import still works, but every call raises: there is no
CPU fallback.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdolinc.so")

FLUX = {"upwind": 0, "burgers": 1, "rusanov": 2}
PRECISION = {"fp64": 0, "fp32": 1, "fp32_bf16": 2}
LIMITER = {"none": 0, "eno3_all": 1, "eno3_flagged": 2, "first_order_flagged": 3, "weno5_all": 4, "weno5_flagged": 5}
RENUMBER = {"none": 0, "morton": 1}
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "MESH", 3: "UNSUPPORTED", 4: "CUDA", 5: "DEVICE_TIMEOUT",
          6: "NONFINITE", 7: "OOM"}

# every entry point declared in include/dolinc.h
ABI_SYMBOLS = (
    "dolinc_mesh_create", "dolinc_mesh_destroy", "dolinc_mesh_get_info", "dolinc_mesh_permutation",
    "dolinc_mesh_geometry", "dolinc_workspace_size", "dolinc_workspace_init", "dolinc_diff_layout",
    "dolinc_differentials", "dolinc_reconstruct_faces", "dolinc_residual", "dolinc_rk_stage",
    "dolinc_rk_step", "dolinc_rk_steps", "dolinc_rk_step_host", "dolinc_set_flags", "dolinc_set_boundary_values", "dolinc_sync_status", "dolinc_profile_enable",
    "dolinc_profile_read", "dolinc_rk_step_noalloc", "dolinc_autotune", "dolinc_set_tuning",
    "dolinc_criterion", "dolinc_indicator_features", "dolinc_mlp_create", "dolinc_mlp_destroy",
    "dolinc_mlp_get_params", "dolinc_mlp_set_params", "dolinc_mlp_forward", "dolinc_mlp_loss_grad",
    "dolinc_mlp_train_step", "dolinc_indicator_infer", "dolinc_batch_create", "dolinc_batch_destroy",
    "dolinc_batch_info", "dolinc_batch_set_spin_limit", "dolinc_batch_workspace_size", "dolinc_batch_rk_step",
    "dolinc_batch_autotune", "dolinc_partition", "dolinc_part_plan", "dolinc_mesh_create_part",
    "dolinc_mesh_part_sizes", "dolinc_part_step_begin", "dolinc_part_step_continue",
    "dolinc_mesh_set_skew_correction", "dolinc_implicit_create", "dolinc_implicit_destroy",
    "dolinc_implicit_set_solver", "dolinc_implicit_step", "dolinc_implicit_info", "dolinc_implicit_rows",
    "dolinc_implicit_set_layout", "dolinc_implicit_layout",
    "dolinc_last_error",
)
KERNEL_KINDS = ("pack", "diff1", "diff2", "diff3", "diff4", "stage", "faces", "diff_pair", "solve")


class DolincError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("dolinc %s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class _Desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_nodes", C.c_int64), ("nodes", C.c_void_p), ("n_cells", C.c_int64),
                ("cell_face_offsets", C.c_void_p), ("cell_faces", C.c_void_p), ("n_faces", C.c_int64),
                ("face_node_offsets", C.c_void_p), ("face_nodes", C.c_void_p), ("face_owner", C.c_void_p),
                ("face_neighbour", C.c_void_p), ("face_periodic_shift", C.c_void_p),
                ("boundary_kind", C.c_void_p), ("renumber", C.c_int)]


class _Scheme(C.Structure):
    _fields_ = [("k", C.c_int), ("r", C.c_int), ("n_diff", C.c_int), ("flux", C.c_int), ("nv", C.c_int),
                ("precision", C.c_int), ("limiter", C.c_int), ("gamma", C.c_double), ("adv", C.c_double * 3)]


class _Info(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_cells", C.c_int64), ("n_faces", C.c_int64),
                ("n_boundary_faces", C.c_int64), ("n_slots", C.c_int64), ("g_min", C.c_double),
                ("g_max", C.c_double), ("volume", C.c_double), ("h_min", C.c_double)]


_lib = None


def load(path=LIB_PATH):
    """Load libdolinc.so; raises if it has not been built (see __graft_entry__.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libdolinc.so is not built (%s): run __graft_entry__.build()" % path)
        L = C.CDLL(path)
        P, S, I, D = C.c_void_p, C.c_size_t, C.c_int, C.c_double
        sig = {
            "dolinc_mesh_create": [P, P], "dolinc_mesh_destroy": [P], "dolinc_mesh_get_info": [P, P],
            "dolinc_mesh_permutation": [P, P], "dolinc_mesh_geometry": [P, P, P, P, P, P],
            "dolinc_workspace_size": [P, P, P], "dolinc_workspace_init": [P, S, P],
            "dolinc_diff_layout": [P, P, I, P, P, P, P],
            "dolinc_differentials": [P, P, P, I, P, P, S, P],
            "dolinc_reconstruct_faces": [P, P, P, P, P, P, S, P],
            "dolinc_residual": [P, P, P, P, P, S, P],
            "dolinc_rk_stage": [P, P, D, I, P, P, P, P, S, P],
            "dolinc_rk_step": [P, P, D, P, P, S, P], "dolinc_rk_step_host": [P, P, D, P, P, P, S, P],
            "dolinc_rk_steps": [P, P, D, I, P, P, S, P],
            "dolinc_set_flags": [P, P], "dolinc_set_boundary_values": [P, C.c_int, P],
            "dolinc_sync_status": [P, P, P], "dolinc_last_error": [],
            "dolinc_profile_enable": [P, I], "dolinc_profile_read": [P, P, P],
            "dolinc_rk_step_noalloc": [P, P, D, P, P],
            "dolinc_autotune": [P, P, P, P, S, C.c_char_p, P, P], "dolinc_set_tuning": [P, P, P],
            "dolinc_criterion": [P, P, P, P, D, D, P, S, P],
            "dolinc_indicator_features": [P, P, P, P, P, S, P],
            "dolinc_mlp_create": [P, C.c_uint64], "dolinc_mlp_destroy": [P],
            "dolinc_mlp_get_params": [P, P], "dolinc_mlp_set_params": [P, P],
            "dolinc_mlp_forward": [P, P, C.c_int64, P, P, P],
            "dolinc_mlp_loss_grad": [P, P, P, C.c_int64, C.c_float, P, P, P],
            "dolinc_mlp_train_step": [P, P, P, C.c_int64, C.c_float, C.c_float, P, P],
            "dolinc_indicator_infer": [P, P, P, P, P, P, P, P, S, P],
            "dolinc_batch_create": [P, I, P], "dolinc_batch_destroy": [P], "dolinc_batch_info": [P, P, P],
            "dolinc_batch_set_spin_limit": [P, C.c_uint], "dolinc_batch_workspace_size": [P, P, P],
            "dolinc_batch_rk_step": [P, P, P, P, P, S, I, P],
            "dolinc_batch_autotune": [P, P, P, P, P, S, P, P, P, P],
            "dolinc_partition": [P, I, P],
            "dolinc_part_plan": [P, P, I, I, P, P, P, P, P, P, P, P],
            "dolinc_mesh_create_part": [P, P, I, I, P], "dolinc_mesh_part_sizes": [P, P],
            "dolinc_part_step_begin": [P, P, D, P, P, S, P, P],
            "dolinc_part_step_continue": [P, P, P, S, P, P],
            "dolinc_mesh_set_skew_correction": [P, I],
            "dolinc_implicit_create": [P, P, D, D, P], "dolinc_implicit_destroy": [P],
            "dolinc_implicit_set_solver": [P, D, I, C.c_uint, I], "dolinc_implicit_step": [P, P, I, P, S, P],
            "dolinc_implicit_info": [P, P], "dolinc_implicit_rows": [P, P, P, P, P],
            "dolinc_implicit_set_layout": [P, I], "dolinc_implicit_layout": [P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_char_p if name == "dolinc_last_error" else (
                None if name in ("dolinc_mesh_destroy", "dolinc_mlp_destroy", "dolinc_batch_destroy",
                                "dolinc_implicit_destroy") else C.c_int)
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise DolincError(status, load().dolinc_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Scheme:
    """dolinc_scheme.  precision: 'fp64' | 'fp32' | 'fp32_bf16'; limiter: 'none' |
    'eno3_all' | 'eno3_flagged' | 'first_order_flagged' | 'weno5_all' | 'weno5_flagged'."""

    def __init__(self, k=3, r=1, n_diff=None, flux="upwind", nv=1, precision="fp64", limiter="none",
                 gamma=1.4, adv=(1.0, 1.0, 0.0)):
        need = max(r, k - r - 2, 2 if limiter in ("eno3_all", "eno3_flagged", "weno5_all", "weno5_flagged") else 1)
        self.k, self.r = k, r
        self.n_diff = need if n_diff is None else n_diff
        self.flux, self.nv, self.precision, self.limiter = flux, nv, precision, limiter
        self.gamma = gamma
        self.adv = tuple(float(a) for a in adv) + (0.0,) * (3 - len(adv))

    def c(self):
        s = _Scheme()
        s.k, s.r, s.n_diff, s.flux, s.nv = self.k, self.r, self.n_diff, FLUX[self.flux], self.nv
        s.precision, s.limiter, s.gamma = PRECISION[self.precision], LIMITER[self.limiter], self.gamma
        for i in range(3):
            s.adv[i] = self.adv[i]
        return s


class _Tuning(C.Structure):
    _fields_ = [("diff_lanes", C.c_int), ("diff_block", C.c_int), ("stage_lanes", C.c_int),
                ("stage_block", C.c_int), ("from_cache", C.c_int), ("diff_ms", C.c_double),
                ("stage_ms", C.c_double)]


def _make_desc(m, renumber):
    """dolinc_mesh_desc of a mesh dict, and the arrays it points to (keep them alive)."""
    a = {}
    for key, dt in (("nodes", np.float64), ("cell_face_offsets", np.int64), ("cell_faces", np.int64),
                    ("face_node_offsets", np.int64), ("face_nodes", np.int64), ("face_owner", np.int64),
                    ("face_neighbour", np.int64), ("face_periodic_shift", np.float64),
                    ("boundary_kind", np.int32)):
        if key in m and m[key] is not None:
            a[key] = np.ascontiguousarray(m[key], dtype=dt)
    d = _Desc()
    d.dim = int(m["dim"])
    d.n_nodes = a["nodes"].shape[0]
    d.nodes = _ptr(a["nodes"])
    d.n_cells = a["cell_face_offsets"].shape[0] - 1
    d.cell_face_offsets = _ptr(a.get("cell_face_offsets"))
    d.cell_faces = _ptr(a.get("cell_faces"))
    d.n_faces = a["face_owner"].shape[0]
    d.face_node_offsets = _ptr(a["face_node_offsets"])
    d.face_nodes = _ptr(a["face_nodes"])
    d.face_owner = _ptr(a["face_owner"])
    d.face_neighbour = _ptr(a["face_neighbour"])
    d.face_periodic_shift = _ptr(a.get("face_periodic_shift"))
    d.boundary_kind = _ptr(a.get("boundary_kind"))
    d.renumber = RENUMBER[renumber] if isinstance(renumber, str) else int(renumber)
    return d, a


class _PartSizes(C.Structure):
    _fields_ = [("n_local", C.c_int64), ("n_owned", C.c_int64), ("n_faces", C.c_int64), ("n_peers", C.c_int32),
                ("n_send", C.c_int64), ("n_recv", C.c_int64)]


class _Halo(C.Structure):
    _fields_ = [("pending", C.c_int), ("order", C.c_int), ("record_bytes", C.c_size_t), ("send_dev", C.c_void_p),
                ("recv_dev", C.c_void_p)]


def dolinc_partition(m, n_parts):
    """Space-filling-curve partition of a mesh dict: the part of every caller cell."""
    d, keep = _make_desc(m, "morton")
    out = np.zeros(d.n_cells, dtype=np.int32)
    _check(load().dolinc_partition(C.byref(d), int(n_parts), _ptr(out)))
    return out


def dolinc_part_plan(m, part_of_cell, n_parts, part, renumber="morton"):
    """Host plan of one part: local cells (caller ids), own flags, peers and the
    per-peer send / receive lists (local indices)."""
    d, keep = _make_desc(m, renumber)
    pc = np.ascontiguousarray(part_of_cell, dtype=np.int32)
    z = _PartSizes()
    L = load()
    _check(L.dolinc_part_plan(C.byref(d), _ptr(pc), int(n_parts), int(part), C.byref(z), *([None] * 7)))
    out = dict(local_cells=np.zeros(z.n_local, dtype=np.int64), owned=np.zeros(z.n_local, dtype=np.uint8),
               peers=np.zeros(z.n_peers, dtype=np.int32), send_off=np.zeros(z.n_peers + 1, dtype=np.int64),
               send_cells=np.zeros(z.n_send, dtype=np.int64), recv_off=np.zeros(z.n_peers + 1, dtype=np.int64),
               recv_cells=np.zeros(z.n_recv, dtype=np.int64))
    _check(L.dolinc_part_plan(C.byref(d), _ptr(pc), int(n_parts), int(part), C.byref(z), _ptr(out["local_cells"]),
                              _ptr(out["owned"]), _ptr(out["peers"]), _ptr(out["send_off"]), _ptr(out["send_cells"]),
                              _ptr(out["recv_off"]), _ptr(out["recv_cells"])))
    out["n_faces"] = z.n_faces
    return out


class Mesh:
    """A library mesh handle built from a mesh dict (see synth.meshes).
    part=(part_of_cell, n_parts, p) builds part p of a partitioned mesh instead
    (dolinc_mesh_create_part): its cells are the plan's local cells (self.plan), in
    that order."""

    def __init__(self, m, renumber="morton", part=None):
        L = load()
        d, self._arrays = _make_desc(m, renumber)
        h = C.c_void_p()
        self.plan = None
        if part is None:
            _check(L.dolinc_mesh_create(C.byref(d), C.byref(h)))
        else:
            pc, n_parts, p = part
            pc = np.ascontiguousarray(pc, dtype=np.int32)
            _check(L.dolinc_mesh_create_part(C.byref(d), _ptr(pc), int(n_parts), int(p), C.byref(h)))
            self.plan = dolinc_part_plan(m, pc, n_parts, p, renumber)
        self.handle = h
        self._finish()

    def _finish(self):
        L = load()
        h = self.handle
        info = _Info()
        _check(L.dolinc_mesh_get_info(h, C.byref(info)))
        self.dim, self.n_cells, self.n_faces = info.dim, info.n_cells, info.n_faces
        self.n_boundary_faces, self.n_slots = info.n_boundary_faces, info.n_slots
        self.g_min, self.g_max, self.volume, self.h_min = info.g_min, info.g_max, info.volume, info.h_min
        perm = np.zeros(self.n_cells, dtype=np.int64)
        _check(L.dolinc_mesh_permutation(h, _ptr(perm)))
        self.perm = perm                              # library index of each caller cell
        self._arrays = None                           # the library copied what it needs

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.dolinc_mesh_destroy(h)
            self.handle = None

    def to_lib(self, u):
        """caller cell order -> library order (last axis)."""
        out = np.empty_like(u)
        out[..., self.perm] = u
        return out

    def from_lib(self, u):
        return u[..., self.perm]

    def geometry(self):
        V = np.zeros(self.n_cells)
        xc = np.zeros((self.n_cells, 3))
        S = np.zeros((self.n_faces, 3))
        w = np.zeros(self.n_faces)
        d = np.zeros((self.n_faces, 3))
        _check(load().dolinc_mesh_geometry(self.handle, _ptr(V), _ptr(xc), _ptr(S), _ptr(w), _ptr(d)))
        return dict(V=V, xc=xc, S=S, w=w, d=d)


def dolinc_mesh_set_skew_correction(mesh, enable=True):
    """Skewness correction of the mesh on or off (every scheme on the mesh)."""
    _check(load().dolinc_mesh_set_skew_correction(mesh.handle, 1 if enable else 0))


def dolinc_workspace_size(mesh, scheme):
    n = C.c_size_t()
    s = scheme.c()
    _check(load().dolinc_workspace_size(mesh.handle, C.byref(s), C.byref(n)))
    return n.value


def workspace(mesh, scheme, device="cuda", stream=None):
    """A zero-status workspace tensor (uint8, 256-byte aligned) for this mesh and scheme."""
    import torch
    n = dolinc_workspace_size(mesh, scheme)
    ws = torch.empty(n + 256, dtype=torch.uint8, device=device)
    off = (-ws.data_ptr()) % 256
    ws = ws[off:off + n]
    _check(load().dolinc_workspace_init(_ptr(ws), n, _stream(stream)))
    return ws


def dolinc_diff_layout(mesh, scheme, order):
    off = np.zeros(order, dtype=np.int64)
    stride = np.zeros(order, dtype=np.int32)
    eb = np.zeros(order, dtype=np.int32)
    tot = C.c_int64()
    s = scheme.c()
    _check(load().dolinc_diff_layout(mesh.handle, C.byref(s), order, _ptr(off), _ptr(stride), _ptr(eb),
                                     C.byref(tot)))
    return off, stride, eb, tot.value


def dolinc_differentials(mesh, scheme, u, order, diff, ws, stream=None):
    s = scheme.c()
    _check(load().dolinc_differentials(mesh.handle, C.byref(s), _ptr(u), int(order), _ptr(diff), _ptr(ws),
                                       ws.numel(), _stream(stream)))


def dolinc_reconstruct_faces(mesh, scheme, u, face_L, face_R, ws, stream=None):
    s = scheme.c()
    _check(load().dolinc_reconstruct_faces(mesh.handle, C.byref(s), _ptr(u), _ptr(face_L), _ptr(face_R),
                                           _ptr(ws), ws.numel(), _stream(stream)))


def dolinc_residual(mesh, scheme, u, R, ws, stream=None):
    s = scheme.c()
    _check(load().dolinc_residual(mesh.handle, C.byref(s), _ptr(u), _ptr(R), _ptr(ws), ws.numel(),
                                  _stream(stream)))


def dolinc_rk_stage(mesh, scheme, dt, stage, u0, us, out, ws, stream=None):
    s = scheme.c()
    _check(load().dolinc_rk_stage(mesh.handle, C.byref(s), float(dt), int(stage), _ptr(u0), _ptr(us), _ptr(out),
                                  _ptr(ws), ws.numel(), _stream(stream)))


def dolinc_rk_step(mesh, scheme, dt, u, ws, stream=None):
    s = scheme.c()
    _check(load().dolinc_rk_step(mesh.handle, C.byref(s), float(dt), _ptr(u), _ptr(ws), ws.numel(),
                                 _stream(stream)))


def dolinc_rk_steps(mesh, scheme, dt, n_steps, u, ws, stream=None):
    """n_steps SSP-RK3 steps in one call (bit-identical to n_steps dolinc_rk_step calls)."""
    s = scheme.c()
    _check(load().dolinc_rk_steps(mesh.handle, C.byref(s), float(dt), int(n_steps), _ptr(u), _ptr(ws), ws.numel(),
                                  _stream(stream)))


def dolinc_rk_step_host(mesh, scheme, dt, u_host, u_dev, ws, stream=None):
    """One SSP-RK3 step of the FP64 state u_host (a CPU tensor or array, updated in
    place; pinned memory is read and written by the step's kernels directly), with
    u_dev a device scratch tensor of the same size.  Asynchronous on the stream."""
    s = scheme.c()
    _check(load().dolinc_rk_step_host(mesh.handle, C.byref(s), float(dt), _ptr(u_host), _ptr(u_dev), _ptr(ws),
                                      ws.numel(), _stream(stream)))


def dolinc_rk_step_noalloc(mesh, scheme, dt, u, stream=None):
    """One SSP-RK3 step using the library's fixed internal workspace (no allocation;
    see include/dolinc.h for its size limit and sharing rules)."""
    s = scheme.c()
    _check(load().dolinc_rk_step_noalloc(mesh.handle, C.byref(s), float(dt), _ptr(u), _stream(stream)))


def dolinc_autotune(mesh, scheme, u, ws, cache_path=None, stream=None):
    """Pick lanes-per-cell and block sizes for this mesh and scheme by timing them on u;
    returns the chosen shape as a dict."""
    s = scheme.c()
    t = _Tuning()
    cp = cache_path.encode() if cache_path else None
    _check(load().dolinc_autotune(mesh.handle, C.byref(s), _ptr(u), _ptr(ws), ws.numel(), cp, _stream(stream),
                                  C.byref(t)))
    return {f: getattr(t, f) for f, _ in _Tuning._fields_}


def dolinc_set_tuning(mesh, scheme, diff_lanes=4, diff_block=256, stage_lanes=4, stage_block=128):
    s = scheme.c()
    t = _Tuning()
    t.diff_lanes, t.diff_block, t.stage_lanes, t.stage_block = diff_lanes, diff_block, stage_lanes, stage_block
    _check(load().dolinc_set_tuning(mesh.handle, C.byref(s), C.byref(t)))


def dolinc_set_boundary_values(mesh, values):
    """values [nv, n_faces] (caller face order): Dirichlet face values / Neumann outward
    normal gradients of the faces whose boundary_kind is 2 / 3."""
    v = np.ascontiguousarray(np.atleast_2d(values), dtype=np.float64)
    _check(load().dolinc_set_boundary_values(mesh.handle, int(v.shape[0]), _ptr(v)))


def dolinc_set_flags(mesh, flags):
    """The library keeps the device pointer, so the mesh object keeps the tensor alive
    until the flags are replaced or cleared (None)."""
    _check(load().dolinc_set_flags(mesh.handle, _ptr(flags)))
    mesh._flags = flags


def dolinc_sync_status(mesh, ws, stream=None):
    """Raises DolincError on a non-finite stage or a device timeout."""
    _check(load().dolinc_sync_status(mesh.handle, _ptr(ws), _stream(stream)))


def dolinc_profile_enable(mesh, enable=True):
    _check(load().dolinc_profile_enable(mesh.handle, 1 if enable else 0))


def dolinc_profile_read(mesh):
    """(ms, launches) per kernel kind (KERNEL_KINDS order), waiting for recorded events."""
    ms = np.zeros(len(KERNEL_KINDS))
    n = np.zeros(len(KERNEL_KINDS), dtype=np.int64)
    _check(load().dolinc_profile_read(mesh.handle, _ptr(ms), _ptr(n)))
    return ms, n


profile_read = dolinc_profile_read


def diff_to_numpy(mesh, scheme, diff, order):
    """Unpack a dolinc_differentials buffer into a list over m = 1..order of
    arrays [nv, n_cells, C_m] (library cell order) of polynomial coefficients."""
    import torch
    off, stride, eb, _ = dolinc_diff_layout(mesh, scheme, order)
    raw = diff.detach()
    out = []
    for m in range(1, order + 1):
        Cm = m + 1 if mesh.dim == 2 else (m + 1) * (m + 2) // 2
        b = int(eb[m - 1])
        dt = {8: torch.float64, 4: torch.float32, 2: torch.bfloat16}[b]
        start = int(off[m - 1]) * b
        n = mesh.n_cells * int(stride[m - 1])
        blk = raw[start:start + n * b].view(dt).reshape(mesh.n_cells, int(stride[m - 1]))
        blk = blk[:, :scheme.nv * Cm].to(torch.float64).cpu().numpy()
        out.append(blk.reshape(mesh.n_cells, scheme.nv, Cm).transpose(1, 0, 2).copy())
    return out


# ---------------------------------------------------------------------------- troubled cells

MLP_PARAMS = 9985


def dolinc_criterion(mesh, scheme, u, flags, ws, kappa=4.0, eps=1e-3, stream=None):
    s = scheme.c()
    _check(load().dolinc_criterion(mesh.handle, C.byref(s), _ptr(u), _ptr(flags), float(kappa), float(eps),
                                   _ptr(ws), ws.numel(), _stream(stream)))


def dolinc_indicator_features(mesh, scheme, u, x24, ws, stream=None):
    s = scheme.c()
    _check(load().dolinc_indicator_features(mesh.handle, C.byref(s), _ptr(u), _ptr(x24), _ptr(ws), ws.numel(),
                                            _stream(stream)))


class MLP:
    """The indicator network (device-resident parameters, Adam state)."""

    def __init__(self, seed=0):
        h = C.c_void_p()
        _check(load().dolinc_mlp_create(C.byref(h), C.c_uint64(seed)))
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.dolinc_mlp_destroy(h)
            self.handle = None

    def get_params(self):
        out = np.zeros(MLP_PARAMS, dtype=np.float32)
        _check(load().dolinc_mlp_get_params(self.handle, _ptr(out)))
        return out

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        assert theta.shape == (MLP_PARAMS,)
        _check(load().dolinc_mlp_set_params(self.handle, _ptr(theta)))

    def forward(self, x, logits=None, flags=None, stream=None):
        _check(load().dolinc_mlp_forward(self.handle, _ptr(x), x.shape[0], _ptr(logits), _ptr(flags),
                                         _stream(stream)))

    def loss_grad(self, x, y, pos_weight, grad=None, loss=None, stream=None):
        _check(load().dolinc_mlp_loss_grad(self.handle, _ptr(x), _ptr(y), x.shape[0], float(pos_weight), _ptr(grad),
                                           _ptr(loss), _stream(stream)))

    def train_step(self, x, y, lr, pos_weight, loss=None, stream=None):
        _check(load().dolinc_mlp_train_step(self.handle, _ptr(x), _ptr(y), x.shape[0], float(lr), float(pos_weight),
                                            _ptr(loss), _stream(stream)))


def dolinc_indicator_infer(mesh, scheme, mlp, u, x24, flags, ws, logits=None, stream=None):
    s = scheme.c()
    _check(load().dolinc_indicator_infer(mesh.handle, C.byref(s), mlp.handle, _ptr(u), _ptr(x24), _ptr(flags),
                                         _ptr(logits), _ptr(ws), ws.numel(), _stream(stream)))


# ---------------------------------------------------------------------------- batches

class Batch:
    """Many meshes advanced together by one persistent launch per SSP-RK3 stage."""

    def __init__(self, meshes):
        L = load()
        arr = (C.c_void_p * len(meshes))(*[m.handle.value for m in meshes])
        h = C.c_void_p()
        _check(L.dolinc_batch_create(arr, len(meshes), C.byref(h)))
        self.handle = h
        n = C.c_int64()
        offs = np.zeros(len(meshes) + 1, dtype=np.int64)
        _check(L.dolinc_batch_info(h, C.byref(n), _ptr(offs)))
        self.n_cells = n.value
        self.cell_offsets = offs
        self.meshes = list(meshes)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.dolinc_batch_destroy(h)
            self.handle = None

    def workspace(self, scheme, stream=None):
        import torch
        n = C.c_size_t()
        s = scheme.c()
        _check(load().dolinc_batch_workspace_size(self.handle, C.byref(s), C.byref(n)))
        ws = torch.empty(n.value + 256, dtype=torch.uint8, device="cuda")
        off = (-ws.data_ptr()) % 256
        ws = ws[off:off + n.value]
        _check(load().dolinc_workspace_init(_ptr(ws), n.value, _stream(stream)))
        return ws

    def to_lib(self, fields):
        """list of per-mesh caller-order fields [nv, n_b] -> one batch field [nv, total]"""
        return np.concatenate([m.to_lib(f) for m, f in zip(self.meshes, fields)], axis=-1)

    def from_lib(self, u):
        o = self.cell_offsets
        return [m.from_lib(u[..., o[b]:o[b + 1]]) for b, m in enumerate(self.meshes)]

    def set_spin_limit(self, polls):
        _check(load().dolinc_batch_set_spin_limit(self.handle, int(polls)))

    def rk_step(self, scheme, dt, u, ws, use_graph=True, stream=None):
        s = scheme.c()
        _check(load().dolinc_batch_rk_step(self.handle, C.byref(s), _ptr(dt), _ptr(u), _ptr(ws), ws.numel(),
                                           1 if use_graph else 0, _stream(stream)))

    def autotune(self, scheme, dt, u, ws, stream=None):
        s = scheme.c()
        b, g, ms = C.c_int(), C.c_int(), C.c_double()
        _check(load().dolinc_batch_autotune(self.handle, C.byref(s), _ptr(dt), _ptr(u), _ptr(ws), ws.numel(),
                                            _stream(stream), C.byref(b), C.byref(g), C.byref(ms)))
        return dict(block=b.value, grid=g.value, ms_per_step=ms.value)


class _SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("solves", C.c_int), ("converged", C.c_int), ("breakdown", C.c_int),
                ("rel_residual", C.c_double), ("total_iterations", C.c_int64), ("total_solves", C.c_int64)]


class Implicit:
    """Semi-implicit DOLINC steps of linear advection on one mesh (dolinc_implicit_*):
    the weight part of every face value at the new level, c_r explicit."""

    def __init__(self, mesh, scheme, dt, theta=1.0):
        h = C.c_void_p()
        s = scheme.c()
        _check(load().dolinc_implicit_create(mesh.handle, C.byref(s), float(dt), float(theta), C.byref(h)))
        self.handle = h
        self.mesh, self.scheme, self.dt, self.theta = mesh, scheme, float(dt), float(theta)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.dolinc_implicit_destroy(h)
            self.handle = None

    def set_solver(self, rel_tol=1e-10, max_iter=1000, spin_limit=1 << 23, warm_start=False):
        _check(load().dolinc_implicit_set_solver(self.handle, float(rel_tol), int(max_iter), int(spin_limit),
                                                 int(warm_start)))

    def set_layout(self, ell):
        """Row layout: ELL width 4 / 6 / 8, or 0 (per face slot)."""
        _check(load().dolinc_implicit_set_layout(self.handle, int(ell)))

    @property
    def layout(self):
        return int(load().dolinc_implicit_layout(self.handle))

    def step(self, u, ws, n_outer=1, stream=None):
        _check(load().dolinc_implicit_step(self.handle, _ptr(u), int(n_outer), _ptr(ws), ws.numel(),
                                           _stream(stream)))

    def info(self):
        i = _SolveInfo()
        _check(load().dolinc_implicit_info(self.handle, C.byref(i)))
        return dict(iterations=i.iterations, solves=i.solves, converged=bool(i.converged),
                    breakdown=bool(i.breakdown), rel_residual=i.rel_residual,
                    total_iterations=i.total_iterations, total_solves=i.total_solves)

    def rows(self):
        """(row_offsets, nbr, off, diag) of V/dt + theta K in library order (host arrays)."""
        nc, ns = self.mesh.n_cells, self.mesh.n_slots
        ro = np.zeros(nc + 1, dtype=np.int32)
        nb = np.zeros(ns, dtype=np.int32)
        off = np.zeros(ns)
        dg = np.zeros(nc)
        _check(load().dolinc_implicit_rows(self.handle, _ptr(ro), _ptr(nb), _ptr(off), _ptr(dg)))
        return ro, nb, off, dg


def dolinc_implicit_create(mesh, scheme, dt, theta=1.0):
    return Implicit(mesh, scheme, dt, theta)


def dolinc_implicit_step(solver, u, ws, n_outer=1, stream=None):
    solver.step(u, ws, n_outer, stream)


def dolinc_implicit_info(solver):
    return solver.info()


class Halo:
    """A pending exchange of a partitioned step (dolinc_halo)."""

    def __init__(self, h):
        self.pending, self.order, self.record_bytes = h.pending, h.order, h.record_bytes
        self.send_dev, self.recv_dev = h.send_dev or 0, h.recv_dev or 0

    def views(self, ws, plan):
        """Per peer: (peer, send bytes, receive bytes) as uint8 views of the workspace ws."""
        rb = self.record_bytes
        s0, r0 = self.send_dev - ws.data_ptr(), self.recv_dev - ws.data_ptr()
        out = []
        for i, q in enumerate(plan["peers"]):
            a, b = int(plan["send_off"][i]) * rb, int(plan["send_off"][i + 1]) * rb
            c, d = int(plan["recv_off"][i]) * rb, int(plan["recv_off"][i + 1]) * rb
            out.append((int(q), ws[s0 + a:s0 + b], ws[r0 + c:r0 + d]))
        return out


def dolinc_part_step_begin(mesh, scheme, dt, u, ws, stream=None):
    h = _Halo()
    s = scheme.c()
    _check(load().dolinc_part_step_begin(mesh.handle, C.byref(s), float(dt), _ptr(u), _ptr(ws), ws.numel(),
                                         _stream(stream), C.byref(h)))
    return Halo(h)


def dolinc_part_step_continue(mesh, scheme, ws, stream=None):
    h = _Halo()
    s = scheme.c()
    _check(load().dolinc_part_step_continue(mesh.handle, C.byref(s), _ptr(ws), ws.numel(), _stream(stream),
                                            C.byref(h)))
    return Halo(h)


def part_rk_step(mesh, scheme, dt, u, ws, exchange, stream=None):
    """One SSP-RK3 step of a part mesh; exchange(halo) moves each pending halo's
    records between the parts (e.g. exchange_collective)."""
    h = dolinc_part_step_begin(mesh, scheme, dt, u, ws, stream)
    while h.pending:
        exchange(h)
        h = dolinc_part_step_continue(mesh, scheme, ws, stream)


def exchange_collective(dist, mesh, ws):
    """An exchange over torch.distributed point-to-point (NCCL: on the current stream):
    this rank is part dist.get_rank() of the partition."""
    def run(h):
        ops = []
        for q, snd, rcv in h.views(ws, mesh.plan):
            if snd.numel():
                ops.append(dist.P2POp(dist.isend, snd, q))
            if rcv.numel():
                ops.append(dist.P2POp(dist.irecv, rcv, q))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
    return run
