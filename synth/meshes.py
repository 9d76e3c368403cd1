"""Seeded unstructured meshes in owner/neighbour face form.

A mesh is a dict with the arrays the C ABI's mesh descriptor takes:

  dim                   2 or 3
  nodes                 float64 [n_nodes, dim]
  cell_face_offsets     int64   [n_cells + 1]   CSR cell -> faces
  cell_faces            int64   [..]
  face_node_offsets     int64   [n_faces + 1]   CSR face -> nodes
  face_nodes            int64   [..]            ordered so that the right-hand
                                                (3D) or clockwise-rotated edge
                                                (2D) normal points out of the owner
  face_owner            int64   [n_faces]
  face_neighbour        int64   [n_faces]       -1 on a boundary face
  face_periodic_shift   float64 [n_faces, dim]  translation that carries the
                                                neighbour cell next to the owner
  boundary_kind         int32   [n_faces]       0 interior/periodic, 1 zero-gradient

plus private keys ('_hf_cell', '_hf_nodes') with each cell's own outward
half-faces, used only to integrate initial data over the cells.

Periodic meshes keep image copies of the nodes on the far planes; faces across
the periodic planes pair cells whose nodes agree modulo the lattice.
"""
import numpy as np


def _assemble(dim, nodes, hf_cell, hf_nodes, node_key, period, boundary_kind=0):
    """Pair half-faces with equal (periodic) node sets into faces.

    hf_cell  [H]      owning cell of each half-face, non-decreasing
    hf_nodes [H, 4]   outward-ordered node ids, padded with -1
    node_key [n]      canonical id of each node (periodic images share one)
    period   [dim]    lattice period per axis (0: not periodic)
    """
    H = hf_cell.shape[0]
    keys = np.where(hf_nodes >= 0, node_key[np.maximum(hf_nodes, 0)], -1)
    keys = np.sort(keys, axis=1)
    order = np.lexsort(keys.T[::-1])
    ks = keys[order]
    same_next = np.all(ks[1:] == ks[:-1], axis=1)
    # group starts
    start = np.ones(H, dtype=bool)
    start[1:] = ~same_next
    gid = np.cumsum(start) - 1
    n_groups = gid[-1] + 1
    counts = np.bincount(gid, minlength=n_groups)
    if np.any(counts > 2):
        raise ValueError("non-manifold mesh: a face is shared by more than two cells")
    first = order[start]
    second = np.full(n_groups, -1, dtype=np.int64)
    pair = counts == 2
    # second member of each pair sits right after the first in sorted order
    pos_first = np.nonzero(start)[0]
    second[pair] = order[pos_first[pair] + 1]
    # owner is the half-face of the lower cell id
    a, b = first.copy(), second.copy()
    swap = pair & (hf_cell[np.maximum(b, 0)] < hf_cell[a])
    a[swap], b[swap] = second[swap], first[swap]
    owner = hf_cell[a]
    neigh = np.where(b >= 0, hf_cell[np.maximum(b, 0)], -1)
    fn = hf_nodes[a]
    # periodic shift: owner face centre minus neighbour face centre, snapped to the lattice
    nn = np.maximum(fn, 0)
    valid = (fn >= 0)[..., None]
    cnt = valid.sum(axis=1)
    ca = (nodes[nn] * valid).sum(axis=1) / cnt
    fb = hf_nodes[np.maximum(b, 0)]
    vb = (fb >= 0)[..., None]
    cb = (nodes[np.maximum(fb, 0)] * vb).sum(axis=1) / vb.sum(axis=1)
    shift = np.zeros((n_groups, dim))
    for k in range(dim):
        if period[k] > 0:
            shift[:, k] = np.round((ca[:, k] - cb[:, k]) / period[k]) * period[k]
    shift[~pair] = 0.0
    # face order: interior faces by (owner, neighbour), then boundary faces by owner
    bnd = ~pair
    forder = np.lexsort((neigh, owner, bnd.astype(np.int64)))
    owner, neigh, fn, shift, bnd = owner[forder], neigh[forder], fn[forder], shift[forder], bnd[forder]
    a, b = a[forder], b[forder]
    # face ids per half-face
    face_of_hf = np.empty(H, dtype=np.int64)
    face_of_hf[a] = np.arange(n_groups)
    hb = b >= 0
    face_of_hf[b[hb]] = np.arange(n_groups)[hb]
    n_cells = int(hf_cell[-1]) + 1
    cell_face_offsets = np.zeros(n_cells + 1, dtype=np.int64)
    np.add.at(cell_face_offsets, hf_cell + 1, 1)
    cell_face_offsets = np.cumsum(cell_face_offsets)
    nper = (fn >= 0).sum(axis=1)
    face_node_offsets = np.zeros(n_groups + 1, dtype=np.int64)
    face_node_offsets[1:] = np.cumsum(nper)
    face_nodes = fn[fn >= 0].astype(np.int64)
    bk = np.where(bnd, boundary_kind, 0).astype(np.int32)
    return dict(
        dim=dim, nodes=np.ascontiguousarray(nodes, dtype=np.float64),
        cell_face_offsets=cell_face_offsets, cell_faces=face_of_hf,
        face_node_offsets=face_node_offsets, face_nodes=face_nodes,
        face_owner=owner.astype(np.int64), face_neighbour=neigh.astype(np.int64),
        face_periodic_shift=np.ascontiguousarray(shift),
        boundary_kind=bk,
        _hf_cell=hf_cell, _hf_nodes=hf_nodes,
    )


def _jitter(nodes, idx, n, amp, h, rng, dim):
    """Move nodes whose lattice indices are all strictly inside (1..n-1) by U(-amp*h, amp*h)."""
    if amp <= 0:
        return nodes
    inner = np.all((idx >= 1) & (idx <= np.asarray(n) - 1), axis=1)
    d = rng.uniform(-amp, amp, size=(nodes.shape[0], dim)) * np.asarray(h)
    nodes = nodes.copy()
    nodes[inner] += d[inner]
    return nodes


def tri_mesh(nx, ny, jitter=0.0, seed=0, boundary="periodic", L=(1.0, 1.0)):
    """Quads of an nx x ny lattice on [0,Lx]x[0,Ly], each split along its
    (i,j)-(i+1,j+1) diagonal into two counter-clockwise triangles.

    boundary: 'periodic' or 'transmissive' (zero-gradient boundary faces).
    Nodes strictly inside the square are jittered by U(-jitter*h, jitter*h).
    """
    rng = np.random.default_rng(seed)
    hx, hy = L[0] / nx, L[1] / ny
    I, J = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    idx = np.stack([I.ravel(), J.ravel()], axis=1)
    nodes = idx * np.array([hx, hy], dtype=np.float64)
    nodes = _jitter(nodes, idx, (nx, ny), jitter, (hx, hy), rng, 2)
    nid = lambda i, j: i * (ny + 1) + j
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00, v10, v11, v01 = nid(i, j), nid(i + 1, j), nid(i + 1, j + 1), nid(i, j + 1)
    nq = nx * ny
    # two triangles per quad: T1 = (v00, v10, v11), T2 = (v00, v11, v01)
    tris = np.empty((2 * nq, 3), dtype=np.int64)
    tris[0::2] = np.stack([v00, v10, v11], axis=1)
    tris[1::2] = np.stack([v00, v11, v01], axis=1)
    nc = 2 * nq
    hf_cell = np.repeat(np.arange(nc), 3)
    hf = np.full((3 * nc, 4), -1, dtype=np.int64)
    hf[:, 0] = tris.ravel()
    hf[:, 1] = np.roll(tris, -1, axis=1).ravel()
    if boundary == "periodic":
        key = (idx[:, 0] % nx) * ny + (idx[:, 1] % ny)
        period = (L[0], L[1])
        bk = 0
    else:
        key = np.arange(nodes.shape[0])
        period = (0.0, 0.0)
        bk = 1
    return _assemble(2, nodes, hf_cell, hf, key, period, bk)


def strip_mesh(widths, height=None, boundary="periodic"):
    """One row of quads with the given widths along x (a 1D mesh in 2D form).

    The strip is periodic in y with one cell across, so every cell is its own
    y-neighbour; along x it is 'periodic' or 'transmissive'.
    """
    widths = np.asarray(widths, dtype=np.float64)
    n = widths.shape[0]
    xs = np.concatenate([[0.0], np.cumsum(widths)])
    Hh = float(height) if height is not None else float(widths.mean())
    nodes = np.zeros((2 * (n + 1), 2))
    nodes[0::2, 0] = xs
    nodes[1::2, 0] = xs
    nodes[1::2, 1] = Hh
    nid = lambda i, j: 2 * i + j
    i = np.arange(n)
    quads = np.stack([nid(i, 0), nid(i + 1, 0), nid(i + 1, 1), nid(i, 1)], axis=1)
    hf_cell = np.repeat(np.arange(n), 4)
    hf = np.full((4 * n, 4), -1, dtype=np.int64)
    hf[:, 0] = quads.ravel()
    hf[:, 1] = np.roll(quads, -1, axis=1).ravel()
    xi = np.repeat(np.arange(n + 1), 2)
    if boundary == "periodic":
        key = (xi % n)
        period = (xs[-1], Hh)
        bk = 0
    else:
        key = xi
        period = (0.0, Hh)
        bk = 1
    return _assemble(2, nodes, hf_cell, hf, key.astype(np.int64), period, bk)


def _lattice3(n, L, jitter, rng):
    h = np.asarray(L, dtype=np.float64) / np.asarray(n)
    I, J, K = np.meshgrid(np.arange(n[0] + 1), np.arange(n[1] + 1), np.arange(n[2] + 1), indexing="ij")
    idx = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    ref = idx * h
    nodes = _jitter(ref, idx, n, jitter, h, rng, 3)
    key = ((idx[:, 0] % n[0]) * n[1] + (idx[:, 1] % n[1])) * n[2] + (idx[:, 2] % n[2])
    return nodes, ref, key


def _corner_ids(n, i, j, k):
    nid = lambda a, b, c: (a * (n[1] + 1) + b) * (n[2] + 1) + c
    return {(a, b, c): nid(i + a, j + b, k + c) for a in (0, 1) for b in (0, 1) for c in (0, 1)}


# outward faces of a positively oriented tetrahedron (0,1,2,3)
_TET_FACES = ((0, 2, 1), (0, 1, 3), (0, 3, 2), (1, 2, 3))


def tet_mesh(n, jitter=0.0, seed=0, L=(1.0, 1.0, 1.0)):
    """Periodic box of n^3 hexes, each split into 5 tetrahedra with the split
    parity alternating with (i+j+k) so the face diagonals agree (n even)."""
    if isinstance(n, int):
        n = (n, n, n)
    if any(m % 2 for m in n):
        raise ValueError("tet_mesh needs even lattice sizes for a conformal periodic split")
    rng = np.random.default_rng(seed)
    nodes, ref, key = _lattice3(n, L, jitter, rng)
    i, j, k = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    v = _corner_ids(n, i, j, k)
    even = ((i + j + k) % 2) == 0
    even_tets = [((1, 0, 0), (0, 0, 0), (1, 1, 0), (1, 0, 1)),
                 ((0, 1, 0), (0, 0, 0), (1, 1, 0), (0, 1, 1)),
                 ((0, 0, 1), (0, 0, 0), (1, 0, 1), (0, 1, 1)),
                 ((1, 1, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1)),
                 ((0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1))]
    odd_tets = [((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)),
                ((1, 1, 0), (1, 0, 0), (0, 1, 0), (1, 1, 1)),
                ((1, 0, 1), (1, 0, 0), (0, 0, 1), (1, 1, 1)),
                ((0, 1, 1), (0, 1, 0), (0, 0, 1), (1, 1, 1)),
                ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1))]
    nh = i.shape[0]
    tets = np.empty((nh, 5, 4), dtype=np.int64)
    for t in range(5):
        for q in range(4):
            tets[:, t, q] = np.where(even, v[even_tets[t][q]], v[odd_tets[t][q]])
    tets = tets.reshape(-1, 4)
    # orient positively on the un-jittered lattice
    p = ref[tets]
    vol = np.einsum("ij,ij->i", p[:, 1] - p[:, 0], np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]))
    neg = vol < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    nc = tets.shape[0]
    hf_cell = np.repeat(np.arange(nc), 4)
    hf = np.full((4 * nc, 4), -1, dtype=np.int64)
    for q, (a, b, c) in enumerate(_TET_FACES):
        hf[q::4, 0] = tets[:, a]
        hf[q::4, 1] = tets[:, b]
        hf[q::4, 2] = tets[:, c]
    return _assemble(3, nodes, hf_cell, hf, key, tuple(float(x) for x in L))


_HEX_FACES = (((0, 0, 0), (0, 0, 1), (0, 1, 1), (0, 1, 0)),   # x-
              ((1, 0, 0), (1, 1, 0), (1, 1, 1), (1, 0, 1)),   # x+
              ((0, 0, 0), (1, 0, 0), (1, 0, 1), (0, 0, 1)),   # y-
              ((0, 1, 0), (0, 1, 1), (1, 1, 1), (1, 1, 0)),   # y+
              ((0, 0, 0), (0, 1, 0), (1, 1, 0), (1, 0, 0)),   # z-
              ((0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)))   # z+
_PRISM_A = (((0, 0, 0), (1, 1, 0), (1, 0, 0)),
            ((0, 0, 1), (1, 0, 1), (1, 1, 1)),
            ((0, 0, 0), (1, 0, 0), (1, 0, 1), (0, 0, 1)),
            ((1, 0, 0), (1, 1, 0), (1, 1, 1), (1, 0, 1)),
            ((1, 1, 0), (0, 0, 0), (0, 0, 1), (1, 1, 1)))
_PRISM_B = (((0, 0, 0), (0, 1, 0), (1, 1, 0)),
            ((0, 0, 1), (1, 1, 1), (0, 1, 1)),
            ((0, 0, 0), (0, 0, 1), (0, 1, 1), (0, 1, 0)),
            ((0, 1, 0), (0, 1, 1), (1, 1, 1), (1, 1, 0)),
            ((0, 0, 0), (1, 1, 0), (1, 1, 1), (0, 0, 1)))


def hexprism_mesh(n, jitter=0.0, seed=0, L=(1.0, 1.0, 1.0), split_fraction=0.5):
    """Periodic box of n^3 hexes; hexes whose lattice column lies in x < split_fraction*Lx
    are split into two prisms by the vertical plane through their (0,0)-(1,1) diagonal."""
    if isinstance(n, int):
        n = (n, n, n)
    rng = np.random.default_rng(seed)
    nodes, ref, key = _lattice3(n, L, jitter, rng)
    i, j, k = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    v = _corner_ids(n, i, j, k)
    split = (i + 0.5) < split_fraction * n[0]
    # per hex: either 1 hex (6 faces) or 2 prisms (5 faces each)
    nh = i.shape[0]
    ncell_per = np.where(split, 2, 1)
    cell_start = np.concatenate([[0], np.cumsum(ncell_per)[:-1]])
    hf_rows, hf_cells = [], []

    def emit(mask, cell_ids, template):
        for face in template:
            row = np.full((mask.sum(), 4), -1, dtype=np.int64)
            for q, c in enumerate(face):
                row[:, q] = v[c][mask]
            hf_rows.append(row)
            hf_cells.append(cell_ids)
    hexm = ~split
    emit(hexm, cell_start[hexm], _HEX_FACES)
    emit(split, cell_start[split], _PRISM_A)
    emit(split, cell_start[split] + 1, _PRISM_B)
    hf = np.concatenate(hf_rows)
    hc = np.concatenate(hf_cells)
    o = np.argsort(hc, kind="stable")
    return _assemble(3, nodes, hc[o], hf[o], key, tuple(float(x) for x in L))


def hex_mesh(xs, ys, zs, periodic=(True, True, True)):
    """Cartesian hexes on the tensor grid of node coordinates xs, ys, zs
    (stretched spacing allowed).  Non-periodic axes get zero-gradient boundaries."""
    xs, ys, zs = (np.asarray(a, dtype=np.float64) for a in (xs, ys, zs))
    n = (len(xs) - 1, len(ys) - 1, len(zs) - 1)
    I, J, K = np.meshgrid(np.arange(n[0] + 1), np.arange(n[1] + 1), np.arange(n[2] + 1), indexing="ij")
    idx = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    nodes = np.stack([xs[idx[:, 0]], ys[idx[:, 1]], zs[idx[:, 2]]], axis=1)
    keyc = [idx[:, a] % n[a] if periodic[a] else idx[:, a] for a in range(3)]
    m = [n[a] + (0 if periodic[a] else 1) for a in range(3)]
    key = (keyc[0] * m[1] + keyc[1]) * m[2] + keyc[2]
    i, j, k = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    v = _corner_ids(n, i.ravel(), j.ravel(), k.ravel())
    nc = n[0] * n[1] * n[2]
    hf = np.full((6 * nc, 4), -1, dtype=np.int64)
    for q, face in enumerate(_HEX_FACES):
        for p, c in enumerate(face):
            hf[q::6, p] = v[c]
    hf_cell = np.repeat(np.arange(nc), 6)
    period = tuple((a[-1] - a[0]) if periodic[t] else 0.0 for t, a in enumerate((xs, ys, zs)))
    return _assemble(3, nodes, hf_cell, hf, key, period, 1)


def mesh_summary(m):
    nf = m["face_owner"].shape[0]
    return dict(dim=m["dim"], n_nodes=m["nodes"].shape[0],
                n_cells=m["cell_face_offsets"].shape[0] - 1, n_faces=nf,
                n_boundary=int((m["face_neighbour"] < 0).sum()))
