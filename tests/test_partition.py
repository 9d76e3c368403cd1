"""Halo-exchanged partitions of one mesh, host side (CPU, no GPU).

The partition is a space-filling curve cut: cells in Morton order split into equal
contiguous ranges.  A part's plan (own cells, depth-1 ghosts, per-peer send and
receive lists) is checked against brute force over the face lists.  The exchange is
then run for real between gloo ranks: every rank computes its part's differentials
pass by pass with the FP64 oracle (on the whole mesh's geometry, restricted to the
part), exchanges the ghosts' records of each order with its peers, and evaluates
the residual; the own cells' residuals must equal the whole mesh's bit for bit
(Sec 2.6: coupled boundaries need only the adjacent cells' data and differentials).
"""
import os
import socket

import numpy as np
import pytest

import oracle
import synth

dg = pytest.importorskip("paper_2404_08952_gb300")

CASES = {
    "tet_euler": lambda: synth.workload("euler3d_tet64", size=6, q=1),
    "tri_riemann": lambda: synth.workload("euler2d_riemann", size=14, q=1),
    "hexprism_order5": lambda: synth.workload("adv3d_hexprism", order=5, size=6, q=1),
}
_cache = {}


def case(name):
    if name not in _cache:
        _cache[name] = CASES[name]()
    return _cache[name]


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(dg.LIB_PATH):
        from paper_2404_08952_gb300 import build
        build.build()
    return dg.load()


def _morton_order(m):
    """Caller ids in the library's Morton order (the single part's local order)."""
    n = m["cell_face_offsets"].shape[0] - 1
    return dg.dolinc_part_plan(m, np.zeros(n, dtype=np.int32), 1, 0)["local_cells"]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("n_parts", [2, 3, 7])
def test_partition_is_contiguous_and_balanced(lib, name, n_parts):
    m = case(name)["mesh"]
    pc = dg.dolinc_partition(m, n_parts)
    order = _morton_order(m)
    n = len(order)
    assert sorted(order.tolist()) == list(range(n))
    want = (np.arange(n) * n_parts) // n                 # equal contiguous ranges of the curve
    assert np.array_equal(pc[order], want)
    counts = np.bincount(pc, minlength=n_parts)
    assert counts.max() - counts.min() <= 1


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("n_parts", [2, 3, 5])
def test_plan_matches_brute_force(lib, name, n_parts):
    m = case(name)["mesh"]
    own_f, nb_f = np.asarray(m["face_owner"]), np.asarray(m["face_neighbour"])
    pc = dg.dolinc_partition(m, n_parts)
    order = _morton_order(m)
    rank_of = np.empty(len(order), dtype=np.int64)
    rank_of[order] = np.arange(len(order))
    plans = [dg.dolinc_part_plan(m, pc, n_parts, p) for p in range(n_parts)]
    inner = nb_f >= 0
    a, b = own_f[inner], nb_f[inner]
    for p, pl in enumerate(plans):
        lc, owned = pl["local_cells"], pl["owned"].astype(bool)
        own = set(np.flatnonzero(pc == p).tolist())
        assert set(lc[owned].tolist()) == own
        ghosts = set(b[(pc[a] == p) & (pc[b] != p)].tolist()) | set(a[(pc[b] == p) & (pc[a] != p)].tolist())
        assert set(lc[~owned].tolist()) == ghosts
        assert np.all(np.diff(rank_of[lc]) > 0)            # the whole mesh's library order
        assert pl["n_faces"] == int(((pc[own_f] == p) | (inner & (pc[np.maximum(nb_f, 0)] == p))).sum())
        assert pl["peers"].tolist() == sorted(set(pc[list(ghosts)].tolist()))
        for i, q in enumerate(pl["peers"]):
            recv = lc[pl["recv_cells"][pl["recv_off"][i]:pl["recv_off"][i + 1]]]
            want = sorted((c for c in ghosts if pc[c] == q), key=lambda c: rank_of[c])
            assert recv.tolist() == want
            send = lc[pl["send_cells"][pl["send_off"][i]:pl["send_off"][i + 1]]]
            adj = set(a[(pc[a] == p) & (pc[b] == q)].tolist()) | set(b[(pc[b] == p) & (pc[a] == q)].tolist())
            assert send.tolist() == sorted(adj, key=lambda c: rank_of[c])
            # what p sends to q is what q expects from p, in the same order
            pq = plans[q]
            j = pq["peers"].tolist().index(p)
            assert send.tolist() == pq["local_cells"][pq["recv_cells"][pq["recv_off"][j]:pq["recv_off"][j + 1]]].tolist()


def test_plan_rejects_bad_input(lib):
    m = case("tet_euler")["mesh"]
    pc = dg.dolinc_partition(m, 2)
    with pytest.raises(dg.DolincError):
        dg.dolinc_part_plan(m, pc, 2, 2)                     # no such part
    with pytest.raises(dg.DolincError):
        dg.dolinc_part_plan(m, pc + 5, 2, 0)                 # entries out of range
    with pytest.raises(dg.DolincError):
        dg.dolinc_part_plan(m, np.zeros_like(pc), 2, 1)      # a part with no cell
    with pytest.raises(dg.DolincError):
        dg.dolinc_partition(m, 0)


# ------------------------------------------------------------------ exchange between gloo ranks

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def part_oracle(O, m, pc, part, plan):
    """The oracle restricted to a part: own cells' faces in the whole mesh's face order,
    with the whole mesh's geometry."""
    lc = plan["local_cells"]
    loc = np.full(O.n_cells, -1, dtype=np.int64)
    loc[lc] = np.arange(len(lc))
    own_f, nb_f = O.owner, O.neigh
    faces = np.flatnonzero((pc[own_f] == part) | ((nb_f >= 0) & (pc[np.maximum(nb_f, 0)] == part)))
    shift = m.get("face_periodic_shift")
    return oracle.Oracle.from_geometry(
        O.dim, loc[own_f[faces]], np.where(nb_f[faces] >= 0, loc[np.maximum(nb_f[faces], 0)], -1),
        None if shift is None else np.asarray(shift)[faces], O.V[lc], O.xc[lc], O.S[faces], O.xf[faces],
        O.w[faces], O.d[faces])


def _exchange(dist, torch, plan, T):
    """Ghost records of T [nv, n_local, A] from their owners (isend / irecv per peer)."""
    ops, bufs = [], []
    for i, q in enumerate(plan["peers"]):
        s = plan["send_cells"][plan["send_off"][i]:plan["send_off"][i + 1]]
        r = plan["recv_cells"][plan["recv_off"][i]:plan["recv_off"][i + 1]]
        snd = torch.from_numpy(np.ascontiguousarray(T[:, s, :]))
        rcv = torch.empty((T.shape[0], len(r), T.shape[2]), dtype=torch.float64)
        ops.append(dist.isend(snd, int(q)))
        ops.append(dist.irecv(rcv, int(q)))
        bufs.append((r, rcv, snd))
    for op in ops:
        op.wait()
    for r, rcv, _ in bufs:
        T[:, r, :] = rcv.numpy()


def _worker(rank, world, port, name, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = CASES[name]()
        m, u = w["mesh"], w["u0"]
        sch = oracle.Scheme(**w["scheme"])
        O = oracle.Oracle(m)
        pc = dg.dolinc_partition(m, world)
        plan = dg.dolinc_part_plan(m, pc, world, rank)
        Ol = part_oracle(O, m, pc, rank, plan)
        owned = plan["owned"].astype(bool)
        T0 = u[:, plan["local_cells"]][:, :, None].copy()
        T0[:, ~owned, :] = np.nan                          # ghosts: only what the exchange brings
        _exchange(dist, torch, plan, T0)
        T = [T0]
        for mm in range(1, sch.n_diff + 1):
            Tm = Ol.gauss_pass(T[-1], mm, sch)
            _exchange(dist, torch, plan, Tm)
            T.append(Tm)
        R = Ol.residual_T(T, sch)
        Rw = O.residual(u, sch)
        got, want = R[:, owned], Rw[:, plan["local_cells"][owned]]
        q.put((rank, bool(np.array_equal(got, want)), float(np.abs(got - want).max()), int(owned.sum())))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("tet_euler", 2), ("tri_riemann", 2), ("hexprism_order5", 3)])
def test_partitioned_residual_equals_whole_mesh(lib, name, world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, qu)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(qu.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sum(o[3] for o in out) == case(name)["u0"].shape[1]     # every cell owned once
    for rank, same, diff, _ in out:
        assert same, (rank, diff)


def _collective_worker(rank, world, port, name, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = CASES[name]()["mesh"]
        pc = dg.dolinc_partition(m, world)
        plan = dg.dolinc_part_plan(m, pc, world, rank)
        lc = plan["local_cells"]
        rb = 16                                        # a 16-byte record: the caller id, twice
        ns, nr = len(plan["send_cells"]), len(plan["recv_cells"])
        ws = torch.zeros(256 + rb * (ns + nr), dtype=torch.uint8)
        send = ws[256:256 + rb * ns].view(torch.int64).view(ns, 2)
        send[:, 0] = torch.from_numpy(lc[plan["send_cells"]])
        send[:, 1] = -send[:, 0]
        h = dg.Halo.__new__(dg.Halo)
        h.pending, h.order, h.record_bytes = 1, 0, rb
        h.send_dev, h.recv_dev = ws.data_ptr() + 256, ws.data_ptr() + 256 + rb * ns
        holder = type("PartMesh", (), {"plan": plan})()
        dg.exchange_collective(dist, holder, ws)(h)
        got = ws[256 + rb * ns:].view(torch.int64).view(nr, 2).numpy()
        want = lc[plan["recv_cells"]]
        q.put((rank, bool(np.array_equal(got[:, 0], want) and np.array_equal(got[:, 1], -want))))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("tet_euler", 2), ("hexprism_order5", 3)])
def test_exchange_collective_delivers_each_ghost_record(lib, name, world):
    """The package's exchange (torch.distributed point-to-point, here over gloo on CPU
    tensors) moves each peer's send region into this rank's receive region: every
    ghost receives its owner's record, in the plan's order."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_collective_worker, args=(r, world, port, name, qu)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(qu.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok in out), out
