"""Benchmark of the DOLINC SSP-RK3 stage on one GB300 (or N replicas under torchrun).

Workload (default): euler3d_tet64 — 64^3 hexes x 5 tetrahedra (1,310,720 cells),
+-15% node jitter, periodic, isentropic vortex, Rusanov flux, scheme order 3
(stencil (3,1) = USR3, differentials through order 2), FP32 differentials/reconstruction/
flux with FP64 geometry master and FP64 state update.  A step is one SSP-RK3 time
step (3 stages, each: differential passes + fused reconstruct/flux/residual/update);
the timed K steps are one dolinc_rk_steps call (the state stays on the device).

Metric: cell-updates per second per RK stage = cells * 3 * steps / time.
The line also carries the FP64 GPU run of the same steps, the mixed-vs-FP64
difference and the full-size error of one GPU stage against the FP64 oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dolinc|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK stage; % HBM roofline; mixed vs FP64 GPU at stated L2 error"
UNIT = "cell-updates/s"
L2_BYTES = 129 * 2 ** 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.enabled = index >= 0
        self.proc = None
        self.lines = []

    def __enter__(self):
        if not self.enabled:
            return self
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def reduce_max(x, dist=None):
    """Max over ranks of a host float (the job's time is its slowest replica)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x, dist=None):
    """Sum over ranks (the job's work is every replica's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return type(x)(t.item())


def _ncoef(dim, m):
    return m + 1 if dim == 2 else (m + 1) * (m + 2) // 2


def _widths(sch):
    sg = 8 if sch.precision == "fp64" else 4

    def sb(m):
        return 8 if sch.precision == "fp64" else (2 if sch.precision == "fp32_bf16" and m >= 2 else 4)
    return sg, sb


def stage_orders(sch):
    """Differential orders the stage reads: the stencil's own need (max(r, k-r-2),
    at least 1), 2 under the ENO3 / WENO5 limiters, never more than are computed."""
    k, r = getattr(sch, "k", 3), getattr(sch, "r", 1)
    need = max(r, k - r - 2, 1)
    if getattr(sch, "limiter", "none") in ("eno3_all", "eno3_flagged", "weno5_all", "weno5_flagged"):
        need = max(need, 2)
    return min(need, sch.n_diff)


def alg_bytes(kind, M, sch, basis="stored"):
    """Algorithmic bytes of one launch, per cell as the scope table's measurement
    section defines them (B_alg), times the cells:
      diff m:  nv (s_{m-1} c_{m-1} + s_m c_m) + Gp
      stage:   nv sum_{m<=N} s_m c_m + Gr + nv (16 + 8 + s_0)
      Gp = nfc 8 + (nfc/2)(D s_g + s_g) + (s_g + 4),  Gr = Gp + (nfc/2) D s_g
    (c_m components of order m, s_m its stored width, nfc slots per cell, D the
    dimension; per slot the neighbour and face indices, per face S_f and omega, per
    cell 1/V and a CSR offset, per face of the stage d_f; the state as FP64 reads of
    u^n and u^(k), an FP64 write and a bulk-precision copy).
    basis "stored" (the roofline's): the widths the build stores (geometry s_g = 4 B
    below FP64) and, in the stage, the orders N the stencil reads (stage_orders).
    basis "table": the scope table's own evaluation, geometry at FP64 widths and the
    stage reading every computed order N = N_d.  pack (not in B_alg): nv (8 + s_0)."""
    if kind == "diff_pair":         # one stage's order-2 pass with the next stage's order-1 pass
        return alg_bytes("diff2", M, sch, basis) + alg_bytes("diff1", M, sch, basis)
    nc, nv, dim = M.n_cells, sch.nv, M.dim
    sg, sb = _widths(sch)
    if basis == "table":
        sg = 8
    nfc = M.n_slots / nc
    gp = nfc * 8 + (nfc / 2) * (dim * sg + sg) + (sg + 4)
    gr = gp + (nfc / 2) * dim * sg
    if kind == "pack":
        return nc * nv * (8 + sb(0))
    if kind.startswith("diff"):
        m = int(kind[4:])
        return nc * (nv * (_ncoef(dim, m - 1) * sb(m - 1) + _ncoef(dim, m) * sb(m)) + gp)
    top = sch.n_diff if basis == "table" else stage_orders(sch)
    return nc * (nv * sum(_ncoef(dim, m) * sb(m) for m in range(top + 1)) + gr + nv * (16 + 8 + sb(0)))


def kernel_bytes(kind, M, sch):
    """Fewest bytes this library's kernel must move per launch: every array it reads
    or writes once (neighbour re-reads served on chip), at the stored widths (FP32
    geometry tables below FP64), without record padding; the stage reads only the
    orders its stencil needs and, below FP64, the increment form's state traffic
    (averaged over the three stages)."""
    nc, nf, ns, dim, nv = M.n_cells, M.n_faces, M.n_slots, M.dim, sch.nv
    sg, sb = _widths(sch)
    if kind == "pack":
        return nc * nv * (8 + sb(0))
    if kind == "diff_pair":         # the two passes' data, their geometry read once
        geo = nc * (4 * sg + 4) + ns * 4 * sg
        return kernel_bytes("diff2", M, sch) + kernel_bytes("diff1", M, sch) - geo
    if kind.startswith("diff"):
        m = int(kind[4:])
        data = nc * nv * (_ncoef(dim, m - 1) * sb(m - 1) + _ncoef(dim, m) * sb(m))
        geo = nc * (4 * sg + 4) + ns * 4 * sg
        return data + geo
    NS = max(sch.r, sch.k - sch.r - 2, 1)
    data = nc * nv * sum(_ncoef(dim, m) * sb(m) for m in range(NS + 1))
    if sch.precision == "fp64":
        state = nc * nv * 8 * (5.0 / 3.0 + 1.0) + nc * nv * sb(0) * (2.0 / 3.0)   # u0/us reads, out, next record
    else:
        state = nc * nv * (8 + 16 + 20) / 3.0    # increment form: D, start record, next record, u0/u in the last
    geo = nc * (4 + 4 * sg) + ns * 8 + nf * 8 * sg
    return data + state + geo


KINDS = ["pack", "diff1", "diff2", "diff3", "diff4", "stage", "faces", "diff_pair", "solve"]


def _stage_roofline(M, sch, ms_stage, peak):
    """B_alg of one whole RK stage (all differential passes + the fused stage) per
    cell, and the achieved GB/s and fraction of the measured peak at ms_stage (stored
    basis; the scope table's FP64-width all-orders figure beside it)."""
    b = sum(alg_bytes("diff%d" % m, M, sch) for m in range(1, sch.n_diff + 1)) + alg_bytes("stage", M, sch)
    bt = sum(alg_bytes("diff%d" % m, M, sch, "table") for m in range(1, sch.n_diff + 1)) + \
        alg_bytes("stage", M, sch, "table")
    gbs = b / (ms_stage / 1e3) / 1e9
    return {"alg_bytes_per_cell": round(b / M.n_cells, 1), "ms_per_stage": round(ms_stage, 5),
            "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
            "table_basis_bytes_per_cell": round(bt / M.n_cells, 1),
            "table_basis_frac": round(bt / (ms_stage / 1e3) / 1e9 / peak, 4)}


def _config(args, w, cells, faces):
    """The workload's config, identical in both arms of the benchmark."""
    return {"workload": args.workload, "cells": cells, "faces": faces,
            "scheme_order": w["info"].get("order"), "stencil_k_r": [w["scheme"]["k"], w["scheme"]["r"]],
            "n_diff": w["scheme"]["n_diff"], "precision": args.precision,
            "flux": w["scheme"]["flux"], "stages_per_step": 3,
            "l2_policy": "inputs larger than L2 (differential records, state and geometry of every cell "
                         "well above the 129 MB L2)",
            "parallelism": "replicas" if int(os.environ.get("WORLD_SIZE", "1")) > 1 else "single GPU"}


def _host_info():
    """Host cores and CPU model (lscpu) of the machine the oracle runs on."""
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            k, _, v = ln.partition(":")
            if k.strip() in ("Model name", "Architecture", "Socket(s)", "Core(s) per socket", "Thread(s) per core"):
                info[k.strip()] = v.strip()
    except Exception:
        pass
    return info


def _oracle_stage_seconds(O, u0, osch, dt, reps=1):
    """Seconds of one SSP-RK3 stage (stage 0) of the oracle, best of reps; and the result."""
    best, ref = None, None
    for _ in range(reps):
        t0 = time.perf_counter()
        ref = O.rk3_stage(u0, u0, osch, dt, 0)
        t = time.perf_counter() - t0
        best = t if best is None else min(best, t)
    return best, ref


def _increment_bound_ratio(O, inc, inc_ref, u0, dt, scheme):
    """Worst cell's |increment - oracle increment| over the per-cell FP32 bound
    dt * 2 * (1/V_c) sum_f |S_f| lam 1e-5 max|u| (stencil order 1; lam the largest wave
    speed of the data; Euler faces carry two states): <= 1 meets the stated 1e-5."""
    if scheme["flux"] == "upwind":
        lam = float(np.linalg.norm(scheme.get("adv", (1.0, 1.0, 0.0))))
    elif scheme["flux"] == "burgers":
        lam = float(np.abs(u0).max() * np.sqrt(O.dim))
    else:
        rho, E = u0[0], u0[-1]
        vel = u0[1:-1] / rho
        p = (scheme.get("gamma", 1.4) - 1.0) * (E - 0.5 * rho * (vel * vel).sum(0))
        lam = float((np.sqrt((vel * vel).sum(0)) + np.sqrt(scheme.get("gamma", 1.4) * p / rho)).max())
    a = np.linalg.norm(O.S, axis=1) * lam * 1e-5 * np.abs(u0).max()
    t = np.zeros(O.n_cells)
    np.add.at(t, O.owner, a)
    nb = O.neigh >= 0
    np.add.at(t, O.neigh[nb], a[nb])
    bound = dt * 2.0 * t / O.V
    return float((np.abs(inc - inc_ref) / bound[None, :]).max())


# GB300's FP64 peak from its unit counts and clock: 152 SMs x 2 FP64 FMA per clock per SM
# x 2 FLOP x 2.07 GHz (the 1.25 TFLOP/s nominal figure)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07


def _fp64_roofline(args, w, M, f):
    """The FP64 path's stage pair against the FP64 ALU peak: FP64 FLOP per face of the
    pair (2 per DFMA, 1 per DADD / DMUL) from the instruction counters of one ncu
    capture (profiles/fp64_flops.json, per face, the same scheme) times the faces, over
    the pair's live per-launch time."""
    pfile = os.path.join(ROOT, "profiles", "fp64_flops.json")
    key = "%s/order%d" % (args.workload, w["info"].get("order", 0))
    try:
        per_face = float(json.load(open(pfile))[key])
    except Exception:
        return None
    kms, kn = f["kms"], f["kn"]
    i = KINDS.index("stage")
    if kn[i] == 0:
        return None
    ms = kms[i] / kn[i]
    gf = per_face * M.n_faces / (ms / 1e3) / 1e9
    return {"bound": "alu", "kernel": "stage (k_flux + k_gather, FP64)", "achieved": round(gf, 1),
            "peak": round(FP64_PEAK_GFLOPS, 1), "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz",
            "unit": "GFLOP/s", "frac": round(gf / FP64_PEAK_GFLOPS, 4), "flop_per_face": per_face,
            "ms_per_launch": round(ms, 5)}


def _l2_rel(a, b):
    """max over variables of ||a_v - b_v||_2 / ||b||_2 (all variables' norm, so a
    variable that is zero in the data, e.g. z-momentum, is measured against the state)."""
    ref = np.sqrt((b ** 2).sum() / b.shape[0])
    return float(np.sqrt(((a - b) ** 2).sum(axis=1)).max() / ref)


def run_dolinc(args):
    import torch
    import paper_2404_08952_gb300 as dg
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    summaries = rank == 0 and not args.no_variants and args.workload == "euler3d_tet64" and world == 1
    # host inputs of the semi-implicit summary: forked workers, before CUDA starts
    imp_inputs = _implicit_inputs(args, 100, 2) if summaries else None
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = synth.workload(args.workload, order=args.order, q=args.quad, size=args.size)
    m, u0, dt = w["mesh"], w["u0"], w["dt"]
    M = dg.Mesh(m, renumber="morton")
    stream = torch.cuda.current_stream()

    def timed_run(prec, scheme_kw, steps, clocks):
        """warm-up + `steps` timed SSP-RK3 steps from u0; returns timing, kernel profile, state."""
        sch = dg.Scheme(precision=prec, **scheme_kw)
        ws = dg.workspace(M, sch)
        u = torch.from_numpy(M.to_lib(u0)).cuda()
        if args.shape:
            dl, db, sl, sb = (int(x) for x in args.shape.split(","))
            dg.dolinc_set_tuning(M, sch, dl, db, sl, sb)
            tune = dict(diff_lanes=dl, diff_block=db, stage_lanes=sl, stage_block=sb, forced=True)
        else:
            tune = dg.dolinc_autotune(M, sch, u, ws) if not args.no_tune else None
        dg.dolinc_rk_steps(M, sch, dt, args.warmup, u, ws)
        finite = True
        try:
            dg.dolinc_sync_status(M, ws)
        except dg.DolincError:
            finite = False
        u_prof = u.clone()          # the same start state for the profiled pass
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(local if clocks else -1) as ck:
            e0.record(stream)
            dg.dolinc_rk_steps(M, sch, dt, steps, u, ws)       # the K steps in one call: state stays on device
            e1.record(stream)
            torch.cuda.synchronize()
        ms = reduce_max(e0.elapsed_time(e1), dist)
        # each kernel's live duration: the same K steps from the same state again, with
        # CUDA events around every launch (the events add about 4% to a step, so they
        # stay out of the timed window above)
        dg.dolinc_profile_enable(M, True)
        dg.dolinc_rk_steps(M, sch, dt, steps, u_prof, ws)
        torch.cuda.synchronize()
        kms, kn = dg.profile_read(M)
        dg.dolinc_profile_enable(M, False)
        del u_prof
        try:
            dg.dolinc_sync_status(M, ws)
        except dg.DolincError:
            finite = False
        return dict(ms=ms, state=u, kms=kms, kn=kn, clocks=ck.summary() if clocks else None, sch=sch, ws=ws,
                    finite=finite, tune=tune)

    results = {args.precision: timed_run(args.precision, w["scheme"], args.steps, True)}
    if args.precision != "fp64":
        results["fp64"] = timed_run("fp64", w["scheme"], args.steps, False)
    kn_main = results[args.precision]["kn"]
    # the profile brackets the face-centric stage pair (k_flux + k_gather) as one entry
    pair = 2 if (results[args.precision]["tune"] or {}).get("stage_lanes") == -2 else 1
    launches_per_step = (int(sum(kn_main)) + (pair - 1) * int(kn_main[KINDS.index("stage")])) / args.steps
    variants = {}
    if not args.no_variants and args.workload == "euler3d_tet64":
        o0 = w["info"]["order"]
        k0, r0 = synth.STENCIL_OF_ORDER[o0]
        minimal = max(r0, k0 - r0 - 2, 1)     # differentials the stencil itself reads
        for prec, order, nd, tag in (("fp32_bf16", o0, o0 - 1, ""), (args.precision, o0, minimal, "_minimal"),
                                     ("fp64", o0, minimal, "_minimal"), (args.precision, 2, 1, ""),
                                     (args.precision, 4, 3, ""), ("fp64", 2, 1, ""), ("fp64", 4, 3, ""),
                                     (args.precision, o0, 2, "_weno5"), ("fp64", o0, 2, "_weno5")):
            k, r = synth.STENCIL_OF_ORDER[order]
            kw = dict(w["scheme"], k=k, r=r, n_diff=nd)
            if tag == "_weno5":
                kw["limiter"] = "weno5_all"
            vr = timed_run(prec, kw, args.steps, False)
            v = {"precision": prec, "scheme_order": 5 if tag == "_weno5" else order,
                 "stencil_k_r": [k, r] if tag != "_weno5" else "WENO5-DOLINC on every face", "n_diff": nd,
                 "value": M.n_cells * world * 3 * args.steps / (vr["ms"] / 1e3),
                 "ms_per_step": vr["ms"] / args.steps, "finite_after_steps": vr["finite"]}
            if order == o0 and tag != "_weno5" and "fp64" in results:
                a = vr["state"].double().cpu().numpy()
                b = results["fp64"]["state"].cpu().numpy()
                v["l2_rel_vs_fp64_after_steps"] = _l2_rel(a, b)
            variants["%s_order%d%s" % (prec, order, tag)] = v
            del vr
    stability = _stability(args, w, M, dg, torch) if (not args.no_variants and args.workload == "euler3d_tet64") \
        else None
    main = results[args.precision]
    cells = M.n_cells
    total_cells = reduce_sum(cells, dist)
    ms_step = main["ms"] / args.steps
    value = total_cells * 3 * args.steps / (main["ms"] / 1e3)
    # dominant kernel and its roofline.  When the scheme computes differential orders
    # its stencil does not read, dolinc_rk_step runs those passes on a side stream
    # concurrently with the stage kernel: the unit is then the concurrent pair, over
    # the window they share (each stage: its time minus the sequential pack share and
    # the passes the stencil reads, all measured live).
    kms, kn = main["kms"], main["kn"]
    peak, peak_src = _peaks()
    sch_m = main["sch"]
    need = max(sch_m.r, sch_m.k - sch_m.r - 2, 1)
    per = lambda kind: kms[KINDS.index(kind)] / max(kn[KINDS.index(kind)], 1)
    paired = (main["tune"] or {}).get("diff_lanes") == 2 and kn[KINDS.index("diff_pair")] > 0
    if paired:
        # paired schedule: no concurrent passes; the unit is the larger of the stage and
        # the paired differential launch
        top = max(("stage", "diff_pair"), key=lambda kd: kms[KINDS.index(kd)])
        unit = [top]
        per_launch_ms = per(top)
        unit_name = top
    elif sch_m.n_diff > need:
        unit = ["stage"] + ["diff%d" % mm for mm in range(need + 1, sch_m.n_diff + 1)]
        pack_share = kms[KINDS.index("pack")] / (3.0 * args.steps)
        per_launch_ms = ms_step / 3.0 - pack_share - sum(per("diff%d" % mm) for mm in range(1, need + 1))
        unit_name = " + ".join(unit) + " (concurrent)"
    else:
        top = int(np.argmax(kms))
        unit = [KINDS[top]]
        per_launch_ms = per(KINDS[top])
        unit_name = KINDS[top]
    bytes_alg = sum(alg_bytes(kd, M, sch_m) for kd in unit)
    bytes_table = sum(alg_bytes(kd, M, sch_m, "table") for kd in unit)
    achieved = bytes_alg / (per_launch_ms / 1e3) / 1e9
    bytes_kern = sum(kernel_bytes(kd, M, sch_m) for kd in unit)
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            tj = json.load(open(tfile))
            keys = ["%s/%s/%s/order%d" % (args.workload, args.precision, kd, w["info"].get("order", 0)) for kd in unit]
            if all(k in tj for k in keys):
                traffic = int(sum(tj[k] for k in keys))
        except Exception:
            traffic = None
    kernels = {KINDS[i]: {"ms_per_launch": round(kms[i] / kn[i], 5), "launches": int(kn[i]),
                          "share": round(kms[i] / sum(kms), 4),
                          "alg_bytes": int(alg_bytes(KINDS[i], M, main["sch"])),
                          "alg_GBs": round(alg_bytes(KINDS[i], M, main["sch"]) / (kms[i] / kn[i] / 1e3) / 1e9, 1),
                          "kernel_bytes": int(kernel_bytes(KINDS[i], M, main["sch"])),
                          "kernel_GBs": round(kernel_bytes(KINDS[i], M, main["sch"]) / (kms[i] / kn[i] / 1e3) / 1e9, 1)}
               for i in range(len(KINDS)) if kn[i] > 0}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64", "data": "synthetic",
        "config": _config(args, w, cells, M.n_faces),
        "workspace_mb": round(main["ws"].numel() / 2 ** 20, 1),
        "launch_shape": main.get("tune"),
        "roofline": {"bound": "hbm", "kernel": unit_name, "achieved": round(achieved, 1), "peak": peak,
                     "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "alg_bytes_per_launch": int(bytes_alg),
                     "alg_basis": "stored widths (FP32 geometry below FP64), stage reads orders 0..%d" % stage_orders(
                         sch_m),
                     "table_basis_bytes_per_launch": int(bytes_table),
                     "table_basis_frac": round(bytes_table / (per_launch_ms / 1e3) / 1e9 / peak, 4),
                     "kernel_bytes_per_launch": int(bytes_kern),
                     "kernel_bytes_frac": round(bytes_kern / (per_launch_ms / 1e3) / 1e9 / peak, 4),
                     "ms_per_launch": round(per_launch_ms, 5),
                     "kernel_timing": "CUDA events around every launch of the K timed steps, run a second "
                                      "time from the same start state (the events stay out of the timed "
                                      "window: they add about 4% to a step)"},
        "kernels": kernels,
        # the whole stage (differential passes + fused stage; pack per step) against the
        # scope table's B_alg per cell per stage
        "stage_roofline": _stage_roofline(M, main["sch"], ms_step / 3.0, peak),
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": main["clocks"],
    }
    if variants:
        line["variants"] = variants
    if stability:
        line["stability"] = stability
    if summaries:
        line["indicator"] = _indicator_summary(args)
        line["batch"] = _batch_summary(args)
        line["semi_implicit"] = _implicit_summary(args, imp_inputs)
    line["finite_after_steps"] = main["finite"]
    if "fp64" in results and args.precision != "fp64":
        f = results["fp64"]
        v64 = total_cells * 3 * args.steps / (f["ms"] / 1e3)
        a = main["state"].double().cpu().numpy()
        b = f["state"].cpu().numpy()
        l2 = _l2_rel(a, b)
        line["fp64_gpu"] = {"value": v64, "ms_per_step": f["ms"] / args.steps,
                            "speedup_mixed_vs_fp64": value / v64,
                            "l2_rel_mixed_vs_fp64_after_steps": l2, "steps_compared": args.steps + args.warmup}
        fr = _fp64_roofline(args, w, M, f)
        if fr:
            line["fp64_gpu"]["roofline"] = fr
    # e2e: the public call with a host state (pinned): every step moves the state from
    # host memory into the step's first kernel and the new state back to host memory
    # from its last one, inside the timed region
    sch = main["sch"]
    ws = main["ws"]
    uh = torch.from_numpy(M.to_lib(u0)).pin_memory()
    ud = torch.empty_like(uh, device="cuda")
    for _ in range(2):
        dg.dolinc_rk_step_host(M, sch, dt, uh, ud, ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        dg.dolinc_rk_step_host(M, sch, dt, uh, ud, ws)
    e1.record(stream)
    torch.cuda.synchronize()
    ems = reduce_max(e0.elapsed_time(e1), dist)
    nbytes = uh.numel() * 8
    line["e2e"] = {"value": total_cells * 3 * args.steps / (ems / 1e3), "unit": UNIT,
                   "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                   "ms_per_step": ems / args.steps}
    # full-size accuracy of one stage against the FP64 oracle, and the CPU baseline
    if rank == 0 and not args.no_oracle:
        import oracle
        osch = oracle.Scheme(**w["scheme"])
        Op = oracle.Oracle(m, parallel=True)
        tomp, ref = _oracle_stage_seconds(Op, u0, osch, dt)
        nthr = oracle.threads(parallel=True)
        del Op
        O = oracle.Oracle(m)
        tcpu, ref1 = _oracle_stage_seconds(O, u0, osch, dt)
        assert np.array_equal(ref, ref1)
        acc = {}
        for prec, r in results.items():
            out = torch.zeros_like(torch.from_numpy(u0)).cuda()
            ud.copy_(torch.from_numpy(M.to_lib(u0)))
            dg.dolinc_rk_stage(M, r["sch"], dt, 0, ud, ud, out, r["ws"])
            got = M.from_lib(out.cpu().numpy())
            inc, inc_ref = got - u0, ref - u0
            acc[prec] = {"l2_rel_stage_increment": float(np.sqrt(((inc - inc_ref) ** 2).sum() / (inc_ref ** 2).sum())),
                         "linf_rel_stage_increment": float(np.abs(inc - inc_ref).max() / np.abs(inc_ref).max())}
            if prec != "fp64":
                acc[prec]["worst_cell_over_per_face_1e-5_bound"] = _increment_bound_ratio(O, inc, inc_ref, u0, dt,
                                                                                          w["scheme"])
        line["accuracy_vs_oracle"] = acc
        line["cpu_baseline"] = {"value": cells / tomp, "unit": UNIT, "cores": nthr, "kind": "oracle",
                                "sample": "one SSP-RK3 stage (stage 0) of the full %s workload (%d cells), "
                                          "FP64 C oracle, OpenMP build on %d threads (face fluxes in "
                                          "parallel, sums in face order)" % (args.workload, cells, nthr),
                                "seconds": tomp,
                                "single_thread": {"value": cells / tcpu, "cores": 1, "seconds": tcpu},
                                "host": _host_info()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _stability(args, w, M, dg, torch):
    """The workload's scheme run to t = args.stab_time on the full mesh, FP32 bulk:
    unlimited (the timed configuration), with the skewness correction, and with the
    troubled-cell criterion switching flagged faces to the first-order fallback
    (criterion evaluated every step, inside the timing).  Each: whether the state
    stayed finite with positive density, the first time it did not, and the
    throughput of the whole run."""
    import numpy as np
    m, u0, dt = w["mesh"], w["u0"], w["dt"]
    steps = int(np.ceil(args.stab_time / dt - 1e-9))
    out = {}
    Ms = None
    for tag, skew, limiter in (("plain", False, "none"), ("skew_corrected", True, "none"),
                               ("criterion_first_order", False, "first_order_flagged")):
        if skew:
            Ms = dg.Mesh(m, renumber="morton")
            dg.dolinc_mesh_set_skew_correction(Ms, True)
        X = Ms if skew else M
        sch = dg.Scheme(precision=args.precision, limiter=limiter, **w["scheme"])
        flags = None
        if limiter != "none":
            flags = torch.zeros(X.n_cells, dtype=torch.uint8, device="cuda")
            dg.dolinc_set_flags(X, flags)
        ws = dg.workspace(X, sch)
        u = torch.from_numpy(X.to_lib(u0)).cuda()
        dg.dolinc_autotune(X, sch, u, ws)
        t_bad, done, ms = None, 0, 0.0
        chunk = 50
        while done < steps and t_bad is None:
            n = min(chunk, steps - done)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(n):
                if flags is not None:
                    dg.dolinc_criterion(X, sch, u, flags, ws)
                dg.dolinc_rk_step(X, sch, dt, u, ws)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            done += n
            ok = True
            try:
                dg.dolinc_sync_status(X, ws)
            except dg.DolincError:
                ok = False
            rho_min = float(u[0].min().item())
            if not ok or not np.isfinite(rho_min) or rho_min <= 0:
                t_bad = done * dt
        r = {"t_end": steps * dt, "steps_run": done, "finite_to_t_end": t_bad is None,
             "first_failure_by_t": t_bad, "rho_min_end": float(u[0].min().item()) if t_bad is None else None,
             "value": X.n_cells * 3 * done / (ms / 1e3), "ms_per_step": ms / done}
        if flags is not None:
            r["flagged_fraction_end"] = float(flags.float().mean().item())
            dg.dolinc_set_flags(X, None)
        out[tag] = r
        del ws, u
    del Ms
    return out


def _sync_cpu(t):
    return t.cpu().numpy()


def _indicator_summary(args):
    """The learned indicator inside the default run, small but in the full
    configuration: a network trained on a few criterion-labelled runs of a reduced mesh,
    then the full 724^2 Riemann mesh advanced with the network switching flagged faces
    to the first-order fallback (FP32) against the criterion doing it (FP32 and the
    plain FP64 GPU method)."""
    a = argparse.Namespace(**vars(args))
    a.ind_runs, a.ind_eval_runs, a.ind_train_size, a.ind_train_steps, a.ind_epochs = 4, 1, 96, 40, 10
    a.size, a.steps = None, 20
    return run_indicator(a, emit=False, forms=("network_fp32", "criterion_fp32", "criterion_fp64"))


def _batch_summary(args):
    """The batched ensemble inside the default run: 64 meshes of the 512-mesh
    distribution, one persistent launch per stage from a CUDA graph, FP32 bulk / FP64
    update, against each mesh stepped by its own FP64 launches."""
    a = argparse.Namespace(**vars(args))
    a.batch_meshes, a.steps, a.warmup = 64, 10, 3
    return run_batch(a, emit=False)


def run_indicator(args, emit=True, forms=None):
    """Learned troubled-cell indicator on the four-quadrant Riemann workload.

    Trains the network on criterion labels of seeded runs (smaller mesh), measures its
    misclassification on held-out runs, then advances one held-out problem on the full
    mesh with the limiter switched by (a) the network, FP32, (b) the criterion, FP32,
    (c) the criterion, FP64 (the plain FP64 GPU method), flagged faces taking the
    first-order fallback; the same with ENO3-DOLINC on flagged faces; no limiter; ENO3
    everywhere.  Reports cell-updates/s per stage (indicator included), whether each
    run stayed finite, and the L1 distance to (c)."""
    import torch
    import paper_2404_08952_gb300 as dg
    from paper_2404_08952_gb300 import indicator as ind
    import synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t_all = time.perf_counter()
    train_size, run_steps, every = args.ind_train_size, args.ind_train_steps, 4
    mk = lambda sd: synth.workload("euler2d_riemann", size=train_size, order=sd, q=2)
    Xs, Ys = [], []
    for x, y in ind.riemann_runs(mk, range(args.ind_runs), run_steps, every, precision=args.precision):
        Xs.append(x)
        Ys.append(y)
    X, Y = torch.cat(Xs), torch.cat(Ys)
    net = dg.MLP(seed=args.seed)
    t0 = time.perf_counter()
    hist, pw = ind.train(net, X, Y, epochs=args.ind_epochs, batch=8192, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # held-out evaluation (seeds never trained on)
    Xh, Yh = [], []
    for x, y in ind.riemann_runs(mk, range(1000, 1000 + args.ind_eval_runs), run_steps, every,
                                 precision=args.precision):
        Xh.append(x)
        Yh.append(y)
    Xh, Yh = torch.cat(Xh), torch.cat(Yh)
    pred = torch.zeros_like(Yh)
    net.forward(Xh, None, pred)
    conf = ind.confusion(_sync_cpu(pred), _sync_cpu(Yh))
    # full-size comparison on one held-out problem
    w = synth.workload("euler2d_riemann", size=args.size or 724, order=2000, q=2)
    cells = int(w["u0"].shape[1])
    steps = args.steps
    res = {}
    fo, eno = "first_order_flagged", "eno3_flagged"
    for name, switch, prec, lim in (("network_fp32", "network", "fp32", fo), ("criterion_fp32", "criterion", "fp32", fo),
                                    ("criterion_fp64", "criterion", "fp64", fo),
                                    ("network_eno3_fp32", "network", "fp32", eno),
                                    ("criterion_eno3_fp64", "criterion", "fp64", eno),
                                    ("none_fp32", "none", "fp32", fo), ("eno3_all_fp32", "all", "fp32", fo)):
        if forms is not None and name not in forms:
            continue
        st, finite, sec, flagged = ind.run_with(w, switch, steps, precision=prec, net=net, flagged_limiter=lim)
        res[name] = dict(state=st, finite=finite, sec_per_step=sec, flagged=flagged,
                         value=cells * 3 / sec)
    ref = res["criterion_fp64"]["state"]
    vol = None
    out = {}
    for k, r in res.items():
        d = r["state"] - ref
        l1 = float(np.abs(d).sum() / max(np.abs(ref).sum(), 1e-300)) if r["finite"] else None
        out[k] = {"value": r["value"], "ms_per_step": r["sec_per_step"] * 1e3, "finite_after_steps": r["finite"],
                  "flagged_fraction": r["flagged"], "l1_rel_vs_criterion_fp64": l1}
    line = {"metric": METRIC, "value": out["network_fp32"]["value"], "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": 0, "ms_per_step": out["network_fp32"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "euler2d_riemann", "cells": cells, "stencil_k_r": [3, 1], "n_diff": 2,
                       "limiter": "first-order fallback on faces of flagged cells (ENO3-DOLINC rows: *_eno3_*)",
                       "indicator": "MLP 24-64-64-64-1 (bf16 weights)",
                       "train_mesh_cells": int(2 * train_size ** 2), "train_runs": args.ind_runs,
                       "train_samples": int(X.shape[0]), "eval_runs": args.ind_eval_runs},
            "indicator": {"train_seconds": t_train, "epochs": args.ind_epochs, "final_loss": hist[-1],
                          "first_loss": hist[0], "pos_weight": pw, "heldout_vs_criterion": conf},
            "forms": out, "seconds_total": time.perf_counter() - t_all}
    if not emit:
        return {"config": line["config"], "indicator": {k: v for k, v in line["indicator"].items()},
                "forms": out, "seconds_total": line["seconds_total"]}
    print(json.dumps(line), flush=True)


def run_batch(args, emit=True):
    """Batched ensemble of 2D Burgers meshes: one persistent cooperative launch per
    stage replayed from a CUDA graph (FP32 bulk, FP64 update), against the plain FP64
    GPU method (each mesh stepped by its own launches)."""
    import torch
    import paper_2404_08952_gb300 as dg
    import synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    t_all = time.perf_counter()
    wl = synth.workload("burgers_batch", q=2, n_meshes=args.batch_meshes)
    ms_ = wl["meshes"]
    meshes = [dg.Mesh(x["mesh"]) for x in ms_]
    bt = dg.Batch(meshes)
    cells = int(bt.n_cells)
    dt = torch.tensor([x["dt"] for x in ms_], dtype=torch.float64, device="cuda")
    u0 = bt.to_lib([x["u0"] for x in ms_])
    out = {}
    for prec in (args.precision, "fp64"):
        sch = dg.Scheme(precision=prec, **wl["scheme"])
        ws = bt.workspace(sch)
        u = torch.from_numpy(u0).cuda()
        tune = bt.autotune(sch, dt, u, ws)
        for _ in range(args.warmup):
            bt.rk_step(sch, dt, u, ws, use_graph=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            bt.rk_step(sch, dt, u, ws, use_graph=True)
        e1.record()
        torch.cuda.synchronize()
        dg.dolinc_sync_status(meshes[0], ws)
        msb = e0.elapsed_time(e1) / args.steps
        out["batched_" + prec] = {"value": cells * 3 / (msb / 1e3), "ms_per_step": msb, "launch_shape": tune,
                                  "gpu_launches_per_step": 3, "state": u.cpu().numpy()}
        del ws
    # plain per-mesh FP64 path (each mesh: its own pack/differential/stage launches)
    sch = dg.Scheme(precision="fp64", **wl["scheme"])
    wss = [dg.workspace(M, sch) for M in meshes]
    us = [torch.from_numpy(M.to_lib(x["u0"])).cuda() for M, x in zip(meshes, ms_)]
    for _ in range(args.warmup):
        for M, x, u, ws in zip(meshes, ms_, us, wss):
            dg.dolinc_rk_step(M, sch, x["dt"], u, ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        for M, x, u, ws in zip(meshes, ms_, us, wss):
            dg.dolinc_rk_step(M, sch, x["dt"], u, ws)
    e1.record()
    torch.cuda.synchronize()
    msp = e0.elapsed_time(e1) / args.steps
    per_mesh = np.concatenate([u.cpu().numpy() for u in us], axis=-1)
    out["per_mesh_fp64"] = {"value": cells * 3 / (msp / 1e3), "ms_per_step": msp,
                            "gpu_launches_per_step": len(meshes) * (1 + 3 * (sch.n_diff + 1))}
    ref = out["batched_fp64"]["state"]
    for k in ("batched_" + args.precision, "batched_fp64"):
        st = out[k].pop("state")
        out[k]["l2_rel_vs_per_mesh_fp64"] = float(np.sqrt(((st - per_mesh) ** 2).sum() / (per_mesh ** 2).sum()))
    line = {"metric": METRIC, "value": out["batched_" + args.precision]["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["batched_" + args.precision]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64",
            "data": "synthetic",
            "config": {"workload": "burgers_batch", "meshes": len(meshes), "cells": cells,
                       "min_cells": int(min(M.n_cells for M in meshes)), "max_cells": int(max(M.n_cells for M in meshes)),
                       "stencil_k_r": [3, 1], "n_diff": 2, "flux": "burgers"},
            "forms": out, "seconds_total": time.perf_counter() - t_all}
    if not emit:
        return {"config": line["config"], "forms": out, "seconds_total": line["seconds_total"]}
    print(json.dumps(line), flush=True)


def run_hexprism(args):
    """Gaussian-pulse advection on the mixed hex/prism mesh (+-20% jitter, periodic).

    Throughput of scheme orders 2..5 (differentials through order p-1) in FP64, FP32
    and FP32 with BF16-stored orders >= 2 at one lattice size, and a convergence sweep:
    each order advanced in FP32 and FP64 to t = T on several lattice sizes, the L2 error
    sqrt(sum V e^2 / sum V) against the exact cell averages of the translated pulse, and
    the measured order between consecutive sizes."""
    import synth
    from synth import fields
    t_all = time.perf_counter()
    workers = max(1, min(16, os.cpu_count() or 1))
    size = args.size or 140
    sizes = sorted(int(x) for x in args.hp_sizes.split(",") if x)
    T = args.hp_time
    orders = (2, 3, 4, 5)
    # host inputs first: the forked quadrature runs before CUDA is initialised
    host = {}
    for n in sorted(set(sizes + [size])):
        t0 = time.perf_counter()
        w = synth.workload("adv3d_hexprism", order=5, size=n, q=args.hp_quad, workers=workers)
        a = np.asarray(w["scheme"]["adv"], dtype=np.float64)
        exact = None
        if n in sizes:
            c = tuple(0.5 + a[k] * T for k in range(3))
            exact = fields.cell_average(w["mesh"], lambda p, c=c: fields.gaussian3d(p, centre=c), q=args.hp_quad,
                                        workers=workers)
        host[n] = (w, exact, time.perf_counter() - t0)
    import torch
    import paper_2404_08952_gb300 as dg
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    thr = {}
    w, _, _ = host[size]
    M = dg.Mesh(w["mesh"], renumber="morton")
    cells = M.n_cells
    peak, peak_src = _peaks()
    for order in orders:
        k, r = synth.STENCIL_OF_ORDER[order]
        for prec in ("fp64", "fp32", "fp32_bf16"):
            if prec == "fp32_bf16" and order < 3:
                continue
            sch = dg.Scheme(precision=prec, **dict(w["scheme"], k=k, r=r, n_diff=order - 1))
            ws = dg.workspace(M, sch)
            u = torch.from_numpy(M.to_lib(w["u0"])).cuda()
            tune = dg.dolinc_autotune(M, sch, u, ws)
            dg.dolinc_rk_steps(M, sch, w["dt"], args.warmup, u, ws)
            u_prof = u.clone()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dg.dolinc_rk_steps(M, sch, w["dt"], args.steps, u, ws)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            # kernel durations from a second pass with per-launch events (outside the window)
            dg.dolinc_profile_enable(M, True)
            dg.dolinc_rk_steps(M, sch, w["dt"], args.steps, u_prof, ws)
            torch.cuda.synchronize()
            kms, kn = dg.profile_read(M)
            dg.dolinc_profile_enable(M, False)
            del u_prof
            finite = True
            try:
                dg.dolinc_sync_status(M, ws)
            except dg.DolincError:
                finite = False
            top = int(np.argmax(kms))
            pl = kms[top] / max(kn[top], 1)
            ab = alg_bytes(KINDS[top], M, sch)
            thr["%s_order%d" % (prec, order)] = {
                "value": cells * 3 * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                "finite_after_steps": finite, "launch_shape": tune,
                "top_kernel": KINDS[top], "top_share": round(kms[top] / sum(kms), 4),
                "top_alg_GBs": round(ab / (pl / 1e3) / 1e9, 1), "top_frac_of_peak": round(ab / (pl / 1e3) / 1e9 / peak, 4)}
            del ws, u
    del M
    conv = {}
    for prec, skew in (("fp32", False), ("fp64", False), ("fp32", True), ("fp64", True)):
        for order in orders:
            k, r = synth.STENCIL_OF_ORDER[order]
            row = []
            for n in sizes:
                w, exact, _ = host[n]
                Mn = dg.Mesh(w["mesh"], renumber="morton")
                if skew:
                    dg.dolinc_mesh_set_skew_correction(Mn, True)
                sch = dg.Scheme(precision=prec, **dict(w["scheme"], k=k, r=r, n_diff=order - 1))
                ws = dg.workspace(Mn, sch)
                u = torch.from_numpy(Mn.to_lib(w["u0"])).cuda()
                dg.dolinc_autotune(Mn, sch, u, ws)
                nsteps = int(np.ceil(T / w["dt"] - 1e-9))
                dt = T / nsteps
                for _ in range(nsteps):
                    dg.dolinc_rk_step(Mn, sch, dt, u, ws)
                finite = True
                try:
                    dg.dolinc_sync_status(Mn, ws)
                except dg.DolincError:
                    finite = False
                got = Mn.from_lib(u.cpu().numpy())[0]
                V = Mn.from_lib(Mn.geometry()["V"])
                e = got - exact
                l2 = float(np.sqrt((V * e * e).sum() / V.sum())) if finite else None
                row.append({"lattice": n, "cells": Mn.n_cells, "steps": nsteps, "finite": finite, "l2": l2,
                            "linf": float(np.abs(e).max()) if finite else None})
                del ws, u, Mn
            for a_, b_ in zip(row, row[1:]):
                if a_["l2"] and b_["l2"]:
                    b_["order_vs_previous"] = float(np.log(a_["l2"] / b_["l2"]) / np.log(b_["lattice"] / a_["lattice"]))
            conv["%s_order%d%s" % (prec, order, "_skew" if skew else "")] = row
    main = thr["fp32_order5"]
    line = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "adv3d_hexprism", "lattice": size, "cells": cells, "headline": "fp32_order5",
                       "flux": "upwind", "adv": list(w["scheme"]["adv"]), "jitter": 0.2,
                       "convergence_time": T, "convergence_lattices": sizes, "quad": args.hp_quad,
                       "peak_GBs": peak, "peak_source": peak_src},
            "forms": thr, "convergence": conv,
            "host_input_seconds": {str(n): round(v[2], 1) for n, v in host.items()},
            "seconds_total": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)


def solve_alg_bytes(M, iterations, solves):
    """Algorithmic bytes of the semi-implicit solve launches: per cell and BiCGSTAB
    iteration the three phases' FP64 vectors (A: p, rh read, v written; B: r, v, rh
    read, s, t written; C: s, p, x, t, v read, x, r, p written) and the scaled rows
    read in A and B (per slot an 8 B coefficient and a 4 B neighbour, per cell a 4 B
    offset); per solve the set-up (R and the row scale read; r, rh, p, x written) and
    the final u += x (x, u read, u written).  Neighbour re-reads are not counted."""
    nc, ns = M.n_cells, M.n_slots
    per_it = nc * 8 * (3 + 5 + 8) + 2 * (ns * 12 + nc * 4)
    per_solve = nc * 8 * (2 + 4) + nc * 8 * 3
    return iterations * per_it + solves * per_solve


def _implicit_inputs(args, size, q):
    """Host inputs of the semi-implicit workload (mesh, initial and exact cell averages
    at t = imp_time), computed by forked workers: call before CUDA is initialised."""
    import synth
    from synth import fields
    t0 = time.perf_counter()
    workers = max(1, min(16, os.cpu_count() or 1))
    w = synth.workload("adv3d_hexprism", order=3, size=size, q=q, workers=workers)
    a = np.asarray(w["scheme"]["adv"], dtype=np.float64)
    c = tuple(0.5 + a[k] * args.imp_time for k in range(3))
    exact = fields.cell_average(w["mesh"], lambda p: fields.gaussian3d(p, centre=c), q=q, workers=workers)
    return dict(w=w, exact=exact, size=size, q=q, seconds=time.perf_counter() - t0)


def run_implicit(args, emit=True, forms=None, inputs=None, rk3_orders=(3, 5)):
    """Semi-implicit DOLINC steps (Sec 2.4: the weight part of every face value at the
    new level, c_r explicit) of the Gaussian pulse on the mixed hex/prism mesh.

    Throughput of one step (explicit residual + one BiCGSTAB solve in one cooperative
    launch) at dt = imp_dt_factor times the explicit step, for backward Euler and
    Crank-Nicolson (one and two outer iterations), FP32 and FP64 residuals, orders 3
    and 5; the solve kernel's roofline; and, to t = imp_time, the L2 error against the
    exact translated pulse beside SSP-RK3 at the explicit step, with each run's time.
    emit=False returns the line instead of printing it; forms and inputs restrict the
    forms and supply precomputed host inputs (_implicit_inputs)."""
    import synth
    t_all = time.perf_counter()
    if inputs is None:
        inputs = _implicit_inputs(args, args.size or 140, args.hp_quad)
    w, exact, size = inputs["w"], inputs["exact"], inputs["size"]
    a = np.asarray(w["scheme"]["adv"], dtype=np.float64)
    T = args.imp_time
    t_host = inputs["seconds"]
    import torch
    import paper_2404_08952_gb300 as dg
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    M = dg.Mesh(w["mesh"], renumber="morton")
    cells = M.n_cells
    V = M.from_lib(M.geometry()["V"])
    peak, peak_src = _peaks()
    dt_exp = w["dt"]
    dt = args.imp_dt_factor * dt_exp
    h = 1.0 / size
    # (precision, scheme order, theta, outer iterations, warm start, row layout: None = default per slot,
    #  6 = ELL of width 6)
    # warm start: 0 from zero, 1 from the last step's solution, 2 extrapolated from the last two
    # (Crank-Nicolson damps no mode, so its increments' high-frequency parts alternate and
    # extrapolation does not pay there; backward Euler's do not)
    forms = forms or [("fp32", 3, 0.5, 1, 1, None), ("fp32", 3, 0.5, 1, 0, None), ("fp32", 3, 0.5, 1, 2, None),
             ("fp32", 3, 0.5, 1, 1, 6), ("fp32", 3, 1.0, 1, 2, None), ("fp32", 3, 1.0, 1, 1, None),
             ("fp64", 3, 0.5, 1, 1, None), ("fp32", 3, 0.5, 2, 1, None), ("fp32", 5, 0.5, 2, 1, None),
             ("fp32", 5, 1.0, 1, 2, None)]

    exact = np.asarray(exact, dtype=np.float64).reshape(-1)

    def l2(u):
        e = M.from_lib(u.cpu().numpy())[0] - exact
        return float(np.sqrt((V * e * e).sum() / V.sum()))

    def timed_steps(fn, n):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    out = {}
    for prec, order, theta, n_outer, warm, layout in forms:
        k, r = synth.STENCIL_OF_ORDER[order]
        sch = dg.Scheme(precision=prec, **dict(w["scheme"], k=k, r=r, n_diff=order - 1))
        ws = dg.workspace(M, sch)
        S = dg.Implicit(M, sch, dt, theta)
        if layout is not None:
            S.set_layout(layout)
        S.set_solver(rel_tol=args.imp_tol, max_iter=500, warm_start=warm)
        u = torch.from_numpy(M.to_lib(w["u0"])).cuda()
        for _ in range(args.warmup):
            S.step(u, ws, n_outer)
        i0 = S.info()
        dg.dolinc_profile_enable(M, True)
        ms = timed_steps(lambda: S.step(u, ws, n_outer), args.steps)
        i1 = S.info()
        kms, kn = dg.profile_read(M)
        dg.dolinc_profile_enable(M, False)
        iters = i1["total_iterations"] - i0["total_iterations"]
        solves = i1["total_solves"] - i0["total_solves"]
        ks = KINDS.index("solve")
        solve_ms = kms[ks] / max(kn[ks], 1)
        ab = solve_alg_bytes(M, iters / max(solves, 1), 1)
        gbs = ab / (solve_ms / 1e3) / 1e9
        # accuracy to T: the implicit steps, dt rounded to divide T
        nI = int(np.ceil(T / dt - 1e-9))
        S2 = dg.Implicit(M, sch, T / nI, theta)
        if layout is not None:
            S2.set_layout(layout)
        S2.set_solver(rel_tol=args.imp_tol, max_iter=500, warm_start=warm)
        u = torch.from_numpy(M.to_lib(w["u0"])).cuda()
        conv = True
        its = []
        for _ in range(nI):
            S2.step(u, ws, n_outer)
            inf = S2.info()
            conv = conv and inf["converged"]
            its.append(inf["iterations"])
        u = torch.from_numpy(M.to_lib(w["u0"])).cuda()
        S2.set_solver(rel_tol=args.imp_tol, max_iter=500, warm_start=warm)
        ms_T = timed_steps(lambda: S2.step(u, ws, n_outer), nI)
        name = "%s_order%d_theta%g_outer%d%s%s" % (prec, order, theta, n_outer, ("", "_warm", "_extrap")[warm],
                                                   "_ell%d" % layout if layout else "")
        out[name] = {
            "value": cells * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
            "iterations_per_solve": iters / max(solves, 1), "solves": solves, "launches": int(sum(kn)),
            "row_layout": S.layout,
            "kernel_ms_share": {KINDS[i]: round(kms[i] / sum(kms), 4) for i in range(len(KINDS)) if kn[i]},
            "solve_roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                               "frac": round(gbs / peak, 4), "alg_bytes_per_cell_iteration":
                                   round(solve_alg_bytes(M, 1, 0) / cells, 1), "ms_per_solve": round(solve_ms, 4)},
            "to_time": {"t": T, "steps": nI, "dt": T / nI, "l2": l2(u), "converged": conv,
                        "iterations_per_step": its, "ms": round(ms_T, 3)}}
        del ws, S, S2, u
    # SSP-RK3 at the explicit step to the same time
    expl = {}
    for prec, order in (("fp32", o) for o in rk3_orders):
        k, r = synth.STENCIL_OF_ORDER[order]
        sch = dg.Scheme(precision=prec, **dict(w["scheme"], k=k, r=r, n_diff=order - 1))
        ws = dg.workspace(M, sch)
        u = torch.from_numpy(M.to_lib(w["u0"])).cuda()
        dg.dolinc_autotune(M, sch, u, ws)
        nE = int(np.ceil(T / dt_exp - 1e-9))
        dg.dolinc_rk_steps(M, sch, T / nE, 2, u, ws)
        u = torch.from_numpy(M.to_lib(w["u0"])).cuda()
        msE = timed_steps(lambda: dg.dolinc_rk_steps(M, sch, T / nE, nE, u, ws), 1)
        expl["%s_order%d_rk3" % (prec, order)] = {"steps": nE, "dt": T / nE, "ms": round(msE, 3), "l2": l2(u)}
        del ws, u
    head = "fp32_order3_theta0.5_outer1_warm"
    main = out[head]
    cpu = None
    if not args.no_oracle:      # the oracle's step (sparse LU) on a bounded sample of the workload
        import oracle
        ws_ = synth.workload("adv3d_hexprism", order=3, size=24, q=2)
        O = oracle.Oracle(ws_["mesh"], parallel=True)
        so = oracle.Scheme(k=3, r=1, n_diff=2, flux="upwind", nv=1, adv=tuple(a))
        t0 = time.perf_counter()
        O.semi_implicit_step(ws_["u0"], so, args.imp_dt_factor * ws_["dt"], 0.5)
        tc = time.perf_counter() - t0
        cpu = {"value": O.n_cells / tc, "unit": "cell-updates/s", "cores": oracle.threads(), "kind": "oracle",
               "sample": "one Crank-Nicolson semi-implicit step (explicit residual + direct sparse LU solve) on "
                         "the 24^3 hex/prism lattice (%d cells), %.1f s" % (O.n_cells, tc)}
    line = {"metric": "cell-updates/s per semi-implicit step (residual + linear solve)", "value": main["value"],
            "unit": "cell-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 residual, f64 solve", "data": "synthetic",
            "config": {"workload": "adv3d_hexprism_implicit", "lattice": size, "cells": cells,
                       "headline": head, "flux": "upwind", "adv": list(w["scheme"]["adv"]),
                       "jitter": 0.2, "dt": dt, "dt_explicit": dt_exp, "cfl_sum": float(np.abs(a).sum() * dt / h),
                       "rel_tol": args.imp_tol, "time": T, "quad": inputs["q"], "peak_GBs": peak,
                       "peak_source": peak_src, "l2_flush": "inputs larger than L2 (vectors and rows > 300 MB)"},
            "roofline": main["solve_roofline"], "gpu_launches": main["launches"],
            "vs_explicit_rk3": {"t": T, "semi_implicit_ms": main["to_time"]["ms"], "semi_implicit_l2": main["to_time"]["l2"],
                                "rk3_ms": expl["fp32_order3_rk3"]["ms"], "rk3_l2": expl["fp32_order3_rk3"]["l2"],
                                "speedup": round(expl["fp32_order3_rk3"]["ms"] / main["to_time"]["ms"], 3)},
            "cpu_baseline": cpu, "forms": out, "explicit_rk3": expl, "host_input_seconds": round(t_host, 1),
            "seconds_total": time.perf_counter() - t_all}
    if not emit:
        return line
    print(json.dumps(line), flush=True)


def _implicit_summary(args, inputs):
    """The semi-implicit variant inside the default run, on a reduced mesh (the 100^3
    hex/prism lattice, 1.5M cells; inputs built before CUDA starts): Crank-Nicolson from
    the previous solution and backward Euler from the extrapolated one, each to t =
    imp_time beside SSP-RK3 USR3 at the explicit step."""
    a = argparse.Namespace(**vars(args))
    a.steps, a.warmup, a.no_oracle, a.size = 10, 3, True, inputs["size"]
    line = run_implicit(a, emit=False, inputs=inputs, rk3_orders=(3,),
                        forms=[("fp32", 3, 0.5, 1, 1, None), ("fp32", 3, 1.0, 1, 2, None)])
    keep = ("metric", "value", "unit", "ms_per_step", "config", "roofline", "vs_explicit_rk3", "forms",
            "explicit_rk3", "host_input_seconds", "seconds_total")
    return {k: line[k] for k in keep}


def bl_mesh(growth, h0=0.002, ymax=0.3, nx=12, nz=3, x0=0.5, x1=1.0, dz=0.01):
    """Boundary-layer mesh: hexes over x in [x0, x1] (transmissive ends), wall-normal
    spacing h0 growing by `growth` up to ymax, nz cells of width dz across
    (periodic); Dirichlet faces on the wall (y = 0) and on the top."""
    import synth
    ys = [0.0]
    h = h0
    while ys[-1] < ymax:
        ys.append(ys[-1] + h)
        h *= growth
    m = synth.hex_mesh(np.linspace(x0, x1, nx + 1), np.array(ys), np.linspace(0.0, nz * dz, nz + 1),
                       periodic=(False, False, True))
    return m


def run_blasius(args):
    """Single-step reconstruction on laminar boundary-layer meshes (the paper's
    boundary-layer case, with its own Blasius data: cell averages of the Blasius
    velocity, Dirichlet wall and top faces).  For wall-normal growth rates 1.1..1.5 and
    stencils USR3, CSR4, USR5: the L2 error of the reconstructed wall-parallel face
    values (both orientations) against the Blasius solution at the face centres, the
    GPU's agreement with the oracle, and the residual throughput with Dirichlet walls
    on a 1.2M-cell mesh of the same family."""
    import synth
    from synth import fields
    import oracle
    t_all = time.perf_counter()
    growths = (1.1, 1.2, 1.3, 1.4, 1.5)
    stencils = ((3, 1, 1), (4, 1, 1), (5, 2, 2))
    host = {}
    for g in growths:
        m = bl_mesh(g)
        O = oracle.Oracle(m)
        bnd = O.neigh < 0
        cap = bnd & ((np.abs(O.xf[:, 1]) < 1e-12) | (O.xf[:, 1] > 0.29))
        m["boundary_kind"] = np.where(cap, 2, np.where(bnd, 1, 0)).astype(np.int32)
        ex = fields.blasius(O.xf)
        u0 = synth.cell_average(m, fields.blasius, q=4, nv=2)
        rows = (~bnd) & (np.abs(O.S[:, 1]) > 0.5 * np.linalg.norm(O.S, axis=1))
        host[g] = (m, O, cap, ex, u0, rows)
    import torch
    import paper_2404_08952_gb300 as dg
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    forms = {}
    worst = 0.0
    for g in growths:
        m, O, cap, ex, u0, rows = host[g]
        M = dg.Mesh(m)
        for (k, r, nd) in stencils:
            key = "growth%.1f_k%d_r%d" % (g, k, r)
            out = {"cells": M.n_cells}
            for prec in ("fp64", "fp32"):
                errs = []
                for v, name in ((0, "u"), (1, "v")):
                    bval = np.where(cap, np.where(np.abs(O.xf[:, 1]) < 1e-12, 0.0, ex[:, v]), 0.0)[None]
                    dg.dolinc_set_boundary_values(M, bval)
                    sch = dg.Scheme(k=k, r=r, n_diff=nd, nv=1, precision=prec, flux="upwind", adv=(1.0, 0.0, 0.0))
                    ws = dg.workspace(M, sch)
                    fL = torch.zeros((1, O.n_faces), dtype=torch.float64, device="cuda")
                    fR = torch.zeros_like(fL)
                    dg.dolinc_reconstruct_faces(M, sch, torch.from_numpy(M.to_lib(u0[v:v + 1])).cuda(), fL, fR, ws)
                    L, R = fL.cpu().numpy()[0], fR.cpu().numpy()[0]
                    e = np.concatenate([L[rows] - ex[rows, v], R[rows] - ex[rows, v]])
                    errs.append(float(np.sqrt(np.mean(e ** 2)) / np.abs(ex[rows, v]).max()))
                    if prec == "fp64":
                        osch = oracle.Scheme(k=k, r=r, n_diff=nd, flux="upwind", adv=(1.0, 0.0, 0.0),
                                             bkind=m["boundary_kind"], bval=bval)
                        OL, OR, _, _ = O.face_values(u0[v:v + 1], osch)
                        d = max(np.abs(L - OL[0]).max(), np.abs(R - OR[0]).max()) / np.abs(OL).max()
                        worst = max(worst, float(d))
                out["l2_rel_error_u_" + prec], out["l2_rel_error_v_" + prec] = errs
            forms[key] = out
    # residual throughput with Dirichlet walls on a large mesh of the family
    m = bl_mesh(1.1, nx=400, nz=100)
    bnd = np.asarray(m["face_neighbour"]) < 0
    nb = np.asarray(m["face_owner"]).shape[0]
    kinds = np.where(bnd, 2, 0).astype(np.int32)
    m["boundary_kind"] = kinds
    M = dg.Mesh(m)
    dg.dolinc_set_boundary_values(M, np.zeros((1, nb)))
    sch = dg.Scheme(k=3, r=1, n_diff=2, nv=1, precision="fp32", flux="upwind", adv=(1.0, 0.0, 0.0))
    ws = dg.workspace(M, sch)
    u = torch.ones((1, M.n_cells), dtype=torch.float64, device="cuda")
    Rr = torch.zeros_like(u)
    dg.dolinc_autotune(M, sch, u, ws)
    for _ in range(args.warmup):
        dg.dolinc_residual(M, sch, u, Rr, ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        dg.dolinc_residual(M, sch, u, Rr, ws)
    e1.record()
    torch.cuda.synchronize()
    dg.dolinc_sync_status(M, ws)
    ms = e0.elapsed_time(e1) / args.steps
    line = {"metric": METRIC, "value": M.n_cells / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "blasius_bl", "growth_rates": list(growths),
                       "stencils_k_r": [[k, r] for k, r, _ in stencils], "nu": 1e-3, "x_range": [0.5, 1.0],
                       "first_cell": 0.002, "y_max": 0.3, "value_from": "residual evaluations, %d cells, "
                       "Dirichlet walls, FP32 USR3 n_diff 2" % M.n_cells},
            "forms": forms, "gpu_vs_oracle_fp64_max_rel": worst, "seconds_total": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)


def run_reference(args):
    """The oracle as the reference arm, on the host cores: each step is one SSP-RK3
    stage of the full workload (the metric's unit of work) by the OpenMP build of the
    FP64 oracle on every core.  --ref-size N times the N^3 member of the family
    instead (a bounded sample) and says so."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import synth
    w = synth.workload(args.workload, order=args.order, size=args.ref_size or args.size, q=args.quad)
    O = oracle.Oracle(w["mesh"], parallel=True)
    nthr = oracle.threads(parallel=True)
    osch = oracle.Scheme(**w["scheme"])
    u = w["u0"]
    for _ in range(args.warmup):
        O.rk3_stage(u, u, osch, w["dt"], 0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.rk3_stage(u, u, osch, w["dt"], 0)
    t = time.perf_counter() - t0
    cells = int(w["u0"].shape[1])
    value = cells * args.steps / t
    full = not args.ref_size
    sample = ("one SSP-RK3 stage per step of the %s workload (%d cells%s), FP64 C oracle, OpenMP build on %d "
              "threads" % (args.workload, cells, "" if full else ", a bounded sample of the family", nthr))
    config = _config(args, w, cells, int(O.n_faces))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthr, "kind": "oracle", "sample": sample,
                         "host": _host_info()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dolinc", choices=["dolinc", "reference"])
    ap.add_argument("--workload", default="euler3d_tet64")
    ap.add_argument("--order", type=int, default=3)
    ap.add_argument("--size", type=int, default=None, help="lattice size (default: the workload's)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--shape", default=None, help="force diff_lanes,diff_block,stage_lanes,stage_block")
    ap.add_argument("--ind-runs", type=int, default=12)
    ap.add_argument("--ind-eval-runs", type=int, default=3)
    ap.add_argument("--ind-train-size", type=int, default=160)
    ap.add_argument("--ind-train-steps", type=int, default=60)
    ap.add_argument("--ind-epochs", type=int, default=30)
    ap.add_argument("--batch-meshes", type=int, default=512)
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp32_bf16"])
    ap.add_argument("--quad", type=int, default=2, help="quadrature points per direction for initial averages")
    ap.add_argument("--ref-size", type=int, default=None,
                    help="reference arm: time this lattice size instead of the full workload")
    ap.add_argument("--no-oracle", action="store_true")
    ap.add_argument("--hp-sizes", default="35,70,140", help="adv3d_hexprism convergence lattices")
    ap.add_argument("--hp-time", type=float, default=0.05, help="adv3d_hexprism convergence end time")
    ap.add_argument("--hp-quad", type=int, default=3, help="adv3d_hexprism quadrature points per direction")
    ap.add_argument("--stab-time", type=float, default=0.4, help="euler3d_tet64 stability runs: end time")
    ap.add_argument("--imp-dt-factor", type=float, default=16.0, help="semi-implicit dt / explicit dt")
    ap.add_argument("--imp-time", type=float, default=0.1, help="semi-implicit accuracy runs: end time")
    ap.add_argument("--imp-tol", type=float, default=1e-6, help="semi-implicit solver relative tolerance")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "euler2d_riemann":
        run_indicator(args)
    elif args.workload == "burgers_batch":
        run_batch(args)
    elif args.workload == "adv3d_hexprism":
        run_hexprism(args)
    elif args.workload == "adv3d_hexprism_implicit":
        run_implicit(args)
    elif args.workload == "blasius_bl":
        run_blasius(args)
    else:
        run_dolinc(args)


if __name__ == "__main__":
    main()
