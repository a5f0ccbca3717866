#!/usr/bin/env python
"""Benchmark of the HDG hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extras]

Workload (N=1): the largest single-GPU configuration, cube48_k2_conv -- unit cube, 48^3
subcubes x 6 Kuhn tetrahedra (663,552 elements, 1,340,928 faces, 8,045,568 trace unknowns),
interior vertices jittered by U(-0.2h, 0.2h)^3 (seed 0), k = 2, convection beta = (y, -x, 0.5 z),
kappa = 1 + 0.5 sin(2 pi z), c = 1, tau = 2.5, manufactured u = sin(pi x) sin(pi y) sin(pi z),
Dirichlet on every face.  Synthetic, seeded.

One step = the whole hot path on one batch of resident inputs:
  assemble + condense (K1, double-float on the FP32 pipe, LU of the non-symmetric Schur
  complement)  ->  trace solve to ||b - H u||/||b|| <= 1e-10 (FP32 inner BiCGStab with FP64
  residuals and refinement, two-level preconditioner)  ->  recover (K2)  ->  postprocess (K5).
value = elements/s over the metric's phases (assemble + condense + recover), timed with CUDA
events on the launching stream; the trace solve's time-to-1e-10 is reported beside it for the
plain FP64 block-Jacobi BiCGStab (zero start), the mixed-precision solve and the two-level
preconditioned solves.  The inputs (3.4 GB) are larger than L2; L2 is also flushed (256 MiB
write) before every step.
Extras (N=1, rank 0, unless --no-extras): the reaction-diffusion workload cube16_k3 (24,576
elements, k = 3) through the same step; the 64-problem mixed-degree batch; the random-field
workload cube32_k2_grf's solve times with and without a learned initial guess.
With --impl reference the FP64 CPU oracle is timed on the host cores on the same workload.
"""

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HEADLINE = "cube48_k2_conv"
EXTRA_RD = "cube16_k3"
# relative tolerance of each FP32 inner solve of the mixed-precision trace solve, per workload
# (measured: the fastest to 1e-10 on GB300 among 1e-2 .. 1e-6; --inner-rtol overrides)
INNER_RTOL = {"cube48_k2_conv": 1e-2, "cube16_k3": 1e-5}
METRIC = "elements/sec (assemble+condense+recover) & time-to-1e-10 solve vs plain FP64 GPU"
UNIT = "elements/s"
# FP64 peak of GB300: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz (max SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP64_MEASURED_TFLOPS = 1.19  # FMA-chain microbenchmark on this machine's GB300 (1 block/SM saturates)
# FP32 FMA pipe: 152 SMs x 128 lanes x 2 flop x 2.07 GHz; measured 74.8 TFLOP/s (FMA chain)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP32_MEASURED_TFLOPS = 74.8
# FP64-equivalent peak of double-float arithmetic on the FP32 pipe: 152 SMs x 128 FP32 lanes x
# 2.07 GHz / 12 FP32 instructions per compensated multiply-add (dacc_mac) x 2 flop
DF_PEAK_TFLOPS = 152 * 128 * 2.070e9 / 12 * 2 / 1e12
HBM_FALLBACK_GBS = 6800.0

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per element of one K1 launch, from
# the ncu captures summarised under profiles/ (captured on a smaller mesh of the same workload
# and scaled by the element count: K1 streams per-element data only, so traffic is proportional
# to it), valid while the kernel's sources (K1_SOURCES, hashed together) are unchanged.
E2E_CHUNKS = 16  # element ranges of the pipelined host-input assembly and host-output recovery

K1_TRAFFIC = {
    ("cube48_k2_conv", "assemble_df.cu"): {
        "sha256": "579987cdf75e34c3d582102c2c596cedd0e7c8fa3f286079bcb9aa3a5639976a",
        "bytes_per_element": (120072448 + 237189632) / 24576,
        "captured": "ncu dram__bytes_read/write of the same kernel on the 16^3 x 6 mesh of the workload (24,576 "
                    "elements), profiles/assemble_df_kernel_conv_k2_cube16.md"},
    ("cube16_k3", "assemble_df.cu"): {
        "sha256": "579987cdf75e34c3d582102c2c596cedd0e7c8fa3f286079bcb9aa3a5639976a",
        "bytes_per_element": (80775936 + 901166592) / 24576,
        "captured": "ncu dram__bytes_read/write of the same kernel on the workload's own mesh (24,576 elements), "
                    "profiles/assemble_df_kernel_cube16_k3.md"},
}
# the sources of each K1 translation unit (the kernel and the device headers it includes)
K1_SOURCES = {"assemble_df.cu": ("assemble_df.cu", "assemble_df.cuh", "device_df.cuh", "device_common.cuh"),
              "assemble_df_lean.cu": ("assemble_df_lean.cu", "assemble_df.cuh", "device_df.cuh", "device_common.cuh"),
              "assemble.cu": ("assemble.cu", "device_common.cuh")}


def _dims(k):
    n = (k + 1) * (k + 2) * (k + 3) // 6
    d2 = (k + 1) * (k + 2) // 2
    return n, d2, 4 * d2, (k + 2) ** 3, (k + 2) ** 2


def flops_per_element_k1(k, conv=False):
    """FP64 flops per element of the K1 algorithm (structured elimination), FMA = 2."""
    n, d2, m, nq, nf = _dims(k)
    NP, MP = n * (n + 1) // 2, m * (m + 1) // 2
    chol = sum(2 * j + 3 + (n - j - 1) * (2 * j + 1) for j in range(n))
    lu = sum(1 + (n - j - 1) + 2 * (n - j - 1) ** 2 for j in range(n))
    nn, np1, np2 = k + 2, (k + 1) * (k + 2) // 2, d2 * (d2 + 1) // 2
    f = 4 * nq                      # |K| w / kappa, |K| w c, |K| w f
    # M_{kappa^-1}, M_c and f^K by sum factorisation (1-D, 2-D, 3-D pair passes), tauPP
    f += 2 * ((2 * np1 + k + 1) * nn ** 3 + (2 * np2 + d2) * nn * nn + (2 * NP + n) * nn)
    f += NP * 8
    f += 18 * n * n                 # C_*^T from C_hat and the cofactors
    f += chol                       # L L^T = M
    f += (3 * n + m) * n * n        # W_* = L^-1 C_*^T, V = L^-1 E^T
    f += NP * (6 * n + 1)           # S_u += sum W^T W
    f += 20 * n * n                 # sum_* n_{l*} W_*
    f += n * m * (2 * n + 1)        # G
    if not conv:
        f += MP * (2 * n + 7)       # (n.n) V^T V + tauDD
        f += chol                   # L_s L_s^T = S_u
        f += (m + 1) * n * n        # H|h = L_s^-1 [G^T|f]
        f += MP * (2 * n + 1) + 2 * m * n  # C -= H^T H, C_f
        return f
    # convection: weights, Gq, B_c, alphaDP, alphaDD, LU, two sets of forward substitutions,
    # and the full (non-symmetric) C
    f += 3 * nq * 8 + 4 * nf * 7    # bw, varpi beta.n
    f += 6 * nq * n                 # Gq
    f += 2 * n * (n + 1) * nq       # B_c (both triangles)
    f += 3 * n * m * nf + 3 * 4 * d2 * d2 * nf  # alphaDP, alphaDD
    f += lu                         # L U = S_u
    f += (m + 1) * n * (n - 1) + m * n * (n + 1)  # [H_col|h] = L^-1 [.], H_row = U^-T G^T
    f += m * m * (4 * n + 4) + 2 * m * n  # C = (n.n) V^T V + tauDD - alphaDD - H_row^T H_col, C_f
    return f


def k1_bytes_per_element(k, conv=False):
    """Algorithmic HBM bytes of K1 per element: kappa, c, f (and beta at the volume and face
    nodes), geometry, perms, tau in; C^K (full), C_f^K and the recovery record out."""
    n, d2, m, nq, nf = _dims(k)
    rec = n * (m + 1) + n * m + 3 * n * n + n * (n + 1) + 12  # [H|h], V, W_*, U_s, U_M, normals
    inp = 8 * (3 * nq + 28) + 4 * 4 + 8 * 4
    if conv:
        inp += 8 * (3 * nq + 3 * 4 * nf)
    return inp + 8 * (m * m + m + rec)


def krylov_bytes_per_iteration(nelt, nfc, k, conv, fp32=True):
    """Algorithmic HBM bytes of one inner Krylov iteration (block-Jacobi part; the coarse
    cycles are not counted, so the fraction below is conservative): every C^K row read once
    per operator application (2 per BiCGStab iteration, 1 per CG iteration), the block
    inverses once per preconditioner application, and the vector passes of the method
    (BiCGStab: 25 vectors read or written per iteration; CG: 12)."""
    n, d2, m, nq, nf = _dims(k)
    w = 4 if fp32 else 8
    nv = nfc * d2
    apps = 2 if conv else 1
    vec = 25 if conv else 12
    return apps * (nelt * m * m * w + nfc * d2 * d2 * w) + vec * nv * w


def _sha(*paths):
    h = hashlib.sha256()
    for path in paths:
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling (every 100 ms, started before the warm-up so that it is running when
    the timed region starts); only the samples stamped inside the timed region are kept."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, t_begin=None, t_end=None):
        """Summary of the samples stamped within [t_begin, t_end] (epoch seconds, 0.1 s slack);
        all samples if none falls inside."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        return self.summarise(out, t_begin, t_end)

    @staticmethod
    def summarise(out, t_begin=None, t_end=None):
        import datetime

        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 10:
                continue
            try:
                sm, mx = float(p[2]), float(p[3])
            except ValueError:
                continue
            try:  # nvidia-smi stamps local time, e.g. 2026/12/04 04:05:15.159
                ts = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            rows.append((ts, sm, mx, {nm for nm, v in zip(names, p[6:10]) if v.lower() == "active"}))
        inside = rows
        window = "all samples"
        if t_begin is not None and t_end is not None:
            sel = [r for r in rows if r[0] is not None and t_begin - 0.1 <= r[0] <= t_end + 0.1]
            if sel:
                inside, window = sel, "timed region"
            else:
                window = "all samples (none stamped inside the timed region)"
        reasons = set().union(*(r[3] for r in inside)) if inside else set()
        return {"sm_mhz": float(np.median([r[1] for r in inside])) if inside else None,
                "sm_max_mhz": max(r[2] for r in inside) if inside else None,
                "samples": len(inside), "window": window, "reasons": sorted(reasons)}


# ------------------------------------------------------------------ oracle timing (CPU)
_ORACLE = {}


def _sub_mesh(coords, elems_sub):
    """The expanded mesh of a set of elements on their own, in the global vertex numbering (so
    each element's geometry, face orientation and perm are those of the full mesh), with the
    faces that the set does not share listed as boundary faces."""
    from oracle.geometry import LOCAL_FACES, ExpandedMesh

    tri = np.sort(elems_sub[:, LOCAL_FACES].reshape(-1, 3), axis=1)
    faces, counts = np.unique(tri, axis=0, return_counts=True)
    return ExpandedMesh(coords, elems_sub, faces[counts == 1], np.zeros((0, 3), np.int64))


def _oracle_init(name, samples):
    """Worker set-up (outside the timed region): for every step, this worker's share of the
    sampled elements as a mesh of their own, with its coefficients at the oracle's nodes."""
    from oracle import convection as cv
    from oracle import hdg as ohdg
    from workloads import get_problem, kuhn_cube

    prob = get_problem(name)
    c, e = kuhn_cube(prob.s, prob.jitter, prob.seed)
    tab = ohdg.Tables(prob.k)
    work = []
    for idx in samples:
        mesh = _sub_mesh(c, np.asarray(e)[np.sort(idx)])
        X, Y, Z = ohdg.volume_nodes(mesh, tab)
        w = dict(mesh=mesh, kap=prob.kappa(X, Y, Z), c=prob.c(X, Y, Z), f=prob.f(X, Y, Z),
                 uhat=np.zeros((mesh.nfc, tab.d2)))
        if prob.beta is not None:
            FX, FY, FZ = cv.element_face_nodes(mesh, tab)
            w.update(bq=prob.beta(X, Y, Z), bf=prob.beta(FX, FY, FZ))
        work.append(w)
    _ORACLE.update(prob=prob, tab=tab, work=work)


def _oracle_chunk(step):
    """Oracle assemble + condense + recover of this worker's elements of one step."""
    from oracle import convection as cv
    from oracle import hdg as ohdg
    o = _ORACLE
    w = o["work"][step]
    blk = ohdg.local_blocks(w["mesh"], o["tab"], w["kap"], w["c"], w["f"], tau=o["prob"].tau)
    if "bq" in w:
        Bc, aDP, aDD = cv.convection_blocks(w["mesh"], o["tab"], w["bq"], w["bf"])
        CK, Cf, X2, xf, _ = cv.local_solvers_conv(blk, Bc, aDP, aDD)
    else:
        CK, Cf, X2, xf = ohdg.local_solvers(blk)
    ohdg.recover(w["mesh"], X2, xf, w["uhat"])
    return w["mesh"].nelt


def oracle_baseline(name, sample_elems, steps=1, warmup=0):
    """Time the oracle as it stands on the host cores: elements/s (assemble+condense+recover)
    on `steps` random samples of `sample_elems` elements of the workload's mesh."""
    import multiprocessing as mp

    from workloads import get_problem

    prob = get_problem(name)
    nelt = 6 * prob.s ** 3
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(0)
    nst = steps + warmup
    picks = [np.sort(rng.choice(nelt, size=sample_elems, replace=False)) for _ in range(nst)]
    per_worker = [[np.array_split(p, cores)[wk] for p in picks] for wk in range(cores)]
    ctx = mp.get_context("spawn")
    env_backup = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_backup:
        os.environ[k] = "1"
    try:
        pools = []
        # one single-process pool per worker, so each worker holds exactly its own share
        for wk in range(cores):
            pools.append(ctx.Pool(1, initializer=_oracle_init, initargs=(name, per_worker[wk])))
        for p in pools:  # wait for every worker's set-up
            p.apply(len, ([],))

        def one(step):
            t0 = time.perf_counter()
            res = [p.apply_async(_oracle_chunk, (step,)) for p in pools]
            done = sum(r.get() for r in res)
            return done, time.perf_counter() - t0
        for s in range(warmup):
            one(s)
        tot_e, tot_t = 0, 0.0
        for s in range(warmup, nst):
            ne, dt = one(s)
            tot_e += ne
            tot_t += dt
    finally:
        for p in pools:
            p.close()
            p.join()
        for k, v in env_backup.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    kind = ("numpy FP64 literal blocks + convection blocks (eq. 9.1) + LU of A_1 + recovery" if prob.beta is not None
            else "numpy FP64 literal blocks + LU of A_1 + recovery")
    return {"value": tot_e / tot_t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{sample_elems} random elements of the {nelt}-element {name} mesh per step x {steps} step(s) "
                      f"(each step's elements as a mesh of their own, set up outside the timed region); {kind}, "
                      f"{cores} spawn workers with 1 BLAS thread each"}


# ------------------------------------------------------------------ multi-rank helpers
def max_over_ranks(vals, world, device):
    """Element-wise maximum of per-rank timings (every rank gets the result)."""
    if world <= 1:
        return list(vals)
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(vals), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_value(nelt, steps, world, phase_ms):
    """Whole-job throughput: every rank processes its own copy of the workload (replicas), so
    the elements of all ranks over the slowest rank's time."""
    return world * nelt * steps / (phase_ms / 1e3)


# ------------------------------------------------------------------ GPU arm
class Workload:
    """A workload's mesh on the GPU and its PDE data at the library's nodes (host copies kept
    for the end-to-end leg)."""

    def __init__(self, name, dev, stream, s=None, rule=0):
        import torch

        from paper_1305_1489_gb300 import HDGMesh
        from workloads import boundary_faces, get_problem, kuhn_cube

        self.name = name
        self.prob = prob = get_problem(name) if s is None else get_problem(name).at(s=s)
        c, e = kuhn_cube(prob.s, prob.jitter, prob.seed)
        d, n = boundary_faces(c, e, prob.classify)
        self.M = M = HDGMesh(c, e, d, n, prob.k, stream=stream)
        if rule:
            M.set_volume_rule(rule)
        self.conv = prob.beta is not None
        X, Y, Z = (t.cpu().numpy() for t in M.volume_nodes())
        FX, FY, FZ = (t.cpu().numpy() for t in M.face_nodes())
        self.X, self.Y, self.Z, self.FX, self.FY, self.FZ = X, Y, Z, FX, FY, FZ
        host = {"kappa": prob.kappa(X, Y, Z), "c": prob.c(X, Y, Z), "f": prob.f(X, Y, Z),
                "uD": prob.uD(FX, FY, FZ)}
        if prob.gN is not None:
            host["gN"] = np.stack(prob.gN(FX, FY, FZ))
        if self.conv:
            EX, EY, EZ = (t.cpu().numpy() for t in M.element_face_nodes())
            host["beta"] = np.stack(prob.beta(X, Y, Z))
            host["beta_f"] = np.stack(prob.beta(EX, EY, EZ))
            host["tau"] = np.full((M.nelt, 4), prob.tau)
        self.host = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in host.items()}
        self.dv = {k: torch.from_numpy(v).to(dev) for k, v in self.host.items()}
        self.set_inputs()

    def set_inputs(self):
        dv = self.dv
        if self.conv:
            self.M.set_coefficients(dv["kappa"], dv["c"], dv["f"], dv["tau"], beta=dv["beta"], beta_faces=dv["beta_f"])
        else:
            self.M.set_coefficients(dv["kappa"], dv["c"], dv["f"])
        self.M.set_boundary_data(dv["uD"], dv.get("gN"))

    def hierarchy(self):
        """The nested P1 levels of the two-level preconditioner, coarsened down to at most 64
        nodes (to a single node on meshes too small for that)."""
        from workloads import kuhn_p1_hierarchy
        h = kuhn_p1_hierarchy(self.prob.s, self.prob.dirichlet_planes, strict=False)
        if len(h[0]) < 2:
            h = kuhn_p1_hierarchy(self.prob.s, self.prob.dirichlet_planes, max_coarsest=1, strict=False)
        return h


def run_workload(W, args, stream, dev, world=1, full=True):
    """The step of workload W timed over args.steps (after args.warmup), and, with full, the
    time-to-1e-10 comparison, the diagnostics, the end-to-end leg and the rooflines."""
    import torch

    from paper_1305_1489_gb300 import HDG_DF32, HDG_FP64, HDG_MIXED_FP32

    M, prob = W.M, W.prob
    nelt = M.nelt
    inner_rtol = args.inner_rtol if args.inner_rtol is not None else INNER_RTOL.get(W.name, 1e-4)
    M.set_inner_tolerance(inner_rtol)
    asm_prec = HDG_DF32 if args.asm == "df32" else HDG_FP64
    hierarchy = W.hierarchy()
    step_prec = HDG_MIXED_FP32 if args.solve == "mixed" else HDG_FP64
    if args.coarse:
        M.set_coarse_space(*hierarchy)
    M.assemble_condense(asm_prec)
    tuned = M.autotune() if args.autotune else None
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def step(rec=None):
        flush.fill_(1.0)
        e0, e1, e2, e3, e4 = ev(), ev(), ev(), ev(), ev()
        e0.record(stream)
        M.assemble_condense(asm_prec)
        e1.record(stream)
        uhat, it, rr = M.solve_trace(rtol=1e-10, maxit=20000, precision=step_prec)
        e2.record(stream)
        q, u = M.recover(uhat)
        e3.record(stream)
        M.postprocess(q, u)
        e4.record(stream)
        if rec is not None:
            rec.append((e0, e1, e2, e3, e4, it, rr))

    clk = ClockSampler(dev.index if dev.index is not None else 0)
    if full:
        clk.start()
        time.sleep(0.5)  # nvidia-smi is up and sampling before the timed region
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    recs = []
    launches0 = M.launches
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tw0 = time.time()
    tstart = ev()
    tstart.record(stream)
    for _ in range(args.steps):
        step(recs)
    tend = ev()
    tend.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t0
    clocks = clk.stop(tw0, time.time()) if full else None
    launches = M.launches - launches0
    total_ms = tstart.elapsed_time(tend)
    t_asm = [a.elapsed_time(b) for a, b, *_ in recs]
    t_sol = [b.elapsed_time(c_) for _, b, c_, *_ in recs]
    t_rec = [c_.elapsed_time(d_) for _, _, c_, d_, *_ in recs]
    t_pp = [d_.elapsed_time(e_) for _, _, _, d_, e_, *_ in recs]
    its = [r[5] for r in recs]
    phase_ms = sum(t_asm) + sum(t_rec)
    phase_ms, total_ms = max_over_ranks([phase_ms, total_ms], world, dev)
    value = job_value(nelt, args.steps, world, phase_ms)
    phases = {"assemble_condense": float(np.mean(t_asm)), "trace_solve": float(np.mean(t_sol)),
              "recover": float(np.mean(t_rec)), "postprocess": float(np.mean(t_pp))}
    peaks = _measured_peaks()
    hbm = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    hbm_note = "of measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "of fallback"
    # roofline of the step's solve: algorithmic bytes of the inner Krylov iterations over their time
    inner_fp32 = step_prec == HDG_MIXED_FP32
    kb = krylov_bytes_per_iteration(nelt, M.nfc, prob.k, W.conv, fp32=inner_fp32)
    it_mean = float(np.mean(its))
    sol_ach = kb / (phases["trace_solve"] / 1e3 / max(it_mean, 1.0)) / 1e9
    solve_roofline = {"bound": "hbm", "achieved": sol_ach, "peak": hbm, "unit": "GB/s", "frac": sol_ach / hbm,
                      "peak_note": hbm_note, "iterations": it_mean,
                      "ms_per_iteration": phases["trace_solve"] / max(it_mean, 1.0),
                      "bytes_per_iteration": kb,
                      "work": ("per inner iteration: " + ("2" if W.conv else "1") + " reads of the "
                               + ("FP32" if inner_fp32 else "FP64") + " C^K and the block inverses, "
                               + ("25" if W.conv else "12") + " vector passes; the coarse cycles, the FP64 "
                               "refinement and the set-up (Galerkin hierarchy, block inverses) are inside the "
                               "time but not in the bytes, so the fraction is a lower bound")}
    out = {"value": value, "nelt": nelt, "nfc": M.nfc, "trace_dofs": M.nfc * M.d2, "k": prob.k,
           "inner_rtol": inner_rtol,
           "phases_ms": phases, "iterations_per_step": it_mean, "gpu_launches": int(launches),
           "ms_per_step": total_ms / args.steps, "wall_s_timed": wall, "clocks": clocks, "autotune": tuned,
           "solve_roofline": solve_roofline, "coarse_levels": [int(x) for x in hierarchy[0]] if args.coarse else None}
    if not full:
        return out

    # time-to-1e-10 (zero start): plain FP64 block-Jacobi, mixed precision, and both with the
    # two-level preconditioner (its Galerkin set-up after the assembly is inside the time)
    solve = {}
    cases = (("plain_fp64", HDG_FP64, False), ("mixed_fp32_fp64", HDG_MIXED_FP32, False),
             ("two_level_fp64", HDG_FP64, True), ("two_level_mixed", HDG_MIXED_FP32, True))
    for name, prec, tl in cases:
        if tl:
            M.set_coarse_space(*hierarchy)
        else:
            M.set_coarse_space(None, None, None)
        ts, its_ = [], []
        for _ in range(args.solve_reps):
            M.assemble_condense(asm_prec)
            torch.cuda.synchronize()
            a, b = ev(), ev()
            a.record(stream)
            uh, it, rr = M.solve_trace(rtol=1e-10, maxit=40000, precision=prec, raise_on_fail=False)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
            its_.append(it)
        solve[name] = {"ms": float(np.median(ts)), "iterations": its_[-1], "relres": rr, "converged": bool(rr <= 1e-10)}
    for name in ("mixed_fp32_fp64", "two_level_fp64", "two_level_mixed"):
        solve["speedup_" + name + "_vs_plain"] = solve["plain_fp64"]["ms"] / solve[name]["ms"]
    solve["method"] = "BiCGStab (non-symmetric trace matrix)" if W.conv else "CG"
    if args.coarse:
        M.set_coarse_space(*hierarchy)
    else:
        M.set_coarse_space(None, None, None)
    out["solve_time_to_1e-10"] = solve

    # discretisation errors (eq. 10.1-10.2) of the step's solution and the HDG projection
    # diagnostics (Section 9, eq. 10.2), timed with CUDA events (outside the metric)
    M.assemble_condense(asm_prec)
    uh, it, rr = M.solve_trace(rtol=1e-10, maxit=20000, precision=step_prec)
    q, u = M.recover(uh)
    X, Y, Z, FX, FY, FZ = W.X, W.Y, W.Z, W.FX, W.FY, W.FZ
    XF, YF, ZF = (t.cpu().numpy() for t in M.element_face_nodes())
    q_vol = torch.from_numpy(np.ascontiguousarray(np.stack(prob.q(X, Y, Z)))).to(dev)
    q_face = torch.from_numpy(np.ascontiguousarray(np.stack(prob.q(XF, YF, ZF)))).to(dev)
    u_vol = torch.from_numpy(np.ascontiguousarray(prob.u(X, Y, Z))).to(dev)
    u_face = torch.from_numpy(np.ascontiguousarray(prob.u(XF, YF, ZF))).to(dev)
    u_fn = torch.from_numpy(np.ascontiguousarray(prob.u(FX, FY, FZ))).to(dev)
    tp = []
    for _ in range(3):
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        Pq, Pu = M.projection(q_vol, u_vol, q_face, u_face)
        b.record(stream)
        torch.cuda.synchronize()
        tp.append(a.elapsed_time(b))
    Pf = M.face_projection(u_fn)
    e_pu, ref_u = M.volume_norm2(Pu - u, None)[0], M.volume_norm2(None, u_vol)[1]
    e_pf, ref_f = M.face_norm2(Pf - uh, None)[0], M.face_norm2(None, u_fn)[1]
    e_u = M.volume_norm2(u, u_vol)[0]
    e_uhat = M.face_norm2(uh, u_fn)[0]
    out["superconvergence"] = {
        "hdg_projection_ms": float(np.median(tp[1:])),
        "eps_u": float(np.sqrt(e_pu / ref_u)), "eps_uhat": float(np.sqrt(e_pf / ref_f)),
        "e_u": float(np.sqrt(e_u / ref_u)), "e_uhat": float(np.sqrt(e_uhat / ref_f)),
        "note": "eq. 10.1-10.2 ratios of the step's solution (trace solve to 1e-10); the HDG projection "
                "(eq. 9.13) time is per launch over all elements"}
    del q_vol, q_face, u_vol, u_face, Pq, Pu

    # the dense mass contraction (eq. 3.55, M_{kappa^-1}) as one GEMM on the tensor cores
    # (BF16 operands, FP32 accumulation) against the CUDA-core FP32 contraction
    out["h2_contraction"] = h2_contraction(W, dev, stream)
    # the HDG_MIXED_BF16 assembly (split-BF16 tensor-core masses, double-float condensation)
    # beside the step's double-float one: time per assembly and the solution's deviation
    if args.asm == "df32" and prob.k >= 1:
        out["mixed_bf16_assembly"] = mixed_bf16_assembly(W, dev, stream, uh, u, step_prec, phases["assemble_condense"])
        M.assemble_condense(asm_prec)

    # end to end through the public API with host buffers (pinned) and copies in the region
    out["e2e"] = e2e_leg(W, args, stream, world, asm_prec, step_prec, flush)

    # roofline of the dominant kernel of the metric (K1).  Its work is the FP64 flop count of
    # the algorithm.  The double-float K1 executes it on the FP32 pipe as compensated
    # multiply-adds (12 FP32 instructions each), so its peak is the FP32 pipe's rate / 12; the
    # FP64 K1 is held to the FP64 pipe.
    k1_ms = phases["assemble_condense"]
    fpe = flops_per_element_k1(prob.k, W.conv)
    achieved = fpe * nelt / (k1_ms / 1e3) / 1e12
    streamed = bool(tuned and tuned.get("k1_streamed"))  # the kernel that streams W_* (k = 4)
    k1_src = ("assemble_df_lean.cu" if streamed else "assemble_df.cu") if args.asm == "df32" else "assemble.cu"
    sha = _sha(*(os.path.join(ROOT, "paper_1305_1489_gb300", "csrc", f) for f in K1_SOURCES[k1_src]))
    trec = K1_TRAFFIC.get((W.name, k1_src), {})
    bpe = trec.get("bytes_per_element") if trec.get("sha256") == sha else None
    df = args.asm == "df32"
    peak = DF_PEAK_TFLOPS if df else FP64_PEAK_TFLOPS
    out["roofline"] = {
        "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
        "traffic": bpe * nelt if bpe else None,
        "traffic_note": (f"ncu dram bytes per element x {nelt} elements ({trec.get('captured')})" if bpe else
                         "no ncu capture of the current K1 sources"),
        "kernel": ((f"assemble_df_lean_kernel<{prob.k}, ..> (K1 with W_* streamed, double-float on the FP32 pipe)"
                    if streamed else
                    f"assemble_df_kernel<{prob.k}, .., CONV={str(W.conv).lower()}> (K1, double-float on the FP32 pipe)")
                   if df else f"assemble_kernel<{prob.k}> (K1, FP64)"),
        "work": "FP64-equivalent flops of the structured elimination (sum-factorised masses)",
        "flops_per_element": fpe, "algorithmic_bytes_per_launch": k1_bytes_per_element(prob.k, W.conv) * nelt,
        "peak_note": ("double-float on the FP32 pipe: 152 SMs x 128 lanes x 2.07 GHz / 12 FP32 instructions per "
                      "compensated multiply-add x 2 flop (derived from unit counts and the maximum clock)" if df else
                      "FP64 pipe: 152 SMs x 2 DFMA/clk x 2.07 GHz (derived from unit counts and the maximum clock); "
                      f"measured FMA microbenchmark {FP64_MEASURED_TFLOPS} TFLOP/s"),
        "frac_of_fp64_pipe": achieved / FP64_PEAK_TFLOPS,
        "fp32_pipe_note": (f"the FP32 FMA pipe's own peak is {FP32_PEAK_TFLOPS:.1f} TFLOP/s derived "
                           f"({FP32_MEASURED_TFLOPS} measured); ncu's FMA-pipe utilisation of this kernel is in "
                           "profiles/")}
    return out


def h2_contraction(W, dev, stream, reps=5):
    """hdg_mass_contraction of 1/kappa on the workload's mesh: tensor cores (mode 0) and CUDA
    cores in FP32 (mode 2), times per launch, throughput and the BF16 result's normwise error
    against the FP32 one."""
    import torch

    M = W.M
    g = torch.from_numpy(np.ascontiguousarray(1.0 / W.host["kappa"])).to(dev)
    n, nq = M.n, M.nq
    npair = n * (n + 1) // 2
    res = {}
    outs = {}
    for name, mode in (("tensor_core_bf16", 0), ("cuda_core_fp32", 2)):
        outs[name] = M.mass_contraction(g, mode)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            M.mass_contraction(g, mode)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = float(np.median(ts))
        flops = 2.0 * M.nelt * nq * npair
        byts = M.nelt * (8 * nq + 4 * npair + 8)
        res[name] = {"ms": ms, "tflops": flops / (ms / 1e3) / 1e12, "gbs": byts / (ms / 1e3) / 1e9}
    a, b = outs["tensor_core_bf16"], outs["cuda_core_fp32"]
    res["bf16_normwise_error_vs_fp32"] = float((a - b).abs().max() / b.abs().max())
    res["note"] = (f"[{M.nelt} x {nq}] . [{nq} x {npair}] per launch; bytes = the FP64 coefficient in, the FP32 "
                   "masses out; HBM-bound at this contraction length")
    return res


def e2e_leg(W, args, stream, world, asm_prec, step_prec, flush):
    """The metric through hdg_assemble_condense_host / hdg_recover_host from pinned host
    buffers: the library copies the inputs chunk by chunk beside the condensation, and the
    recovered fields beside the recovery; the trace solve runs between them, untimed."""
    import torch

    M, nelt = W.M, W.M.nelt
    pin = {k: torch.from_numpy(v).pin_memory() for k, v in W.host.items()}
    hq = torch.empty((nelt, 3, M.n), dtype=torch.float64).pin_memory()
    hu = torch.empty((nelt, M.n), dtype=torch.float64).pin_memory()
    h2d = sum(v.numel() * 8 for v in pin.values())
    d2h = (hq.numel() + hu.numel()) * 8
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    e2e_ms, t_asm, t_rec = 0.0, [], []
    for i in range(args.warmup + args.steps):
        flush.fill_(1.0)
        a, b, cc, dd = ev(), ev(), ev(), ev()
        a.record(stream)
        M.assemble_condense_host(pin, asm_prec, chunks=args.e2e_chunks)
        b.record(stream)
        uh, it, rr = M.solve_trace(rtol=1e-10, maxit=20000, precision=step_prec)
        cc.record(stream)
        M.recover_host(uh, hq, hu, chunks=args.e2e_chunks)
        dd.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            t_asm.append(a.elapsed_time(b))
            t_rec.append(cc.elapsed_time(dd))
            e2e_ms += t_asm[-1] + t_rec[-1]
    return {"value": world * nelt * args.steps / (e2e_ms / 1e3), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "assemble_host_ms": float(np.mean(t_asm)), "recover_host_ms": float(np.mean(t_rec)),
            "assemble_host_ms_median": float(np.median(t_asm)), "assemble_host_ms_max": float(np.max(t_asm)),
            "phases": "hdg_assemble_condense_host (H2D of " + ",".join(W.host) + " from pinned host memory "
                      f"in {args.e2e_chunks} chunks beside the condensation) + hdg_recover_host (recovery with "
                      "the D2H of q, u beside it); the trace solve runs between them and is excluded, as in "
                      "value"}


def mixed_bf16_assembly(W, dev, stream, uh_ref, u_ref, step_prec, df32_ms, reps=5):
    """hdg_assemble_condense(HDG_MIXED_BF16) on the workload: time per assembly (the tensor-core
    contraction of the masses and the condensation from them), the contraction alone, and the
    relative difference of the step's solution (trace and u, solved to 1e-10 the same way)
    from the double-float assembly's."""
    import torch

    from paper_1305_1489_gb300 import HDG_MIXED_BF16

    M = W.M

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    masses = [None]

    def contraction():
        masses[0] = M.mixed_masses()

    ms_tc = timed(contraction)
    stride = masses[0].shape[1]
    masses[0] = None
    ms_asm = timed(lambda: M.assemble_condense(HDG_MIXED_BF16))
    uh, it, rr = M.solve_trace(rtol=1e-10, maxit=20000, precision=step_prec)
    q, u = M.recover(uh)
    n, nq = M.n, M.nq
    npair = n * (n + 1) // 2
    return {"ms": ms_asm, "df32_ms": df32_ms, "speedup_vs_df32": df32_ms / ms_asm,
            "tc_contraction_ms": ms_tc,
            "tc_contraction_gbs": M.nelt * (3 * 8 * nq + 4 * stride) / (ms_tc / 1e3) / 1e9,
            "tc_contraction_tflops": 2.0 * 6 * M.nelt * nq * (2 * npair + n) / (ms_tc / 1e3) / 1e12,
            "solve_iterations": it, "relres": rr,
            "uhat_rel_diff_vs_df32": float((uh - uh_ref).abs().max() / uh_ref.abs().max()),
            "u_rel_diff_vs_df32": float((u - u_ref).abs().max() / u_ref.abs().max()),
            "note": "masses M_{kappa^-1}, M_c and f^K from three-way BF16 splits (six tcgen05 products, FP32 "
                    "accumulation), then the double-float condensation; tflops counts the six split products"}


def run_rule_comparison(dev, stream, reps=5):
    """The FP64 assembly (direct quadrature sums) of the reaction-diffusion workload on the
    conical rule ((k+2)^3 = 125 nodes at k = 3) and on the smaller symmetric rule (70 nodes):
    time per launch, and the discretisation errors of the step's solution on each rule."""
    import torch

    from paper_1305_1489_gb300 import HDG_FP64, HDG_MIXED_FP32, HDG_RULE_CONICAL, HDG_RULE_SYMMETRIC

    out = {"workload": f"{EXTRA_RD} (24,576 elements, k = 3), FP64 assembly"}
    for name, rule in (("conical", HDG_RULE_CONICAL), ("symmetric", HDG_RULE_SYMMETRIC)):
        W = Workload(EXTRA_RD, dev, stream, rule=rule)
        M = W.M
        M.assemble_condense(HDG_FP64)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            M.assemble_condense(HDG_FP64)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        M.set_inner_tolerance(1e-5)
        uh, it, rr = M.solve_trace(rtol=1e-12, maxit=20000, precision=HDG_MIXED_FP32)
        q, u = M.recover(uh)
        prob = W.prob
        u_vol = torch.from_numpy(np.ascontiguousarray(prob.u(W.X, W.Y, W.Z))).to(dev)
        u_fn = torch.from_numpy(np.ascontiguousarray(prob.u(W.FX, W.FY, W.FZ))).to(dev)
        e_u, ref_u = M.volume_norm2(u, u_vol)
        e_f, ref_f = M.face_norm2(uh, u_fn)
        out[name] = {"nq": M.nq, "k1_fp64_ms": float(np.median(ts)),
                     "coefficient_bytes_per_element": 3 * 8 * M.nq,
                     "e_u": float(np.sqrt(e_u / ref_u)), "e_uhat": float(np.sqrt(e_f / ref_f))}
        M.close()
        del W
        torch.cuda.empty_cache()
    out["speedup"] = out["conical"]["k1_fp64_ms"] / out["symmetric"]["k1_fp64_ms"]
    return out


def run_batch(args):
    """64 independent cube problems (s ~ U{8..24}, k ~ U{1..4}, kappa = 10^U(-1,1), c ~ U[0,5],
    Dirichlet everywhere, seed 4) solved as one batch: one CUDA graph launch (double-float
    assembly, PCG to 1e-10 for every problem, recovery): FP64 block-Jacobi, FP64 two-level,
    and two-level with FP32 inner / FP64 outer refinement.  Returns elements/s of each."""
    import torch

    from paper_1305_1489_gb300 import HDG_DF32, HDG_MIXED_FP32, HDGBatch, build
    from workloads import boundary_faces, kuhn_cube, kuhn_p1_hierarchy
    from workloads.problems import batch_problems

    build()
    probs = batch_problems(args.batch_n)
    meshes = []
    for p in probs:
        c, e = kuhn_cube(p.s)
        d, n = boundary_faces(c, e, p.classify)
        meshes.append((c, e, d, n, p.k))
    B = HDGBatch(meshes)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()  # noqa: E731
    nelt = 0
    for G in B.groups:
        M = G["mesh"]
        nelt += M.nelt
        X, Y, Z = (t.cpu().numpy() for t in M.volume_nodes())
        FX, FY, FZ = (t.cpu().numpy() for t in M.face_nodes())
        kap, cq, fq = (np.zeros_like(X) for _ in range(3))
        uD = np.zeros_like(FX)
        for i, p in enumerate(G["probs"]):
            pr = probs[p]
            es = slice(G["elem_off"][i], G["elem_off"][i + 1])
            fs = slice(G["face_off"][i], G["face_off"][i + 1])
            kap[es], cq[es], fq[es] = pr.kappa(X[es], Y[es], Z[es]), pr.c(X[es], Y[es], Z[es]), pr.f(X[es], Y[es], Z[es])
            uD[fs] = pr.uD(FX[fs], FY[fs], FZ[fs])
        M.set_coefficients(dev(kap), dev(cq), dev(fq))
        M.set_boundary_data(dev(uD))

    def timed():
        relres, iters = B.run(precision=HDG_DF32, rtol=1e-10, maxit=40000)  # warm-up + graph build
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.batch_reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(B.stream)
            relres, iters = B.run(precision=HDG_DF32, rtol=1e-10, maxit=40000)
            b.record(B.stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = float(np.median(ts))
        return {"groups": [{"k": G["k"], "problems": int(len(G["probs"])), "elements": int(G["mesh"].nelt),
                            "iterations": int(it)} for G, it in zip(B.groups, iters)],
                "ms_per_batch": ms, "elements_per_s": nelt / (ms / 1e3), "max_relres": float(relres.max())}

    tuned = B.autotune(HDG_DF32)
    out = {"workload": "64 cube problems, s ~ U{8..24}, k ~ U{1..4}, kappa = 10^U(-1,1), c ~ U[0,5], seed 4",
           "problems": len(probs), "elements": int(nelt), "graph_launches_per_batch": 1,
           "autotune": tuned, "block_jacobi": timed()}
    B.set_coarse_spaces([kuhn_p1_hierarchy(p.s, p.dirichlet_planes, max_coarsest=1, strict=False) for p in probs])
    out["two_level"] = timed()
    B.set_inner_tolerance(args.inner_rtol if args.inner_rtol is not None else 1e-5)
    B.set_solve_precision(HDG_MIXED_FP32)
    out["two_level_mixed"] = timed()
    for key in ("two_level", "two_level_mixed"):
        out["speedup_" + key] = out["block_jacobi"]["ms_per_batch"] / out[key]["ms_per_batch"]
    B.close()
    return out


def run_learned(args, train=None, evaluate=None, bj_eval=None, epochs=None):
    """The learned initial guess on the random-field workload: 32^3 x 6 Kuhn cube (196,608
    elements), k = 2, kappa = exp(g) with g a Gaussian random field (sigma 1, correlation
    length 0.2, 128 Fourier modes), c = f = 1, u = 0 on the whole boundary.  The network
    (g at the 3,375 interior nodes of the 16^3 grid -> tanh layer -> the coarse P1 field on that
    grid) is trained with the library's kernels on the coarse Galerkin projections of the
    trace solutions of `train` fields and evaluated on `evaluate` held-out fields: energy
    error of the initial guess, and PCG iterations and time to 1e-10 from the zero start and
    from the learned guess (guess time included), for block-Jacobi and two-level PCG in FP64
    and mixed precision."""
    import torch

    from paper_1305_1489_gb300 import HDG_FP64, HDG_MIXED_FP32, HDGMesh, build
    from paper_1305_1489_gb300.learned import CoarseSpace, LearnedGuess
    from workloads import boundary_faces, kuhn_coarse_interpolation, kuhn_cube, kuhn_grid_points, kuhn_p1_hierarchy
    from workloads.problems import cube32_k2_grf, grf_frequencies, grf_sample

    train = args.learned_train if train is None else train
    evaluate = args.learned_eval if evaluate is None else evaluate
    bj_eval = args.learned_bj_eval if bj_eval is None else bj_eval
    epochs = args.learned_epochs if epochs is None else epochs
    build()
    prob = cube32_k2_grf(0)
    c, e = kuhn_cube(prob.s)
    d, n = boundary_faces(c, e, prob.classify)
    M = HDGMesh(c, e, d, n, prob.k)
    M.set_boundary_data(torch.zeros(M.nfc, M.nf, dtype=torch.float64, device="cuda"))
    M.set_inner_tolerance(args.inner_rtol if args.inner_rtol is not None else 1e-5)
    ones = torch.ones(M.nelt, M.nq, dtype=torch.float64, device="cuda")
    sc = prob.s // 2
    nodes, weights, nc = kuhn_coarse_interpolation(prob.s, sc, interior_only=True)
    cs = CoarseSpace(nodes, weights, nc)
    lg = LearnedGuess(M, cs, grf_frequencies(), 1.0, ones, ones, kuhn_grid_points(sc), hidden=(256,), seed=3)
    hierarchy = kuhn_p1_hierarchy(prob.s, prob.dirichlet_planes)
    sync = torch.cuda.synchronize

    t0 = time.perf_counter()
    A, T, its = lg.generate([grf_sample(i) for i in range(train)])
    sync()
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    hist = lg.fit(A, T, epochs=epochs, batch=64, lr=1e-3)
    sync()
    t_fit = time.perf_counter() - t0
    lg.fold_normalisation()
    c_mean = torch.from_numpy(T.mean(axis=0)).cuda()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    rows = []
    M.set_coarse_space(*hierarchy)
    for j in range(evaluate):
        amps = grf_sample(100_000 + j)
        lg.set_field(amps)
        u, _, _ = M.solve_trace(1e-11, 20000)
        uHu = float((u * M.apply(u)).sum())

        def energy(x):
            err = u - x
            return float((err * M.apply(err)).sum()) / uHu
        row = {"energy_net": energy(lg.guess(amps)[0]), "energy_mean": energy(cs.guess(M, c_mean)[0])}
        variants = [("two_level", True)] + ([("block_jacobi", False)] if j < bj_eval else [])
        for pname, tl in variants:
            if not tl:
                M.set_coarse_space(None, None, None)
            for prec_name, prec in (("fp64", HDG_FP64), ("mixed", HDG_MIXED_FP32)):
                for start in ("zero", "learned"):
                    lg.set_field(amps)  # fresh assembly: the Galerkin set-up is inside the time
                    sync()
                    a, b = ev(), ev()
                    a.record()
                    if start == "learned":
                        uh, it, rr, used = lg.solve(amps, rtol=1e-10, maxit=40000, precision=prec, assemble=False)
                    else:
                        uh, it, rr = M.solve_trace(1e-10, 40000, precision=prec)
                    b.record()
                    sync()
                    row[f"{pname}_{prec_name}_{start}"] = (it, a.elapsed_time(b), rr)
            if not tl:
                M.set_coarse_space(*hierarchy)
        rows.append(row)

    def med(key, idx):
        vals = [r[key][idx] for r in rows if key in r]
        return float(np.median(vals)) if vals else None
    out = {"workload": "cube32_k2_grf: 32^3x6 Kuhn tets (196,608 elements), k=2, kappa=exp(GRF), c=f=1, u_D=0",
           "train_fields": train, "eval_fields": evaluate, "block_jacobi_eval_fields": min(bj_eval, evaluate),
           "network": {"sizes": lg.sizes, "epochs": epochs, "final_loss": hist[-1][1]},
           "generate_s": t_gen, "train_s": t_fit, "coarse_solve_iterations_median": float(np.median(its)),
           "energy_error_median": {"zero_start": 1.0, "mean_field_guess": float(np.median([r["energy_mean"] for r in rows])),
                                   "learned_guess": float(np.median([r["energy_net"] for r in rows]))},
           "median_iterations_and_ms": {}}
    for pname in ("block_jacobi", "two_level"):
        for prec_name in ("fp64", "mixed"):
            for start in ("zero", "learned"):
                k_ = f"{pname}_{prec_name}_{start}"
                out["median_iterations_and_ms"][k_] = {"iterations": med(k_, 0), "ms": med(k_, 1),
                                                       "max_relres": max([r[k_][2] for r in rows if k_ in r] or [0.0])}
    M.close()
    return out


def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_1305_1489_gb300 import build

    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_1305_1489_gb300", "libhdg.so")):
        build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    W = Workload(HEADLINE, dev, stream)
    r = run_workload(W, args, stream, dev, world, full=True)
    W.M.close()
    del W
    torch.cuda.empty_cache()
    prec = "df32" if args.asm == "df32" else "f64"
    out = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": prec,
        "dtype_note": ("assembly and condensation in double-float (pairs of FP32 on the FP32 pipe, about 48-bit "
                       "significand; C^K, C_f and the records match the FP64 oracle to 1e-11 relative); trace "
                       "solve in FP32 inner BiCGStab iterations with FP64 residuals and refinement to 1e-10; "
                       "recovery and postprocess in double-float" if prec == "df32" else "FP64 throughout"),
        "data": "synthetic",
        "config": {"workload": f"{HEADLINE}: unit cube 48^3x6 Kuhn tets ({r['nelt']} elements), interior vertices "
                               "jittered +-0.2h (seed 0), k=2, beta=(y,-x,0.5z), kappa=1+0.5 sin(2 pi z), c=1, tau=2.5, "
                               "Dirichlet on every face",
                   "nelt": r["nelt"], "nfc": r["nfc"], "trace_dofs": r["trace_dofs"], "k": r["k"],
                   "l2": "inputs (3.4 GB) larger than L2, and L2 flushed before every step (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "solve_in_step": ("mixed FP32/FP64" if args.solve == "mixed" else "FP64")
                   + " BiCGStab to 1e-10 relative residual, "
                   + ("two-level (block-Jacobi + P1 V-cycle) preconditioner" if args.coarse else
                      "block-Jacobi preconditioner"),
                   "inner_rtol": r["inner_rtol"], "coarse_levels": r["coarse_levels"], "autotune": r["autotune"]},
        "phases_ms": r["phases_ms"], "iterations_per_step": r["iterations_per_step"],
        "solve_time_to_1e-10": r["solve_time_to_1e-10"], "superconvergence": r["superconvergence"],
        "e2e": r["e2e"], "gpu_launches": r["gpu_launches"], "clocks": r["clocks"], "roofline": r["roofline"],
        "solve_roofline": r["solve_roofline"], "h2_contraction": r["h2_contraction"], "wall_s_timed": r["wall_s_timed"],
    }
    if "mixed_bf16_assembly" in r:
        out["mixed_bf16_assembly"] = r["mixed_bf16_assembly"]
    if world == 1 and rank == 0 and args.extras:
        out["extras"] = run_extras(args, dev, stream)
    return out


def run_extras(args, dev, stream):
    """The other configurations, each on its own (an extra that fails is recorded as such and
    cannot lose the headline line)."""
    import copy

    import torch

    extras = {}

    def guarded(name, fn):
        try:
            extras[name] = fn()
        except Exception as exc:  # noqa: BLE001
            extras[name] = {"error": repr(exc)}
        torch.cuda.empty_cache()

    def cube4():
        # the small FP64 workload: plain method (FP64 assembly, FP64 block-Jacobi PCG, no coarse space)
        a1 = copy.copy(args)
        a1.asm, a1.solve, a1.coarse = "fp64", "fp64", False
        W1 = Workload("cube4_k1", dev, stream)
        r1 = run_workload(W1, a1, stream, dev, 1, full=False)
        W1.M.close()
        return {"workload": f"cube4_k1: unit cube 4^3x6 Kuhn tets ({r1['nelt']} elements), k=1, kappa=c=tau=1, "
                            "Dirichlet everywhere, u = sin sin sin; FP64 assembly and FP64 block-Jacobi PCG to 1e-10 "
                            "(plain method)",
                **{k: r1[k] for k in ("value", "phases_ms", "iterations_per_step", "ms_per_step", "gpu_launches")}}

    def cube16():
        W2 = Workload(EXTRA_RD, dev, stream)
        r2 = run_workload(W2, args, stream, dev, 1, full=True)
        W2.M.close()
        return {"workload": f"{EXTRA_RD}: unit cube 16^3x6 Kuhn tets ({r2['nelt']} elements), k=3, variable kappa and "
                            "c, Dirichlet x=0,1 + Neumann elsewhere (reaction-diffusion, CG)",
                **{k: r2[k] for k in ("value", "phases_ms", "iterations_per_step", "ms_per_step", "solve_time_to_1e-10",
                                      "superconvergence", "e2e", "roofline", "solve_roofline", "gpu_launches",
                                      "inner_rtol")}}

    guarded("cube4_k1", cube4)
    guarded(EXTRA_RD, cube16)
    guarded("symmetric_rule", lambda: run_rule_comparison(dev, stream))
    guarded("batch_64", lambda: run_batch(args))
    guarded("cube32_k2_grf_learned", lambda: run_learned(args, train=args.extra_learned_train,
                                                         evaluate=args.extra_learned_eval, bj_eval=1,
                                                         epochs=args.learned_epochs))
    return extras



def profile_k1(name, s_sub, launches=2, asm="df32", autotune=True):
    """Small case for ncu captures of K1: the workload's problem on an s^3 x 6 mesh, autotuned as
    in the bench (the tuned launch shape appears in the kernel's template arguments)."""
    import torch

    from paper_1305_1489_gb300 import HDG_DF32, HDG_FP64, build

    build()
    W = Workload(name, torch.device("cuda", 0), torch.cuda.current_stream(), s=s_sub)
    M = W.M
    prec = HDG_DF32 if asm == "df32" else HDG_FP64
    M.assemble_condense(prec)
    tuned = M.autotune() if autotune else None
    for _ in range(launches):
        M.assemble_condense(prec)
    torch.cuda.synchronize()
    print(json.dumps({"profile_k1": {"workload": name, "s": s_sub, "nelt": M.nelt, "launches": launches, "asm": asm,
                                     "autotune": tuned}}))


def run_reference(args, rank):
    if rank != 0:
        return None
    base = oracle_baseline(HEADLINE, sample_elems=args.ref_sample, steps=args.steps, warmup=min(args.warmup, 1))
    return {
        "impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{HEADLINE}: unit cube 48^3x6 Kuhn tets (663552 elements), jittered, k=2, convection",
                   "impl": "FP64 CPU oracle (numpy), host cores"},
        "cpu_baseline": base,
        "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-sample", type=int, default=8192, help="oracle elements per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-steps", action="store_true", help="timed steps only, no comparisons or extras (profiling)")
    ap.add_argument("--workload", default=HEADLINE, help="workload of --only-steps")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the reaction-diffusion, batch and random-field extras")
    ap.add_argument("--asm", default="df32", choices=["df32", "fp64"],
                    help="assembly arithmetic: double-float on the FP32 pipe or native FP64")
    ap.add_argument("--inner-rtol", type=float, default=None,
                    help="FP32 inner solve tolerance (default: per workload, INNER_RTOL)")
    ap.add_argument("--solve", default="mixed", choices=["mixed", "fp64"], help="trace solve precision in the step")
    ap.add_argument("--solve-reps", type=int, default=2, help="repetitions of each time-to-1e-10 solve")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default persistent grid of the solve kernels")
    ap.add_argument("--no-coarse", dest="coarse", action="store_false",
                    help="block-Jacobi only (no two-level preconditioner) in the step")
    ap.add_argument("--batch-only", action="store_true", help="time only the batch and exit")
    ap.add_argument("--batch-n", type=int, default=64)
    ap.add_argument("--batch-reps", type=int, default=3)
    ap.add_argument("--profile-k1", type=int, default=0, help="run K1 twice on an s^3 x 6 mesh and exit")
    ap.add_argument("--profile-workload", default=HEADLINE)
    ap.add_argument("--e2e-only", action="store_true", help="the end-to-end leg alone (timing of the host pipeline)")
    ap.add_argument("--e2e-chunks", type=int, default=E2E_CHUNKS, help="element ranges of the host pipeline")
    ap.add_argument("--profile-solve", type=int, default=0,
                    help="two-level mixed trace solves and two recoveries on an s^3 x 6 mesh of --profile-workload, "
                         "then exit")
    ap.add_argument("--profile-tc", type=int, default=0,
                    help="run the tensor-core mass contraction twice on an s^3 x 6 mesh and exit")
    ap.add_argument("--learned", action="store_true", help="train and evaluate the learned guess and exit")
    ap.add_argument("--learned-train", type=int, default=2000)
    ap.add_argument("--learned-eval", type=int, default=200)
    ap.add_argument("--learned-bj-eval", type=int, default=20, help="held-out fields also timed with block-Jacobi")
    ap.add_argument("--learned-epochs", type=int, default=60)
    ap.add_argument("--extra-learned-train", type=int, default=200, help="training fields of the learned extra")
    ap.add_argument("--extra-learned-eval", type=int, default=8, help="held-out fields of the learned extra")
    args = ap.parse_args()
    if args.profile_k1:
        profile_k1(args.profile_workload, args.profile_k1, asm=args.asm)
        return
    if args.profile_solve:
        import torch

        from paper_1305_1489_gb300 import HDG_DF32, HDG_MIXED_FP32, build
        build()
        W = Workload(args.profile_workload, torch.device("cuda", 0), torch.cuda.current_stream(), s=args.profile_solve)
        M = W.M
        M.set_inner_tolerance(INNER_RTOL.get(args.profile_workload, 1e-4))
        M.set_coarse_space(*W.hierarchy())
        M.assemble_condense(HDG_DF32)
        runs = []
        for _ in range(2):
            uh, it, rr = M.solve_trace(rtol=1e-10, maxit=20000, precision=HDG_MIXED_FP32)
            runs.append({"iterations": it, "relres": rr})
        for _ in range(2):  # and the recovery (K2) of the last solution
            M.recover(uh)
        torch.cuda.synchronize()
        print(json.dumps({"profile_solve": {"workload": args.profile_workload, "s": args.profile_solve,
                                            "nelt": M.nelt, "runs": runs}}))
        return
    if args.profile_tc:
        import torch

        from paper_1305_1489_gb300 import build
        build()
        W = Workload(args.profile_workload, torch.device("cuda", 0), torch.cuda.current_stream(), s=args.profile_tc)
        res = h2_contraction(W, torch.device("cuda", 0), torch.cuda.current_stream(), reps=1)
        for _ in range(2):  # the split-BF16 contraction of the HDG_MIXED_BF16 assembly
            W.M.mixed_masses()
        torch.cuda.synchronize()
        print(json.dumps({"profile_tc": {"nelt": W.M.nelt, **res}}))
        return
    if args.e2e_only:
        import torch

        from paper_1305_1489_gb300 import HDG_DF32, HDG_MIXED_FP32, build
        build()
        dev = torch.device("cuda", 0)
        stream = torch.cuda.Stream(device=dev)
        torch.cuda.set_stream(stream)
        W = Workload(args.workload, dev, stream)
        W.M.set_inner_tolerance(INNER_RTOL.get(W.name, 1e-4))
        W.M.set_coarse_space(*W.hierarchy())
        W.M.assemble_condense(HDG_DF32)
        tuned = W.M.autotune() if args.autotune else None
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        print(json.dumps({"e2e_only": e2e_leg(W, args, stream, 1, HDG_DF32, HDG_MIXED_FP32, flush),
                          "autotune": tuned}))
        return
    if args.only_steps:
        import torch

        from paper_1305_1489_gb300 import build
        build()
        dev = torch.device("cuda", 0)
        stream = torch.cuda.Stream(device=dev)
        torch.cuda.set_stream(stream)
        W = Workload(args.workload, dev, stream)
        r = run_workload(W, args, stream, dev, 1, full=False)
        print(json.dumps({"only_steps": {k: r[k] for k in ("value", "phases_ms", "iterations_per_step", "ms_per_step",
                                                            "gpu_launches", "solve_roofline", "autotune")}}))
        return
    if args.batch_only:
        print(json.dumps({"batch": run_batch(args)}))
        return
    if args.learned:
        print(json.dumps({"learned": run_learned(args)}))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank)
        if out is not None:
            print(json.dumps(out))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    out = run_gpu(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = oracle_baseline(HEADLINE, sample_elems=args.ref_sample, steps=1, warmup=1)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
