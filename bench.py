#!/usr/bin/env python3
"""Benchmark: FGMRES solves/s to a 1e-8 relative residual on the Q2-Q1 lid-driven
Stokes cavity, 256x256 mesh (592,387 dofs), 8 right-hand sides per launch.

One step = one batched flexible-GMRES solve of the 8 right-hand sides with the
EMIN-AMG V-cycle as preconditioner: every part of the hot path runs in it (block
residual, Braess-Sarazin Schur right-hand side, multicolor Gauss-Seidel,
velocity/pressure update, restriction, prolongation, coarsest solve, FP64
Arnoldi).  `value` uses the FP32 V-cycle inside FP64 FGMRES; the plain FP64
V-cycle is timed beside it.  Inputs are resident in HBM when the timed region
starts; `e2e` repeats the measurement through the host-buffer entry point.

--impl reference times the FP64 CPU oracle on the host cores instead.
Under torchrun each rank solves its own seeded batch (weak scaling, no
data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MESH = 256
NRHS = 8
ARNOLDI_NV = 12        # basis vectors of the timed Gram-Schmidt pass
FP64_PEAK_TFLOPS = 1.25  # GB300 nominal dense FP64 rate (1/64 of its FP32 rate)
RTOL = 1e-8
RESTART = 100
MAXIT = 300
METRIC = "solves/s @1e-8 rel resid: FP32 V-cycle vs FP64; HBM GB/s; p50/p99 latency"
WORKLOAD = (f"2D Stokes Q2-Q1 leaky lid-driven cavity, {MESH}x{MESH} mesh (592,387 dofs), nu=1, "
            f"{NRHS} seeded uniform[-1,1] body loads batched in one launch, FGMRES to {RTOL:g}")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving stream")
    ap.add_argument("--no-vanka", action="store_true", help="skip the Vanka-smoother side line")
    ap.add_argument("--no-ilu", action="store_true", help="skip the ILU(1)-smoother side line")
    ap.add_argument("--no-picard", action="store_true", help="skip the Picard (steady Navier-Stokes) side line")
    ap.add_argument("--no-setup", action="store_true", help="skip the setup-time side line")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the side line with the other workloads (16x16 pinned, 512x512 Oseen x32, 48^3)")
    ap.add_argument("--configs", action="store_true",
                    help="instead of the default run: time the other workloads (16x16 pinned Stokes, 512x512 "
                         "Oseen x32, 48^3 Stokes) with the FP64 and FP32 V-cycles, and the oracle on the first two")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-active", type=int, default=None, help="requests running at once (default SERVE_ACTIVE)")
    ap.add_argument("--serve-merge", type=int, default=None, help="columns stacked per cohort (default SERVE_MERGE)")
    ap.add_argument("--ncu", action="store_true",
                    help="short run for an ncu launch list: one warm-up solve, then one solve (FP32 V-cycle) "
                         "inside a cudaProfilerStart/Stop range")
    ap.add_argument("--ncu-config", default=None, choices=sorted(CONFIGS),
                    help="like --ncu on one of the other configs (FP32 V-cycle, its own right-hand sides)")
    ap.add_argument("--ncu-setup", action="store_true",
                    help="short run for ncu: a hierarchy for the bench workload, a first device reuse of it, then "
                         "a second device reuse inside a cudaProfilerStart/Stop range")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    """nvidia-smi every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# algorithmic bytes per kernel launch: each kernel's compulsory reads and writes (matrix
# values and column indices once, the vectors it gathers K values per entry from, and the
# vectors it reads and writes once per row), as the formulas below state

def algorithmic_bytes(H, level, cls, K, s, zero_fraction=0.25):
    """Compulsory bytes of one launch of kernel class `cls` on `level`: each matrix
    entry (value + int32 column) and row pointer read once, each vector operand
    read or written once (K right-hand sides of s bytes each).
    The Gauss-Seidel class is one fused launch: all gs_iters iterations over all colors.
    The velocity predictor's first sweep of a cycle starts from x = 0 and reads no
    matrix; `zero_fraction` of its launches are of that kind (1 of 4 in V(2,2))."""
    info = H.level_info(level)
    d, nv, np_ = info["dim"], info["n_v"], info["n_p"]
    N = d * nv + np_
    mat = lambda nnz, rows: nnz * (s + 4) + (rows + 1) * 4  # noqa: E731
    vec = lambda n: n * K * s  # noqa: E731
    if cls == "velocity":
        full = mat(info["nnz_A"], nv) + mat(info["nnz_Bt"], d * nv) + nv * s + vec(d * nv) + vec(N) + vec(d * nv)
        zero = nv * s + vec(d * nv) + vec(d * nv)
        return zero_fraction * zero + (1 - zero_fraction) * full
    if cls == "schur_rhs":
        return mat(info["nnz_B"], np_) + vec(d * nv) + 2 * vec(np_)
    if cls == "gs_color":
        # one fused launch = gs_iters Gauss-Seidel iterations over all colors: every pass
        # reads the matrix (off-diagonal entries, row pointers, 1/S_ii and the row order),
        # while the vector operands g (read) and dp (read and written) count once per launch
        nnz_off = info["nnz_S"] - np_
        return H.params.gs_iters * (mat(nnz_off, np_) + np_ * (4 + s)) + 3 * vec(np_)
    if cls == "update":
        return mat(info["nnz_Bt"], d * nv) + nv * s + vec(d * nv) + 2 * vec(np_) + vec(N)
    if cls == "residual":
        return (mat(info["nnz_A"], nv) + mat(info["nnz_Bt"], d * nv) + mat(info["nnz_B"], np_) + 3 * vec(N))
    if cls == "restrict":
        c = H.level_info(level + 1)
        return (mat(info["nnz_R"], c["n_v"]) + mat(info["nnz_Rp"], c["n_p"]) + vec(N)
                + vec(c["dim"] * c["n_v"] + c["n_p"]))
    if cls == "prolong":
        c = H.level_info(level + 1)
        return (mat(info["nnz_P"], nv) + mat(info["nnz_Pp"], np_) + 2 * vec(N) + vec(c["dim"] * c["n_v"] + c["n_p"]))
    if cls == "coarse":
        return N * N * 8 + 2 * vec(N)
    if cls == "vanka":
        raise KeyError("vanka bytes are counted per step by vanka_bytes")
    raise KeyError(cls)


def vanka_bytes(H, level, K, s):
    """Compulsory bytes of one Vanka step (all colors) on `level`: every block's
    inverse (m^2 values), for every dof of every block its row of the block matrix
    (values, columns, and the K gathered x values per entry), f read and x
    written for the block's dofs (K values each)."""
    import numpy as np
    info = H.level_info(level)
    d, nv = info["dim"], info["n_v"]
    V = H.level_vanka(level)
    m = np.diff(V["ptr"]).astype(np.int64)
    rA = np.diff(H.level_matrix(level, "A")[0])
    rBt = np.diff(H.level_matrix(level, "Bt")[0])
    rB = np.diff(H.level_matrix(level, "B")[0])
    q = V["dofs"].astype(np.int64)
    nu = d * nv
    row_nnz = np.where(q < nu, rA[np.minimum(q, nu - 1) % nv] + rBt[np.minimum(q, nu - 1)],
                       rB[np.maximum(q - nu, 0)])
    return int((m * m).sum() * s + (row_nnz * (4 + s + K * s)).sum() + 2 * K * s * len(q))


def ilu_bytes(H, level, K, s, from_zero):
    """Compulsory bytes of one ILU(1) step's two substitutions on `level`: the factors
    (values and columns, row pointers, the ticket order, the permutation, the pivots'
    reciprocals), for every factor entry the K values of the row it refers to, and r
    read, y written and read, d written, x written (and read unless from zero), K
    values per row each."""
    F = H.level_ilu(level)
    n = len(F["perm"])
    nnz = len(F["lower"][1]) + len(F["upper"][1])
    return int(nnz * (s + 4) + nnz * K * s + 2 * (n + 1) * 4 + 2 * n * 4 + 2 * n * 4 + n * s
               + (5 if from_zero else 6) * n * K * s)


def load_traffic(kernel, level, K, s):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the
    current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
    except ValueError:
        return None
    if rec.get("source_sha") != source_sha():
        return None
    e = rec.get("kernels", {}).get(f"{kernel}/L{level}/K{K}/{'f32' if s == 4 else 'f64'}")
    return e.get("dram_bytes_per_launch") if e else None


# the files that define the V-cycle kernels and their launches: the committed DRAM
# counters of a V-cycle kernel stay valid while these are unchanged
VCYCLE_KERNEL_SOURCES = ("device.cuh", "vcycle.cuh", "vcycle_inst.cu")


def source_sha():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1607_02489_gb300", "csrc")
    for f in VCYCLE_KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# CPU oracle leg

CPU_SAMPLE = ("the FP64 oracle (numpy/scipy) solving 1 of the 8 right-hand sides of the same "
              "256x256 lid-cavity workload to 1e-8 with the same method; hierarchy set up beforehand, untimed")


CONFIGS = {
    "C1": dict(name="2D Stokes 16x16, pinned pressure, 1 rhs", kind="pinned", n=16, nrhs=1),
    "C3": dict(name="2D Oseen 512x512 on [-1,1]^2, recirculating wind, Re=10, 32 rhs", kind="oseen", n=512,
               nrhs=32, Re=10.0),
    "C4": dict(name="3D Stokes 48^3 lid-driven cube, 1 rhs", kind="lid3d", n=48, nrhs=1),
}


def _config_problem(c, nrhs=None):
    from synth import oseen_recirculating_2d, stokes_lid_3d, stokes_pinned_2d
    k = nrhs or c["nrhs"]
    if c["kind"] == "pinned":
        return stokes_pinned_2d(c["n"], nrhs=k)
    if c["kind"] == "oseen":
        return oseen_recirculating_2d(c["n"], Re=c["Re"], nrhs=k)
    return stokes_lid_3d(c["n"], nrhs=k)


def _oracle_config_worker(key, q):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import setup_hierarchy, fgmres
    p = _config_problem(CONFIGS[key], nrhs=1)
    t0 = time.perf_counter()
    Ho = setup_hierarchy(p)
    t1 = time.perf_counter()
    x, it, rel, _ = fgmres(Ho, p.b, rtol=RTOL, restart=RESTART, maxit=MAXIT)
    q.put((t1 - t0, time.perf_counter() - t1, int(it[0])))


def run_oracle_config(key):
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    pr = ctx.Process(target=_oracle_config_worker, args=(key, q))
    pr.start()
    res = q.get()
    pr.join()
    return res


def config_records(g, torch, reps=3):
    """The other workloads of the method (16x16 pinned Stokes, 512x512 Oseen x32 at Re 10,
    48^3 Stokes): setup seconds, and solves/s with the FP64 and FP32 V-cycles (inputs
    resident, CUDA events over `reps` solves after one warm-up solve), the FGMRES
    iterations and the V-cycle kernels' algorithmic bandwidth."""
    import numpy as np
    peak = measured_peaks()[0]
    out = {}
    for key, c in CONFIGS.items():
        p = _config_problem(c)
        k = c["nrhs"]
        b = torch.tensor(p.b, device="cuda")
        x = torch.zeros_like(b)
        rec = {"workload": c["name"], "dofs": int(p.N), "nrhs": k}
        for fp32 in (0, 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            H = g.Hierarchy(p, max_nrhs=k, vcycle_fp32=fp32)
            setup_s = time.perf_counter() - t0
            H.fgmres(b, x, rtol=RTOL, restart=60, maxit=MAXIT)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                st, its, rel = H.fgmres(b, x, rtol=RTOL, restart=60, maxit=MAXIT)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            s = 4 if fp32 else 8
            vms, vcnt = H.profile_vcycle(k, reps=2)
            vbytes = sum(algorithmic_bytes(H, l, cl, k, s) * vcnt[l, j] / 2
                         for l in range(vms.shape[0]) for j, cl in enumerate(g.KERNEL_CLASSES) if vcnt[l, j])
            gbs = vbytes / (vms.sum() / 2 / 1000.0) / 1e9
            rec["fp32" if fp32 else "fp64"] = {"solves_per_s": k / (ms / 1000.0), "ms_per_solve_batch": ms,
                                               "status": int(st), "iterations_max": int(np.max(its)),
                                               "relres_max": float(np.max(rel)), "vcycle_kernels_GBs": gbs,
                                               "vcycle_kernels_frac": gbs / peak, "setup_s": setup_s,
                                               "gs_variants": [v for v, _, _ in H.gs_variants(k)]}
            del H
            torch.cuda.empty_cache()
        out[key] = rec
    return out


def configs_main(args):
    """One JSON line with the other workloads (config_records) and the oracle (1 core,
    1 right-hand side) on the 16x16 pinned problem and the 512x512 Oseen problem."""
    import torch
    oracle = {}
    if not args.no_cpu_baseline:
        for key in ("C1", "C3"):  # before any CUDA work in this process
            setup_s, solve_s, its = run_oracle_config(key)
            oracle[key] = {"solves_per_s": 1.0 / solve_s, "seconds": solve_s, "setup_s_untimed": setup_s,
                           "iterations": its, "cores": 1, "sample": "1 right-hand side"}
    import paper_1607_02489_gb300 as g
    g._build.build()
    out = config_records(g, torch)
    for key, rec in oracle.items():
        out[key]["oracle"] = rec
    print(json.dumps({"metric": METRIC, "configs": out, "peak_GBs": measured_peaks()[0], "data": "synthetic"}),
          flush=True)


def setup_line(g, torch, p):
    """Setup seconds of the bench workload (592,387 dofs), host against device
    (amg_params.device_setup): a fresh hierarchy, and hierarchies for the next
    matrices of a sequence with the same structure reusing its coarsening (Section
    6.1; the first device reuse also builds the structure's patterns and maps, later
    ones share them).  Each includes the upload of the FP32 V-cycle."""
    from synth import make_problem
    q = make_problem(MESH, 2, 0.0, 1.0, bc="lid", nu=0.5, nrhs=1, seed=1)
    out = {}
    for dev in (0, 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = g.Hierarchy(p, max_nrhs=NRHS, vcycle_fp32=1, device_setup=dev)
        t1 = time.perf_counter()
        R1 = g.Hierarchy(q, reuse=H, max_nrhs=NRHS, vcycle_fp32=1, device_setup=dev)
        t2 = time.perf_counter()
        R2 = g.Hierarchy(p, reuse=R1, max_nrhs=NRHS, vcycle_fp32=1, device_setup=dev)
        t3 = time.perf_counter()
        out["device" if dev else "host"] = {"fresh_s": t1 - t0, "first_reuse_s": t2 - t1, "reuse_s": t3 - t2}
        del R2, R1, H
    return {"workload": "the bench's 256x256 lid cavity (fresh), then two more matrices of the same structure "
                        "(nu = 0.5, then nu = 1 again) reusing the coarsening", **out,
            "paper_context": {"setup_s": 13.34, "incremental_setup_s": 3.60,
                              "source": "Table 1 and Section 6.1 (BS(2,2), 592,387 dofs; MueLu, hardware unstated)"}}


def _oracle_worker(n_solves, q):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from synth import stokes_lid_2d
    from oracle import setup_hierarchy, fgmres
    p = stokes_lid_2d(MESH, nrhs=1, seed=0)
    Ho = setup_hierarchy(p)
    times = []
    its = []
    x = None
    for _ in range(n_solves):
        t0 = time.perf_counter()
        x, it, rel, _ = fgmres(Ho, p.b, rtol=RTOL, restart=RESTART, maxit=MAXIT)
        times.append(time.perf_counter() - t0)
        its.append(int(it[0]))
    q.put((times, its, x[:, 0]))


def run_oracle(n_solves):
    """Time the oracle in a fresh single-threaded process (spawned, so no CUDA state is forked)."""
    import multiprocessing as mp
    env_before = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["MKL_NUM_THREADS"] = "1"
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    pr = ctx.Process(target=_oracle_worker, args=(n_solves, q))
    pr.start()
    times, its, x = q.get()
    pr.join()
    if env_before is None:
        os.environ.pop("OMP_NUM_THREADS", None)
    return times, its, x


def reference_main(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    times, its, _ = run_oracle(args.warmup + args.steps)
    timed = times[args.warmup:]
    total = sum(timed)
    value = len(timed) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / len(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "1 right-hand side per step"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": CPU_SAMPLE, "iterations": its[-1]},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# Picard: steady Navier-Stokes lid cavity with reused coarsening

def picard_line(g, torch, n=64, nu=0.01):
    """The Picard sequence of the steady lid cavity (Section 6.2's test systems) with
    the GPU solver: each Oseen step assembled on the host (untimed input), its
    hierarchy built reusing the first Oseen step's coarsening, solved by FGMRES with
    the FP32 V-cycle to 1e-11; stops at the paper's 1e-8 nonlinear residual."""
    import numpy as np
    from synth import lid_cavity_problem
    p = lid_cavity_problem(n, nu)
    b = torch.tensor(p.b, device="cuda")
    x = torch.zeros_like(b)
    H = g.Hierarchy(p, max_nrhs=1, vcycle_fp32=1)
    H.fgmres(b, x, rtol=1e-11, restart=100, maxit=400)
    xs = x.cpu().numpy()[:, 0]
    H_first, setup_fresh, setup_reuse, solve_ms, its_all, res = None, [], [], [], [], []
    for _ in range(100):
        q = lid_cavity_problem(n, nu, wind_nodal=xs[:2 * p.n_v].reshape(2, p.n_v))
        r = float(np.linalg.norm(q.b[:, 0] - q.full_matrix() @ xs))
        res.append(r)
        if r < 1e-8:
            break
        t0 = time.perf_counter()
        if H_first is None:
            H = H_first = g.Hierarchy(q, max_nrhs=1, vcycle_fp32=1)
            setup_fresh.append(time.perf_counter() - t0)
        else:
            H = g.Hierarchy(q, reuse=H_first, max_nrhs=1, vcycle_fp32=1)
            setup_reuse.append(time.perf_counter() - t0)
        bq = torch.tensor(q.b, device="cuda")
        xq = torch.zeros_like(bq)
        H.fgmres(bq, xq, rtol=1e-11, restart=100, maxit=400)  # first solve: capture and autotuning
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        xq.zero_()
        e0.record()
        st, its, rel = H.fgmres(bq, xq, rtol=1e-11, restart=100, maxit=400)
        e1.record()
        torch.cuda.synchronize()
        solve_ms.append(e0.elapsed_time(e1))
        its_all.append(int(its[0]))
        xs = xq.cpu().numpy()[:, 0]
    return {"workload": f"steady Navier-Stokes leaky lid cavity, (-1,1)^2, {n}x{n}, nu={nu:g}, Picard from the "
                        "Stokes solution, FGMRES / FP32 V-cycle to 1e-11 per step",
            "picard_steps": len(solve_ms), "final_nonlinear_residual": res[-1], "converged": res[-1] < 1e-8,
            "setup_s_fresh": float(np.mean(setup_fresh)) if setup_fresh else None,
            "setup_s_reused_coarsening": float(np.mean(setup_reuse)) if setup_reuse else None,
            "solve_ms_per_step": float(np.mean(solve_ms)), "fgmres_iterations": its_all}


# ----------------------------------------------------------------------------
# replicas: one independent batch per GPU

def replica_aggregate(dist, device, seconds, units):
    """Weak scaling over ranks: (max of the ranks' times, sum of their units of work).
    Every rank calls it; with one process it returns its arguments."""
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def rank_batch(rank, mesh=MESH, nrhs=NRHS):
    """The seeded batch a rank solves: the lid cavity with right-hand-side seed = rank."""
    from synth import stokes_lid_2d
    return stokes_lid_2d(mesh, nrhs=nrhs, seed=rank)


# ----------------------------------------------------------------------------
# serving: a Poisson stream of Oseen solves over 15 resident hierarchies

SERVE_RATE = 200.0
SERVE_WARM = 12
SERVE_ACTIVE = 8
SERVE_RESTART = 50
SERVE_MERGE = 8
SERVE_WORKLOAD = ("Poisson arrivals at 200 req/s (seed 0) of 2D Oseen Q2-Q1 solves on [-1,1]^2 with the "
                  "recirculating wind, n from {64,128,256,384,512}, Re from {1,10,100}, 1-8 uniform[-1,1] "
                  "right-hand sides each, FP32 V-cycle / FP64 FGMRES to 1e-8, host buffers in and out")


def serve(g, torch, dev, n_requests, seed=0, max_active=None, merge_k=None):
    """Builds the 15 hierarchies (untimed: setup is per matrix), runs a short
    warm-up stream, then the timed stream; latency = arrival to result on the host."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor
    from synth import MESHES, REYNOLDS, oseen_recirculating_2d, serving_stream, homogeneous_rhs

    def build(key):
        n, Re = key
        torch.cuda.set_device(dev)
        p = oseen_recirculating_2d(n, Re=Re, nrhs=1)
        return key, (p, g.Hierarchy(p, max_nrhs=8, vcycle_fp32=1))

    t0 = time.perf_counter()
    keys = [(n, Re) for n in MESHES for Re in REYNOLDS]
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        hs = dict(ex.map(build, keys))
    setup_s = time.perf_counter() - t0

    def requests(stream):
        out = []
        for r in stream:
            p, H = hs[(r["n"], r["Re"])]
            b = torch.from_numpy(homogeneous_rhs(p, r["nrhs"], r["rhs_seed"])).pin_memory()
            out.append(dict(t=r["t"], H=H, b=b, x=torch.zeros_like(b).pin_memory(), rtol=RTOL, n=r["n"],
                            nrhs=r["nrhs"]))
        return out

    max_active = max_active or SERVE_ACTIVE
    merge_k = SERVE_MERGE if merge_k is None else merge_k

    def one_stream(policy):
        sv = g.Server(max_active=max_active, restart=SERVE_RESTART, maxit=MAXIT, merge_k=merge_k, policy=policy)
        t0 = time.perf_counter()
        for key in keys:  # one slot per (hierarchy, K) up front: no allocation or capture in the stream
            for k in (1, 2, 4, 8):
                sv.reserve(hs[key][1], k, 1)
        reserve_s = time.perf_counter() - t0
        g.run_stream(sv, requests(serving_stream(SERVE_WARM, SERVE_RATE, seed=1000 + seed)))
        reqs = requests(serving_stream(n_requests, SERVE_RATE, seed=seed))
        l0, c0 = sv.stats()["kernel_launches"], sv.stats()["cohorts"]
        res = g.run_stream(sv, reqs)
        st = sv.stats()
        sv.close()
        ok = all(r["status"] == g.AMG_OK and np.all(r["relres"] <= RTOL) for r in res)
        lat = np.array([r["done"] - r["arrival"] for r in res])
        wall = max(r["done"] for r in res) - min(r["arrival"] for r in res)
        rhs = sum(q["nrhs"] for q in reqs)
        by_n = {}
        for q, r in zip(reqs, res):
            by_n.setdefault(q["n"], []).append(1000.0 * (r["done"] - r["arrival"]))
        return {"workload": SERVE_WORKLOAD, "policy": ["submission order", "smallest work first"][policy],
                "requests": len(reqs), "rhs_solves": rhs, "all_converged": bool(ok),
                "wall_s": wall, "requests_per_s": len(reqs) / wall, "solves_per_s": rhs / wall,
                "offered_rps": SERVE_RATE, "max_active": max_active, "restart": SERVE_RESTART,
                "merge_k": merge_k, "cohorts": int(st["cohorts"] - c0),
                "latency_ms": {"p50": float(np.percentile(lat, 50) * 1000),
                               "p99": float(np.percentile(lat, 99) * 1000), "max": float(lat.max() * 1000)},
                "latency_p50_ms_by_mesh": {str(n): float(np.percentile(v, 50)) for n, v in sorted(by_n.items())},
                "queued_p50_ms": float(np.percentile([r["queued"] for r in res], 50) * 1000),
                "iterations_max": int(max(int(np.max(r["iters"])) for r in res)),
                "gpu_launches": int(st["kernel_launches"] - l0), "slots_created": int(st["slots_created"]),
                "slots_released": int(st["slots_released"]), "errors": int(st["errors"]),
                "setup_s_untimed": setup_s, "reserve_s_untimed": reserve_s}

    out = one_stream(0)
    sjf = one_stream(1)
    out["smallest_work_first"] = {k: sjf[k] for k in ("solves_per_s", "requests_per_s", "latency_ms",
                                                      "latency_p50_ms_by_mesh", "cohorts", "all_converged")}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return reference_main(args)
    if args.configs:
        return configs_main(args)
    if args.ncu or args.ncu_setup or args.ncu_config:
        args.no_cpu_baseline = True
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # the CPU oracle runs first, in a spawned process, before any CUDA work
    cpu = None
    x_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t, its_cpu, x_oracle = run_oracle(1)
        cpu = {"value": 1.0 / t[0], "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": CPU_SAMPLE,
               "seconds": t[0], "iterations": its_cpu[0]}

    import paper_1607_02489_gb300 as g
    g._build.build()
    p = rank_batch(rank)
    if args.ncu_setup:
        from synth import make_problem
        q = make_problem(MESH, 2, 0.0, 1.0, bc="lid", nu=0.5, nrhs=1, seed=1)
        H = g.Hierarchy(p, max_nrhs=NRHS, vcycle_fp32=1)
        R1 = g.Hierarchy(q, reuse=H, max_nrhs=NRHS, vcycle_fp32=1)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        R2 = g.Hierarchy(p, reuse=R1, max_nrhs=NRHS, vcycle_fp32=1)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(f"device reuse setup: {R2.num_levels()} levels", flush=True)
        return
    if args.ncu or args.ncu_config:
        if args.ncu_config:
            p = _config_problem(CONFIGS[args.ncu_config])
        H = g.Hierarchy(p, max_nrhs=p.b.shape[1], vcycle_fp32=1)
        b = torch.tensor(p.b, device=dev)
        x = torch.zeros_like(b)
        for rep in range(2):
            n0 = H.kernel_launches()
            if rep == 1:  # the profiled range (ncu --profile-from-start off): the second solve only
                torch.cuda.profiler.start()
            st, its, rel = H.fgmres(b, x, rtol=RTOL, restart=RESTART, maxit=MAXIT)
            torch.cuda.synchronize()
            if rep == 1:
                torch.cuda.profiler.stop()
            print(f"solve {rep}: status {st}, iterations {its.tolist()}, kernels {H.kernel_launches() - n0}",
                  flush=True)
        return
    H32 = g.Hierarchy(p, max_nrhs=NRHS, vcycle_fp32=1)
    H64 = g.Hierarchy(p, max_nrhs=NRHS)
    b = torch.tensor(p.b, device=dev)
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(H, steps, warm):
        for _ in range(warm):
            st, its, rel = H.fgmres(b, x, rtol=RTOL, restart=RESTART, maxit=MAXIT)
            assert st == g.AMG_OK, st
        barrier()
        torch.cuda.synchronize()
        n0 = H.kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lat = []
        e0.record(stream)
        for _ in range(steps):
            t0 = time.perf_counter()
            st, its, rel = H.fgmres(b, x, rtol=RTOL, restart=RESTART, maxit=MAXIT)
            lat.append(time.perf_counter() - t0)
            assert st == g.AMG_OK and np.all(rel <= RTOL), (st, rel)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms, solves = replica_aggregate(dist, dev, e0.elapsed_time(e1), NRHS * steps)
        return ms, solves, H.kernel_launches() - n0, its, rel, lat

    sampler = ClockSampler(local)
    sampler.start()
    ms32, solves, launches32, its32, rel32, lat32 = timed(H32, args.steps, args.warmup)
    clocks = sampler.stop()
    x32 = x[:, 0].cpu().numpy()
    ms64, _, launches64, its64, rel64, lat64 = timed(H64, args.steps, args.warmup)
    x64 = x[:, 0].cpu().numpy()
    accuracy = None
    if x_oracle is not None:
        nu = 2 * p.n_v

        def err(a):  # relative 2-norm error, pressure compared up to its constant
            d = a - x_oracle
            d[nu:] -= d[nu:].mean()
            ref = x_oracle.copy()
            ref[nu:] -= ref[nu:].mean()
            return float(np.linalg.norm(d) / np.linalg.norm(ref))

        accuracy = {"fp32_vcycle_vs_oracle": err(x32), "fp64_vcycle_vs_oracle": err(x64),
                    "what": "relative 2-norm error of right-hand side 0's FGMRES solution (both stopped at "
                            f"{RTOL:g}) against the FP64 oracle's, pressure mean removed"}

    value = solves / (ms32 / 1000.0)
    value64 = solves / (ms64 / 1000.0)

    # end to end through the host-buffer entry point (pinned host memory)
    bh = torch.tensor(p.b).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    for _ in range(max(1, args.warmup)):
        H32.fgmres_host(bh, xh, rtol=RTOL, restart=RESTART, maxit=MAXIT)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st, its_e, rel_e = H32.fgmres_host(bh, xh, rtol=RTOL, restart=RESTART, maxit=MAXIT)
    torch.cuda.synchronize()
    e2e_s, _ = replica_aggregate(dist, dev, time.perf_counter() - t0, 0)
    e2e = {"value": solves / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(bh.numel() * 8),
           "d2h_bytes_per_step": int(xh.numel() * 8)}

    # dominant V-cycle kernel, timed live with CUDA events on the launching stream
    H32.vcycle(b, x)
    reps = 20
    ms_tab, cnt_tab = H32.profile_vcycle(NRHS, reps=reps)
    lvl, ci = np.unravel_index(np.argmax(ms_tab), ms_tab.shape)
    cls = g.KERNEL_CLASSES[ci]
    avg_ms = ms_tab[lvl, ci] / cnt_tab[lvl, ci]
    bytes_launch = algorithmic_bytes(H32, int(lvl), cls, NRHS, 4)
    peak, peak_kind = measured_peaks()
    achieved = bytes_launch / (avg_ms / 1000.0) / 1e9
    vcycle_ms = ms_tab.sum() / reps
    vcycle_bytes = sum(algorithmic_bytes(H32, l, c, NRHS, 4) * cnt_tab[l, k] / reps
                       for l in range(ms_tab.shape[0]) for k, c in enumerate(g.KERNEL_CLASSES) if cnt_tab[l, k])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": load_traffic(cls, int(lvl), NRHS, 4),
                "kernel": f"{cls} (level {int(lvl)}, fp32, {NRHS} rhs)", "peak_kind": peak_kind,
                "bytes_per_launch": bytes_launch, "avg_launch_us": avg_ms * 1000.0,
                "vcycle_kernels_GBs": vcycle_bytes / (vcycle_ms / 1000.0) / 1e9,
                "vcycle_kernels_frac": vcycle_bytes / (vcycle_ms / 1000.0) / 1e9 / peak}
    # the FGMRES Arnoldi kernels, bound by FP64 arithmetic: one Gram-Schmidt pass with
    # ARNOLDI_NV basis vectors (about the middle of a 22-23 iteration solve), CUDA events
    NV = ARNOLDI_NV
    ms_dot, ms_upd = H32.profile_arnoldi(NRHS, NV, reps=10)
    fma = (NV + 1) * p.N * NRHS
    arnoldi = {"bound": "fp64", "kernels": f"k_mdot_partial / k_maxpy, {NV} basis vectors of {p.N} x {NRHS}",
               "achieved": [2 * fma / (t / 1000.0) / 1e12 for t in (ms_dot, ms_upd)],
               "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "peak_kind": "nominal (GB300 FP64, no measured figure)",
               "frac": [2 * fma / (t / 1000.0) / 1e12 / FP64_PEAK_TFLOPS for t in (ms_dot, ms_upd)],
               "avg_launch_us": [1000.0 * ms_dot, 1000.0 * ms_upd],
               "dram_algorithmic_GBs": [8.0 * (NV + 1) * p.N * NRHS / (t / 1000.0) / 1e9 for t in (ms_dot, ms_upd)]}
    gs_variants = [f"L{l}: {v}{' x' + str(c) if v == 'cluster' else (' shape ' + str(c) if v == 'pipelined' else '')}"
                   f" ({1000.0 * t:.1f} us)"
                   for l, (v, c, t) in enumerate(H32.gs_variants(NRHS))]
    breakdown = {f"L{l}/{c}": round(float(ms_tab[l, k] / reps * 1000.0), 2)
                 for l in range(ms_tab.shape[0]) for k, c in enumerate(g.KERNEL_CLASSES) if cnt_tab[l, k]}

    # the Vanka smoother (Section 5.1) on the same workload: FP32 and FP64 V-cycles
    vanka = None
    if not args.no_vanka and world == 1:
        V32 = g.Hierarchy(p, max_nrhs=NRHS, vcycle_fp32=1, smoother=1, pre=1, post=1)
        V64 = g.Hierarchy(p, max_nrhs=NRHS, smoother=1, pre=1, post=1)
        vsteps = max(2, args.steps // 2)
        msv32, sv32, _, itsv32, relv32, _ = timed(V32, vsteps, args.warmup)
        msv64, sv64, _, itsv64, _, _ = timed(V64, vsteps, args.warmup)
        V32.vcycle(b, x)
        vms, vcnt = V32.profile_vcycle(NRHS, reps=10)
        vi = g.KERNEL_CLASSES.index("vanka")
        l0_ms = vms[0, vi] / 10
        l0_bytes = 2 * vanka_bytes(V32, 0, NRHS, 4)  # V(1,1): two steps per cycle on level 0
        vanka = {"workload": "same 256x256 lid cavity, 8 rhs, Vanka(1,1), omega 0.5, FGMRES to 1e-8",
                 "value": sv32 / (msv32 / 1000.0), "unit": "solves/s", "fp64_vcycle_value": sv64 / (msv64 / 1000.0),
                 "iterations": itsv32.tolist(), "iterations_fp64": itsv64.tolist(),
                 "relres_max": float(np.max(relv32)),
                 "vcycle_us_by_kernel": {f"L{l}/{c}": round(float(vms[l, k] / 10 * 1000.0), 2)
                                         for l in range(vms.shape[0]) for k, c in enumerate(g.KERNEL_CLASSES)
                                         if vcnt[l, k]},
                 "level0_step_GBs": l0_bytes / (l0_ms / 1000.0) / 1e9,
                 "level0_step_frac": l0_bytes / (l0_ms / 1000.0) / 1e9 / measured_peaks()[0]}
        del V32, V64

    # the ILU(1) smoother (Section 5) on the same workload, FP64 V-cycle, FGMRES to the
    # paper's 1e-6 (Table 1 reports 17 iterations at this size)
    ilu = None
    if not args.no_ilu and world == 1:
        I64 = g.Hierarchy(p, max_nrhs=NRHS, smoother=2, pre=1, post=1)
        isteps = 3

        def itimed(H, steps, warm):
            for _ in range(warm):
                st, its, rel = H.fgmres(b, x, rtol=1e-6, restart=RESTART, maxit=MAXIT)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                st, its, rel = H.fgmres(b, x, rtol=1e-6, restart=RESTART, maxit=MAXIT)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1), st, its, rel

        msi, sti, itsi, reli = itimed(I64, isteps, 3)
        I64.vcycle(b, x)
        ims, icnt = I64.profile_vcycle(NRHS, reps=3)
        ii = g.KERNEL_CLASSES.index("ilu")
        F0 = I64.level_ilu(0)
        sub_us = float(ims[0, ii] / icnt[0, ii] * 1000.0)
        step_bytes = (ilu_bytes(I64, 0, NRHS, 8, True) + ilu_bytes(I64, 0, NRHS, 8, False)) / 2
        ilu = {"workload": "same 256x256 lid cavity, 8 rhs, ILU(1)(1,1), natural order, FP64 V-cycle, "
                           "FGMRES to 1e-6 (the paper's tolerance)",
               "value": NRHS * isteps / (msi / 1000.0), "unit": "solves/s", "status": int(sti),
               "iterations": itsi.tolist(), "relres_max": float(np.max(reli)), "paper_iterations": 17,
               "vcycle_us_by_kernel": {f"L{l}/{c}": round(float(ims[l, k] / 3 * 1000.0), 2)
                                       for l in range(ims.shape[0]) for k, c in enumerate(g.KERNEL_CLASSES)
                                       if icnt[l, k]},
               "level0": {"rows": len(F0["perm"]), "factor_nnz": len(F0["lower"][1]) + len(F0["upper"][1]),
                          "depth": F0["depth_lower"], "substitution_us": sub_us,
                          "us_per_dependency_level": sub_us / F0["depth_lower"],
                          "step_GBs": step_bytes / (2 * sub_us * 1e-6) / 1e9,
                          "bound": "latency: depth x one L2 round trip per dependency level"}}
        del I64

    picard = None
    if not args.no_picard and world == 1:
        picard = picard_line(g, torch)

    setup = None
    if not args.no_setup and world == 1:
        setup = setup_line(g, torch, p)

    serving = None
    if not args.no_serve:
        serving = serve(g, torch, dev, args.serve_requests, seed=rank, max_active=args.serve_active,
                        merge_k=args.serve_merge)
        if world > 1:
            wall, reqs = replica_aggregate(dist, dev, serving["wall_s"], serving["requests"])
            _, rhs = replica_aggregate(dist, dev, serving["wall_s"], serving["rhs_solves"])
            serving["all_ranks"] = {"requests_per_s": reqs / wall, "solves_per_s": rhs / wall}

    configs = None
    if not args.no_configs and world == 1:
        del H64
        torch.cuda.empty_cache()
        configs = config_records(g, torch, reps=2)

    if rank == 0:
        lat_sorted = sorted(lat32)
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycle / f64 FGMRES", "data": "synthetic",
                "config": {"workload": WORKLOAD, "nrhs_per_launch": NRHS, "restart": RESTART,
                           "l2": "inputs larger than L2 (hierarchy + Krylov basis > 1 GB)",
                           "parallelism": f"weak: {world} independent batch(es), one per GPU"},
                "fp64_vcycle": {"value": value64, "unit": "solves/s", "ms_per_step": ms64 / args.steps,
                                "iterations": its64.tolist(), "gpu_launches": launches64},
                "iterations": its32.tolist(), "relres_max": float(np.max(rel32)),
                "step_latency_ms": {"p50": 1000 * lat_sorted[len(lat_sorted) // 2],
                                    "p99": 1000 * lat_sorted[min(len(lat_sorted) - 1, int(0.99 * len(lat_sorted)))]},
                "latency_ms": (None if serving is None else
                               {"p50": serving["latency_ms"]["p50"], "p99": serving["latency_ms"]["p99"],
                                "source": "serving stream (arrival to result on the host)"}),
                "serving": serving, "accuracy": accuracy, "vanka": vanka, "ilu": ilu, "picard": picard,
                "setup": setup, "configs": configs,
                "e2e": e2e, "gpu_launches": launches32, "clocks": clocks, "roofline": roofline,
                "arnoldi_roofline": arnoldi,
                "vcycle_us_by_kernel": breakdown, "gs_variants": gs_variants,
                "row_shapes": {f"L{l}": "".join(str(v) for v in d.values()) for l, d in H32.row_shapes(NRHS).items()},
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
