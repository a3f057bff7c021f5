"""Benchmark: FP64 Stokes-operator applies on the radial-jump shell (lateral level 7, 129 radial layers).

One step = one apply each of A, B, B^T and diag(A) (the operator applications of the
hot path) on 63.4 M velocity DoFs + 2.66 M pressure DoFs.  value = DoFs processed per
second, summed over the four operators (A, diag: velocity DoFs; B, B^T: velocity +
pressure DoFs), whole job over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: independent replicas, one per rank (the apply does not shard without a
halo exchange; no collective on the data path), scaling "weak".
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

R_IN, R_OUT = 0.55, 1.0


def measured_hbm_gbs():
    """Copy bandwidth of the GB300s (MEASURED_PEAKS.json beside this file), else the
    earlier measurement 6771.8 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6771.8


HBM_GBS = measured_hbm_gbs()
LAW = dict(E=math.log(1e3), jump_r=0.9, jump_factor=30.0)  # x30 below r = 0.9, contrast 1e3
# Algorithmic FP64 work of one A apply per hexahedral cell (2 wedges, one-point rule), FMA = 2
# flops: the differences-only gather, the factorised Jacobian, strain, stress, the stress times
# the inverse Jacobian and the differences-only scatter of Eq. epsq / Eq. localapply, counted
# from their structure at 240 flops per wedge.
A_FLOPS_PER_CELL = 480.0
# ncu figures of the A tile kernel with the packed double-float element op (level 6, 65 layers,
# 2,621,440 cells, one launch): DRAM bytes (126.14 MB read + 49.46 MB written) and issued warp
# instructions (262,034,000) per cell, scaled to the bench size by cells; None once the kernel
# changes.
A_TRAFFIC_BYTES_PER_CELL = (126.14e6 + 49.46e6) / 2621440
A_WARP_INST_PER_CELL = 262034000 / 2621440
# Issue rate derived from unit counts: 152 SMs x 4 schedulers x 1 warp instruction per clock.
ISSUE_SLOTS_PER_CLOCK = 152 * 4
# Hourglass-control coefficient of the solves and the serving stream that use it.
HG_KAPPA = 0.3
# Kernel launches of one A + B + B^T + diag step: A 2 (tile, interface), B 4 (tile, interface,
# restriction, interface), B^T 3 (prolongation, tile, interface), diag 3 (tile, boundary-layer
# gather, interface); FP64 levels with N >= 32 add one tile-line pass to each of the four tile
# kernels.
def launches_per_step(level):
    return 12 + (4 if level >= 5 else 0)
# FP64 peak derived from unit counts and clocks: 152 SMs x 2 DFMA / clk x 2 flops x 2.07 GHz;
# the roofline uses the DFMA rate measured live by tn_probe_fma_peak, this figure is context.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--level", type=int, default=7)
    ap.add_argument("--n_r", type=int, default=129)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-solve", dest="no_solve", action="store_true",
                    help="do not run the Stokes-solve and serving measurements after the operator steps")
    ap.add_argument("--serve-requests", dest="serve_requests", type=int, default=256,
                    help="requests of the seeded serving stream measured after the solves (the full stream is 256)")
    ap.add_argument("--e2e-steps", dest="e2e_steps", type=int, default=50,
                    help="steps of the end-to-end run through tn_operator_steps_host")
    ap.add_argument("--convection", action="store_true",
                    help="instead of the operator step: the coupled Stokes-energy run of the largest single-GPU "
                         "shell (--level/--n_r, default level 8, 257 layers; --conv-steps steps)")
    ap.add_argument("--conv-steps", dest="conv_steps", type=int, default=10)
    ap.add_argument("--largest-shell", dest="largest_shell", action="store_true",
                    help="instead of the operator step: one Stokes solve on the largest single-GPU shell "
                         "(level 8, 257 layers) and its resident device memory")
    return ap.parse_args()


def dof_counts(level, n_r):
    nv = 3 * (10 * 4 ** level + 2) * n_r
    npr = (10 * 4 ** (level - 1) + 2) * ((n_r - 1) // 2 + 1)
    return nv, npr, 4 * nv + 2 * npr  # A + diag: nv each; B, B^T: nv + np each


def workload_name(level, n_r):
    return f"radial-jump shell l={level} (N={2 ** level}), {n_r} radial layers, FP64 A+B+BT+diag apply"


# ---------------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.path = index, None, None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 7]
        os.unlink(self.path)
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[4 + i] and "Not" not in r[4 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------- oracle arm
def _oracle_sample_setup(level, n_r, layers, seed, frac=1.0, first_cell=0):
    """Inputs of one oracle sample: the wedges of the first ``frac`` of the lateral triangles
    (diamond-major order) in ``layers`` radial cells of the same shell starting at radial cell
    ``first_cell`` (same lateral resolution and radial spacing).  B (CSR) is assembled here, outside
    the timed region."""
    from oracle import operators as O
    from oracle.fields import viscosity
    from oracle.mesh import ShellMesh
    from paper_2609_21633_gb300 import inputs
    dr = (R_OUT - R_IN) / (n_r - 1)
    om = ShellMesh(level, layers + 1, R_IN + dr * first_cell, R_IN + dr * (first_cell + layers))
    T = inputs.temperature(om.node_xyz(), R_IN, R_OUT) + inputs.normal(om.n_nodes, seed + 7, 0.01)
    eta = viscosity(om, T, LAW["E"], jump_r=LAW["jump_r"], jump_factor=LAW["jump_factor"])
    P = O.boundary_projectors(om)
    u = inputs.normal((3, om.n_nodes), seed + 8)
    pm = O.pressure_mesh(om)
    p = inputs.normal(pm.n_nodes, seed + 9)
    Pm = O.projector_matrix(P)
    wedges = np.arange(max(1, int(round(frac * om.n_wedges))))
    B = O.assemble_B(om, O.prolongation(om, pm), wedges=wedges)
    share = len(wedges) / om.n_wedges
    return dict(om=om, eta=eta, P=P, u=u, p=p, Pm=Pm, B=B, wedges=wedges,
                dofs=share * (4 * 3 * om.n_nodes + 2 * pm.n_nodes), share=share)


def _oracle_sample_run(c):
    """The timed part: matrix-free A, the B and B^T products, and diag(A) of the sample."""
    from oracle import operators as O
    O.apply_A_constrained(c["om"], c["eta"], c["u"], c["P"], wedges=c["wedges"])
    c["B"] @ (c["Pm"] @ c["u"].ravel())
    c["Pm"] @ (c["B"].T @ c["p"])
    O.diag_A_constrained(c["om"], c["eta"], c["P"], wedges=c["wedges"])


def oracle_step_sample(level, n_r, layers, seed, frac=1.0):
    """Time the CPU oracle, single-threaded, on a bounded sample of the workload (the innermost
    ``layers`` radial cells).  Returns (seconds, DoFs processed, description)."""
    c = _oracle_sample_setup(level, n_r, layers, seed, frac)
    t0 = time.perf_counter()
    _oracle_sample_run(c)
    dt = time.perf_counter() - t0
    desc = (f"{len(c['wedges']) // 2} of {10 * 4 ** level * (n_r - 1)} cells (innermost {layers} radial cells, "
            f"{100 * c['share']:.0f}% of their wedges) of the same shell, one A+B+BT+diag step (B assembled "
            f"before the timed region), numpy/scipy, 1 thread")
    return dt, c["dofs"], desc


def _oracle_worker(level, n_r, layers, seed, first_cell, barrier, out):
    c = _oracle_sample_setup(level, n_r, layers, seed, 1.0, first_cell)
    barrier.wait()
    t0 = time.monotonic()
    _oracle_sample_run(c)
    out.put((t0, time.monotonic(), c["dofs"]))


def oracle_step_sample_parallel(level, n_r, layers, seed, procs):
    """The oracle on all host cores: ``procs`` spawned processes, each the single-threaded sample
    on its own ``layers`` radial cells (worker w starts at radial cell w * layers), started together
    after their set-up.  Returns (wall seconds, DoFs processed, description)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    procs = max(1, min(procs, (n_r - 1) // layers))
    barrier, out = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(level, n_r, layers, seed, w * layers, barrier, out))
          for w in range(procs)]
    for p in ps:
        p.start()
    res = [out.get() for _ in ps]
    for p in ps:
        p.join()
    wall = max(r[1] for r in res) - min(r[0] for r in res)
    desc = (f"{procs * layers * 10 * 4 ** level} of {10 * 4 ** level * (n_r - 1)} cells (radial cells "
            f"0..{procs * layers - 1}, {layers} per process) of the same shell, one A+B+BT+diag step, "
            f"numpy/scipy, {procs} spawned processes of 1 thread each")
    return wall, sum(r[2] for r in res), desc


def oracle_config0_solve():
    """The oracle's FP64 Stokes solve of the level-4 / 17-layer shell (T of degree 3 / order 2,
    viscosity contrast 10, Ra = 7e3, free-slip) to 1e-8: flexible GMRES with the oracle V-cycle,
    single-threaded.  Returns (seconds, iterations, oracle-evaluated residual)."""
    from oracle.fields import viscosity
    from oracle.mesh import ShellMesh
    from oracle.solver import StokesSystem
    from paper_2609_21633_gb300 import inputs
    t0 = time.perf_counter()
    om = ShellMesh(4, 17, R_IN, R_OUT)
    T = inputs.temperature(om.node_xyz(), R_IN, R_OUT)
    eta = viscosity(om, T, math.log(10.0))
    S = StokesSystem(om, eta)
    b = S.rhs(T, 7e3)
    u, p, its = S.fgmres_solve(b, eta, tol=1e-8)
    dt = time.perf_counter() - t0
    return dt, its, S.residual(b, u, p)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    samples = []
    # size each step so that warm-up + timed steps take about two and a half minutes
    frac = min(1.0, 150.0 / 21.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_step_sample(args.level, args.n_r, 2, args.seed, frac)
    for _ in range(args.steps):
        dt, ndof, desc = oracle_step_sample(args.level, args.n_r, 2, args.seed, frac)
        samples.append((dt, ndof))
    tot_t = sum(s[0] for s in samples)
    value = sum(s[1] for s in samples) / tot_t / 1e9
    line = {
        "impl": "reference", "metric": "Stokes-apply GDoF/s (FP64 A+B+BT+diag step)", "value": value,
        "unit": "GDoF/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / len(samples), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.level, args.n_r), "sample": desc},
        "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------------------- ranks
def max_over_ranks(value, dist, device):
    """Largest value over all ranks (the slowest replica's time); the value itself without a
    process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_throughput(world, units_per_rank, seconds):
    """Whole-job throughput of `world` replicas that each processed `units_per_rank` units,
    timed by the slowest replica."""
    return world * units_per_rank / seconds


# ---------------------------------------------------------------------------------------- GPU arm
def layout_temperature(tn, m, noise_seed=None, noise_scale=0.01):
    """Prescribed temperature (degree 3, order 2, amplitude 0.01) at every layout node of level 0,
    plus optional seeded nodal noise that is identical on all copies of a node; 0 on padding."""
    from paper_2609_21633_gb300 import inputs
    info = tn.tn_mesh_info(m, 0)
    canon = tn.tn_mesh_canonical_index(m, 0)
    valid = canon >= 0
    pts = tn.tn_mesh_lateral_points(m, 0)
    N, P, n_r = info["N"], info["pitch"], info["n_r"]
    radii = R_IN + ((R_OUT - R_IN) * np.arange(n_r)) / (n_r - 1)
    lat = np.zeros((10, N + 1, P, 3))
    lat[:, :, : N + 1] = pts
    xyz = (radii[None, :, None, None, None] * lat[:, None]).reshape(-1, 3)
    T = np.zeros(info["n_layout"])
    T[valid] = inputs.temperature(xyz[valid], R_IN, R_OUT)
    if noise_seed is not None:
        noise = inputs.normal(info["n_layout"], noise_seed, noise_scale)
        T[valid] += noise[canon[valid]]
    return T


def solve_case(tn, torch, dev, level, n_r, E, Ra, mode, eta_storage=0, hg_kappa=0.0, quad=1):
    """One Stokes solve to 1e-8 (multigrid set-up excluded from the time).  Returns the stats and
    the solution (u, p) on the unique nodes, as host FP64 arrays."""
    m = tn.tn_mesh_create(level, n_r, R_IN, R_OUT, eta_storage=eta_storage, hg_kappa=hg_kappa,
                          radial_quad_points=quad)
    try:
        info, pinfo = tn.tn_mesh_info(m, 0), tn.tn_mesh_info(m, 1)
        Td = torch.tensor(layout_temperature(tn, m), device=dev)
        tn.tn_set_temperature(m, Td, E)
        f = [torch.zeros(info["n_layout"], device=dev, dtype=torch.float64) for _ in range(3)]
        tn.tn_buoyancy(m, Td, Ra, f)
        u = [torch.zeros_like(f[0]) for _ in range(3)]
        p = torch.zeros(pinfo["n_layout"], device=dev, dtype=torch.float64)
        tn.tn_mg_setup(m, torch.float64 if mode == tn.TN_SOLVE_F64 else torch.float32)
        torch.cuda.synchronize()
        st = tn.tn_stokes_solve(m, f, None, u, p, tn.tn_solve_default_opts(mode=mode), check=False)
        nv = 3 * info["n_unique_nodes"]
        npr = pinfo["n_unique_nodes"]
        cu, cp = tn.tn_mesh_canonical_index(m, 0), tn.tn_mesh_canonical_index(m, 1)
        ku, kp = cu == np.arange(cu.size), cp == np.arange(cp.size)
        sol = (np.stack([t.cpu().numpy()[ku] for t in u]), p.cpu().numpy()[kp])
        return {"iterations": st["iterations"], "refinements": st["refinements"], "seconds": st["seconds"],
                "rel_residual": st["rel_residual"], "converged": bool(st["converged"]), "dofs": nv + npr}, sol
    finally:
        tn.tn_mesh_destroy(m)


def serving_stream(tn, n_req=256, seed=0, load=0.7, hg_kappa=0.3, eta_storage=1, mode=None, repeated=False,
                   max_batch=1):
    """Serving workload: seeded Stokes requests (lateral level U{3..6}, radial layers U{9,17,33,65},
    viscosity contrast log-uniform in [1, 1e4], temperature perturbation degree U{2..8}, order
    U{0..l}, amplitude U[0.01, 0.05], Ra = 7e3), solved to 1e-8 by FP64 FGMRES with the FP32
    preconditioner (mode, default TN_SOLVE_F64_PREC32), hourglass control kappa = hg_kappa,
    FP32-path viscosity storage eta_storage (1 = BF16).
    Phase 1 submits all requests at once (saturated throughput); phase 2 submits them with
    Poisson arrivals at `load` x the saturated rate and reports latency percentiles.
    repeated: shapes from four only (lateral level U{4, 5}, radial layers U{17, 33}), the stream on
    which same-shape requests meet; max_batch: the server's lockstep batch size."""
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(n_req):
        l = int(rng.integers(4, 6)) if repeated else int(rng.integers(3, 7))
        nr = int(rng.choice([17, 33])) if repeated else int(rng.choice([9, 17, 33, 65]))
        contrast = 10.0 ** rng.uniform(0.0, 4.0)
        deg = int(rng.integers(2, 9))
        order = int(rng.integers(0, deg + 1))
        amp = float(rng.uniform(0.01, 0.05))
        reqs.append(dict(lateral_level=l, radial_layers=nr, E=math.log(contrast), Ra=7e3, t_degree=deg,
                         t_order=order, t_amplitude=amp))
    mode = tn.TN_SOLVE_F64_PREC32 if mode is None else mode
    srv = tn.tn_server_create(tn.tn_server_default_opts(max_active=4, hg_kappa=hg_kappa, eta_storage=eta_storage,
                                                        mode=mode, max_batch=max_batch))
    try:
        tickets = [tn.tn_server_submit(srv, **q) for q in reqs]
        res = [tn.tn_server_wait(srv, t) for t in tickets]
        t_first = min(r["t_submit"] for r in res)
        sat = n_req / (max(r["t_end"] for r in res) - t_first)
        ok_sat = sum(1 for r in res if r["status"] == tn.TN_OK)
        rate = load * sat
        gaps = rng.exponential(1.0 / rate, size=n_req)
        due = np.cumsum(gaps)
        t0 = time.perf_counter()
        tickets = []
        for q, d in zip(reqs, due):
            wait = d - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            tickets.append(tn.tn_server_submit(srv, **q))
        res = [tn.tn_server_wait(srv, t) for t in tickets]
        lat = np.array([r["t_end"] - r["t_submit"] for r in res])
        span = max(r["t_end"] for r in res) - min(r["t_submit"] for r in res)
        ok = sum(1 for r in res if r["status"] == tn.TN_OK)
        its = [r["iterations"] for r in res]
        batched = [r["batch"] for r in res]
        return {"requests": n_req, "stream": ("seeded %d-request stream of four shapes (level 4-5, 17 or 33 layers)"
                                              % n_req) if repeated else "first %d of the seeded 256-request stream" % n_req,
                "max_batch": max_batch, "mean_batch": float(np.mean([b if b > 0 else 1 for b in batched])),
                "saturated_solves_per_s": sat, "saturated_converged": ok_sat,
                "poisson_rate_per_s": rate, "solves_per_s": n_req / span, "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "converged": ok,
                "max_rel_residual": max(r["rel_residual"] for r in res), "median_iterations": float(np.median(its)),
                "max_active": 4,
                "mode": {0: "FP64", 1: "FP32 inner + FP64 refinement", 2: "FP64 FGMRES + FP32 preconditioner"}[mode]
                + ", rtol 1e-8",
                "hg_kappa": hg_kappa, "eta_storage": ["f32", "bf16", "f16"][eta_storage]}
    finally:
        tn.tn_server_destroy(srv)


def largest_shell(tn, torch, repeats=2):
    """Largest single-GPU coupled-run shell: lateral level 8 (257 x 257 nodes per diamond), 257
    radial layers (505 M velocity DoFs), Ra = 1e5, temperature viscosity contrast 1e2, free-slip;
    one mixed-precision Stokes solve to 1e-8 (FP32 inner FGMRES(30) / V-cycle, FP64 refinement,
    hourglass control kappa = 0.3, BF16 viscosity), through the serving API, which builds the
    temperature field on the device.  Reports each request's time (mesh creation, set-up and
    solve; the second request reuses the resident hierarchy) and the device memory it holds."""
    free0, total = torch.cuda.mem_get_info()
    srv = tn.tn_server_create(tn.tn_server_default_opts(max_active=1, memory_fraction=0.95, hg_kappa=HG_KAPPA,
                                                        eta_storage=tn.TN_ETA_BF16))
    out = {"workload": "icosahedral shell l=8 (N=256), 257 radial layers, Ra=1e5, viscosity contrast 1e2",
           "velocity_dofs": dof_counts(8, 257)[0], "pressure_dofs": dof_counts(8, 257)[1],
           "device_memory_gb": total / 1e9, "runs": []}
    try:
        for _ in range(repeats):
            t = tn.tn_server_submit(srv, 8, 257, math.log(100.0), 1e5, 3, 2, 0.01)
            r = tn.tn_server_wait(srv, t)
            free1, _ = torch.cuda.mem_get_info()
            out["runs"].append({"status": r["status"], "iterations": r["iterations"], "refinements": r["refinements"],
                                "rel_residual": r["rel_residual"], "seconds": r["t_end"] - r["t_start"],
                                "resident_gb": (free0 - free1) / 1e9})
    finally:
        tn.tn_server_destroy(srv)
    return out


def convection_run(tn, torch, level, n_r, steps):
    """Coupled run (Eq. energy with the Stokes solve each step): Ra = 1e5, viscosity contrast 1e2
    (exp(ln 100 (1/2 - T))), free-slip, T = conductive profile + 0.01 cos(2 phi) P_3^2 perturbation,
    surfaces held at 1 and 0; Stokes in FP32 inner solves with FP64 refinement to 1e-8, hourglass
    control kappa = 0.3 and BF16 viscosity; energy by explicit SUPG / Heun substeps at CFL 0.5.
    Reports every step (Nu_top, V_rms, dt, substeps, solve iterations, times) and device memory."""
    free0, total = torch.cuda.mem_get_info()
    t0 = time.perf_counter()
    m = tn.tn_mesh_create(level, n_r, R_IN, R_OUT, hg_kappa=HG_KAPPA, eta_storage=tn.TN_ETA_BF16)
    try:
        info, pinfo = tn.tn_mesh_info(m, 0), tn.tn_mesh_info(m, 1)
        T = torch.tensor(layout_temperature(tn, m), device="cuda")
        u = [torch.zeros(info["n_layout"], device="cuda", dtype=torch.float64) for _ in range(3)]
        p = torch.zeros(pinfo["n_layout"], device="cuda", dtype=torch.float64)
        opts = tn.tn_convection_default_opts(Ra=1e5, E=math.log(100.0), mode=tn.TN_SOLVE_MIXED)
        stats = tn.tn_convection_steps(m, T, u, p, steps, opts, check=False)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        return {"workload": f"coupled Stokes-energy run, shell l={level} (N={2 ** level}), {n_r} radial layers, "
                            "Ra=1e5, viscosity contrast 1e2", "velocity_dofs": dof_counts(level, n_r)[0],
                "pressure_dofs": dof_counts(level, n_r)[1], "temperature_dofs": (10 * 4 ** level + 2) * n_r,
                "steps": stats, "seconds_total": time.perf_counter() - t0,
                "resident_gb": (free0 - free1) / 1e9, "device_memory_gb": total / 1e9,
                "stokes": "FP32 inner FGMRES / V-cycle, FP64 refinement to 1e-8, kappa 0.3, BF16 viscosity",
                "energy": "one-point W1 SUPG residual, lumped mass, Heun substeps, CFL 0.5"}
    finally:
        tn.tn_mesh_destroy(m)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.convection:
        import torch
        import paper_2609_21633_gb300 as tn
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        level = args.level if args.level != 7 else 8
        n_r = args.n_r if args.n_r != 129 else 257
        print(json.dumps(convection_run(tn, torch, level, n_r, args.conv_steps)))
        return 0
    if args.largest_shell:
        import torch
        import paper_2609_21633_gb300 as tn
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(largest_shell(tn, torch)))
        return 0
    import torch
    import paper_2609_21633_gb300 as tn
    from paper_2609_21633_gb300 import inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream()

    m = tn.tn_mesh_create(args.level, args.n_r, R_IN, R_OUT)
    info, pinfo = tn.tn_mesh_info(m, 0), tn.tn_mesh_info(m, 1)
    n = info["n_layout"]
    canon = torch.from_numpy(tn.tn_mesh_canonical_index(m, 0))
    Td = torch.tensor(layout_temperature(tn, m, args.seed + 100 * rank), device=dev)
    tn.tn_set_temperature(m, Td, LAW["E"], LAW["jump_r"], LAW["jump_factor"])

    def field(seed, size, can=None):
        v = inputs.normal(size, seed)
        if can is not None:
            v = np.where(can >= 0, v[np.maximum(can, 0)], 0.0)
        return torch.tensor(v, device=dev)

    pcanon = tn.tn_mesh_canonical_index(m, 1)
    u = [field(args.seed + 10 * rank + c, n, canon.numpy()) for c in range(3)]
    p = field(args.seed + 10 * rank + 5, pinfo["n_layout"], pcanon)
    yA = [torch.empty(n, device=dev, dtype=torch.float64) for _ in range(3)]
    yBT = [torch.empty(n, device=dev, dtype=torch.float64) for _ in range(3)]
    dA = [torch.empty(n, device=dev, dtype=torch.float64) for _ in range(3)]
    q = torch.empty(pinfo["n_layout"], device=dev, dtype=torch.float64)

    def timed_steps(uu, pp, yy, qq, bb, dd, steps, warmup, sample_clocks):
        """Warm-up, then `steps` timed steps; returns (ms total, per-op mean ms, clocks)."""
        ev = {k: [] for k in ("A", "B", "BT", "diag")}

        def step(record):
            for name, fn in (("A", lambda: tn.tn_apply_A(m, 0, uu, yy, st)),
                             ("B", lambda: tn.tn_apply_B(m, 0, uu, qq, st)),
                             ("BT", lambda: tn.tn_apply_BT(m, 0, pp, bb, st)),
                             ("diag", lambda: tn.tn_diag_A(m, 0, dd, st))):
                if record:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    fn()
                    e1.record(st)
                    ev[name].append((e0, e1))
                else:
                    fn()

        for _ in range(warmup):
            step(False)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clocks = ClockSampler(local)
        if sample_clocks:
            clocks.start()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(st)
        for _ in range(steps):
            step(True)
        t1.record(st)
        torch.cuda.synchronize()
        clk = clocks.stop() if sample_clocks else None
        per = {k: sum(a.elapsed_time(b) for a, b in v) / len(v) for k, v in ev.items()}
        return t0.elapsed_time(t1), per, clk, step

    ms, per_op, clk, step = timed_steps(u, p, yA, q, yBT, dA, args.steps, max(3, args.warmup), True)
    ms = max_over_ranks(ms, dist, dev)
    if dist:
        dist.barrier()
    # the A apply with the element op in IEEE binary64 (the default evaluates it in double-float
    # on the FP32 pipe): same shell, temperature and input, timed alone
    m64 = tn.tn_mesh_create(args.level, args.n_r, R_IN, R_OUT, fp64_element=tn.TN_FP64_ELEM_BINARY64)
    tn.tn_set_temperature(m64, Td, LAW["E"], LAW["jump_r"], LAW["jump_factor"])
    for _ in range(3):
        tn.tn_apply_A(m64, 0, u, yA, st)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    b0.record(st)
    for _ in range(args.steps):
        tn.tn_apply_A(m64, 0, u, yA, st)
    b1.record(st)
    torch.cuda.synchronize()
    a_binary64_ms = b0.elapsed_time(b1) / args.steps
    tn.tn_mesh_destroy(m64)
    # the same step in FP32 (the inner-solve precision of the mixed path)
    u32 = [t.float() for t in u]
    p32, q32 = p.float(), q.float()
    yA32, yBT32, dA32 = [[t.float() for t in v] for v in (yA, yBT, dA)]
    ms32, per32, _, _ = timed_steps(u32, p32, yA32, q32, yBT32, dA32, args.steps, max(3, args.warmup), False)
    del u32, p32, q32, yA32, yBT32, dA32

    nv, npr, ndof = dof_counts(args.level, args.n_r)
    value = job_throughput(world, ndof * args.steps, ms / 1e3) / 1e9

    # ---- end to end through the C ABI with host buffers: every step copies its inputs from pinned
    # host memory, runs A, B, B^T and diag(A), and copies all ten outputs back (the library
    # pipelines the copies of neighbouring steps with the compute)
    hu = [t.cpu().pin_memory() for t in u]
    hp = p.cpu().pin_memory()
    outs = yA + [q] + yBT + dA
    # two pinned output sets, alternated step by step (no two steps of one call write the same
    # host buffer, as the entry point requires)
    hout = [[torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in outs] for _ in range(2)]
    h2d = sum(t.numel() * t.element_size() for t in hu) + hp.numel() * hp.element_size()
    d2h = sum(t.numel() * t.element_size() for t in hout[0])

    def e2e_steps_run(k):
        tn.tn_operator_steps_host(m, [hu] * k, [hp] * k, [hout[i % 2] for i in range(k)], stream=st)

    e2e_steps = max(2, args.e2e_steps)
    e2e_steps_run(2)  # allocates the library's device buffer sets
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(st)
    e2e_steps_run(e2e_steps)
    c1.record(st)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(c0.elapsed_time(c1), dist, dev)
    e2e_value = job_throughput(world, ndof * e2e_steps, e2e_ms / 1e3) / 1e9

    if rank == 0:
        cells = 10 * 4 ** args.level * (args.n_r - 1)
        a_flops = A_FLOPS_PER_CELL * cells
        achieved = a_flops / (per_op["A"] / 1e3) / 1e12
        dfma_peak = tn.tn_probe_fma_peak(torch.float64, st)  # measured live, same clocks as the step
        ffma_peak = tn.tn_probe_fma_peak(torch.float32, st)
        sm_hz = 1e6 * ((clk or {}).get("sm_mhz") or 2070.0)
        issue_peak = ISSUE_SLOTS_PER_CLOCK * sm_hz / 1e12
        issue_achieved = A_WARP_INST_PER_CELL * cells / (per_op["A"] / 1e3) / 1e12
        line = {
            "metric": "Stokes-apply GDoF/s (FP64 A+B+BT+diag step)", "value": value, "unit": "GDoF/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.level, args.n_r), "velocity_dofs": nv, "pressure_dofs": npr,
                       "dofs_per_step": ndof, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (3 x %.0f MB velocity components)" % (n * 8 / 1e6)},
            "per_op_ms": per_op,
            "A_ms_binary64_element": a_binary64_ms,
            "roofline": {"bound": "alu", "kernel": "A apply, double-float element op (tile kernel + tile-line "
                                                  "and interface passes)",
                         "achieved": issue_achieved, "peak": issue_peak, "unit": "Twarp-inst/s (issue)",
                         "frac": issue_achieved / issue_peak,
                         "traffic": A_TRAFFIC_BYTES_PER_CELL * cells if A_TRAFFIC_BYTES_PER_CELL else None,
                         "warp_inst_per_cell": A_WARP_INST_PER_CELL,
                         "peak_note": "instruction issue, 152 SMs x 4 schedulers x 1 warp instruction/clk at the "
                                      "median SM clock under load; instructions per cell from ncu (level 6 / 65)",
                         "fp64_equiv_tflops": achieved, "flops_per_cell": A_FLOPS_PER_CELL,
                         "fp64_equiv_over_dfma_peak": achieved / dfma_peak, "dfma_peak_tflops": dfma_peak,
                         "dfma_peak_derived_tflops": FP64_PEAK_TFLOPS, "ffma_peak_tflops": ffma_peak,
                         "binary64_element": {"A_ms": a_binary64_ms,
                                              "tflops": A_FLOPS_PER_CELL * cells / (a_binary64_ms / 1e3) / 1e12,
                                              "frac_of_dfma_peak": A_FLOPS_PER_CELL * cells / (a_binary64_ms / 1e3)
                                              / 1e12 / dfma_peak},
                         "hbm_frac_of_measured": (64.0 * cells) / (per_op["A"] / 1e3) / HBM_GBS / 1e9},
            "f32_step": {"ms_per_step": ms32 / args.steps, "per_op_ms": per32,
                         "value": ndof / (ms32 / args.steps / 1e3) / 1e9, "unit": "GDoF/s",
                         "A_hbm_frac_of_measured": (32.0 * cells) / (per32["A"] / 1e3) / HBM_GBS / 1e9},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": "GDoF/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "gpu_launches": launches_per_step(args.level) * args.steps,
        }
        if world == 1 and not args.no_solve:
            # Stokes solves to 1e-8: FP64 against FP32 inner solves with FP64 refinement
            solves = {}
            for name, lvl, nr, E in (("l4_17_contrast1e1", 4, 17, math.log(10.0)),
                                     ("l6_65_contrast1e4", 6, 65, math.log(1e4))):
                r64, s64 = solve_case(tn, torch, dev, lvl, nr, E, 7e3, tn.TN_SOLVE_F64)
                rmx, smx = solve_case(tn, torch, dev, lvl, nr, E, 7e3, tn.TN_SOLVE_MIXED)
                rbf, sbf = solve_case(tn, torch, dev, lvl, nr, E, 7e3, tn.TN_SOLVE_MIXED, eta_storage=tn.TN_ETA_BF16)
                for r, sx in ((rmx, smx), (rbf, sbf)):  # solution difference against the FP64 solve
                    r["u_rel_diff_vs_fp64"] = float(np.linalg.norm(sx[0] - s64[0]) / np.linalg.norm(s64[0]))
                    r["p_rel_diff_vs_fp64"] = float(np.linalg.norm(sx[1] - s64[1]) / np.linalg.norm(s64[1]))
                # the hourglass-controlled system (Eq. hgstab, kappa = 0.3): FP64 and mixed
                h64, t64 = solve_case(tn, torch, dev, lvl, nr, E, 7e3, tn.TN_SOLVE_F64, hg_kappa=HG_KAPPA)
                hbf, tbf = solve_case(tn, torch, dev, lvl, nr, E, 7e3, tn.TN_SOLVE_MIXED, eta_storage=tn.TN_ETA_BF16,
                                      hg_kappa=HG_KAPPA)
                hbf["u_rel_diff_vs_fp64"] = float(np.linalg.norm(tbf[0] - t64[0]) / np.linalg.norm(t64[0]))
                # FP64 FGMRES with the FP32 preconditioner (BF16 viscosity in it)
                hpc, tpc = solve_case(tn, torch, dev, lvl, nr, E, 7e3, tn.TN_SOLVE_F64_PREC32,
                                      eta_storage=tn.TN_ETA_BF16, hg_kappa=HG_KAPPA)
                hpc["u_rel_diff_vs_fp64"] = float(np.linalg.norm(tpc[0] - t64[0]) / np.linalg.norm(t64[0]))
                hbf["p_rel_diff_vs_fp64"] = float(np.linalg.norm(tbf[1] - t64[1]) / np.linalg.norm(t64[1]))
                # discretisation change of the control: its FP64 solution against the plain one
                h64["u_rel_diff_vs_plain"] = float(np.linalg.norm(t64[0] - s64[0]) / np.linalg.norm(s64[0]))
                # the other remedy of Sec. 4: the second radial quadrature point, FP64 and FP64
                # FGMRES with the FP32 preconditioner (BF16 viscosity in it)
                q64, u64 = solve_case(tn, torch, dev, lvl, nr, E, 7e3, tn.TN_SOLVE_F64, quad=2)
                qpc, upc = solve_case(tn, torch, dev, lvl, nr, E, 7e3, tn.TN_SOLVE_F64_PREC32,
                                      eta_storage=tn.TN_ETA_BF16, quad=2)
                q64["u_rel_diff_vs_plain"] = float(np.linalg.norm(u64[0] - s64[0]) / np.linalg.norm(s64[0]))
                qpc["u_rel_diff_vs_fp64"] = float(np.linalg.norm(upc[0] - u64[0]) / np.linalg.norm(u64[0]))
                solves[name] = {"fp64": r64, "mixed": rmx, "mixed_bf16_eta": rbf,
                                "mixed_speedup": r64["seconds"] / rmx["seconds"],
                                "mixed_bf16_eta_speedup": r64["seconds"] / rbf["seconds"],
                                "hg%.1f_fp64" % HG_KAPPA: h64, "hg%.1f_mixed_bf16_eta" % HG_KAPPA: hbf,
                                "hg%.1f_fp64_prec32_bf16_eta" % HG_KAPPA: hpc,
                                "quad2_fp64": q64, "quad2_fp64_prec32_bf16_eta": qpc,
                                "hg_mixed_bf16_eta_speedup_vs_plain_fp64": r64["seconds"] / hbf["seconds"]}
            line["solves"] = solves
            if args.serve_requests > 0:
                line["serving"] = serving_stream(tn, args.serve_requests, args.seed, hg_kappa=HG_KAPPA)
                # a stream whose shapes repeat, without and with lockstep batching of same-shape requests
                line["serving_repeated_shapes"] = {
                    "max_batch_1": serving_stream(tn, 96, args.seed + 1, hg_kappa=HG_KAPPA, repeated=True, max_batch=1),
                    "max_batch_4": serving_stream(tn, 96, args.seed + 1, hg_kappa=HG_KAPPA, repeated=True, max_batch=4)}
        if world == 1:
            cores = os.cpu_count() or 1
            dtp, ndp, descp = oracle_step_sample_parallel(args.level, args.n_r, 2, args.seed, cores)
            dt, nd, desc = oracle_step_sample(args.level, args.n_r, 2, args.seed)
            line["cpu_baseline"] = {"value": ndp / dtp / 1e9, "unit": "GDoF/s", "cores": min(cores, (args.n_r - 1) // 2),
                                    "kind": "oracle", "sample": descp, "seconds": dtp,
                                    "single_core": {"value": nd / dt / 1e9, "unit": "GDoF/s", "cores": 1,
                                                    "sample": desc, "seconds": dt}}
            if not args.no_solve:
                ot, oits, ores = oracle_config0_solve()
                gpu0 = line["solves"]["l4_17_contrast1e1"]["fp64"]
                line["cpu_baseline"]["config0_solve"] = {
                    "oracle_seconds": ot, "oracle_iterations": oits, "oracle_rel_residual": ores, "cores": 1,
                    "gpu_fp64_seconds": gpu0["seconds"], "gpu_fp64_iterations": gpu0["iterations"],
                    "what": "level 4 / 17 layers, contrast 10, Ra 7e3, free-slip, to 1e-8: oracle flexible GMRES "
                            "with its V-cycle (set-up included) beside the GPU FP64 solve (set-up excluded)"}
        print(json.dumps(line))
    tn.tn_mesh_destroy(m)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
