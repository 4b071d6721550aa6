"""Throughput of the GB300 gas-kinetic scheme on the 2D decaying-turbulence workload.

Workload (one bench step): 1024 x 1024 cells on [0, 2 pi)^2, periodic; random-phase solenoidal
velocity with E(k) ~ k^4 exp(-2 (k/8)^2) at turbulent Mach 0.3, rho = 1, p = 1/gamma; k-epsilon
turbulent relaxation time from seeded log-normal k, epsilon fields; multi-dimensional expansion,
van Leer MUSCL; FP32 flux arithmetic with the state accumulated in IEEE double (FP32 bulk, FP64
accumulation); 200 CFL time steps (CFL 0.5) from the initial state.  Inputs are synthetic (seed
1302).  The same workload with the state kept as a float pair (about 48 bits) is timed the same way
and reported beside it (`float_pair_form`).

Metric: interface-flux evaluations per second (distinct faces: 2 per cell per time step on the
periodic 2D grid); cell updates per second are reported beside it.  The step kernel's time per
launch (roofline) is taken inside the timed region, from the end of the state copy-in to the end of
the last time step (the step kernels run in their captured graphs), divided by the steps.  `value` is timed with CUDA events on the library's stream with
the inputs resident in HBM; `e2e` through the same C ABI from pinned host buffers, host<->device
copies included.  The L2 cache is flushed (a 256 MiB write) between bench steps; within one bench
step the 200 time steps work on a state that fits in L2, as the algorithm allows.

`--impl reference` times the CPU oracle (the plain FP64 statement of the method) on the host cores on
a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "turb2d_1024_keps_multid_fp32_acc64"
N = 1024
NSTEPS = 200
CFL = 0.5
MU = 1e-5
SEED = 1302


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default=None, choices=["fp32", "fp32_acc64", "fp64"])
    p.add_argument("--workload", default="turb2d_1024",
                   choices=["turb2d_1024", "turb2d_512", "turb2d_1024_transport", "sod1d_400", "shock_bl_1024x384", "turb3d_256",
                            "turb3d_160", "shock_bl_512x192",
                            "corner2d_528x136", "corner2d_2112x544", "steady_corner_528x136",
                            "steady_corner_2112x544", "naca2d_608x160", "naca2d_608x160_transport",
                            "steady_naca_608x160", "steady_naca_608x160_transport"])
    p.add_argument("--expand", default=None, choices=["directional", "multid"],
                   help="expansion of the body-fitted and steady workloads (default: directional)")
    p.add_argument("--reconstruction", default="muscl2", choices=["muscl2", "muscl3", "weno5"],
                   help="face reconstruction (the default is the second-order MUSCL the metric is quoted on)")
    p.add_argument("--rarefaction", default="dt", choices=["dt", "tauhat"],
                   help="degree of rarefaction in the time coefficients: tau/dt (default) or tau/tauhat")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--lusgs-tile", type=int, default=16, choices=[16, 32],
                   help="LU-SGS tile edge of the steady workloads")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--serving", action="store_true", help="measure the serving form only")
    p.add_argument("--no-serving", action="store_true", help="leave the serving summary out")
    p.add_argument("--requests", type=int, default=4000)
    p.add_argument("--accuracy", action="store_true", help="report FP32-form errors against the oracle")
    p.add_argument("--profile", type=int, default=0, metavar="NSTEPS",
                   help="capture mode for ncu: set the workload's state and take NSTEPS time steps, untimed, "
                        "then exit (no warm-up, no bench line)")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, device=None):
    """Largest value of x over the ranks of the default process group (the job's wall time is the
    slowest rank's); each rank processes its own replica, so units add up across ranks."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def workload_inputs():
    from paper_1302_2132_gb300 import inputs
    return inputs.turbulence(N, 2, seed=SEED)


def make_workload(name, precision):
    """Workload descriptions: the default is the 2D decaying turbulence the metric is quoted on; the
    others are the remaining configurations, measured with the same timing rules."""
    from paper_1302_2132_gb300 import inputs
    if name == "turb2d_1024":
        spec = workload_inputs()
        return dict(spec=spec, kw=dict(gamma=1.4, mu=MU, turb_model="keps", C_mu=0.09, C_a=0.0, limiter="vanleer",
                                       expand="multid"), nsteps=NSTEPS, t_end=0.0,
                    precision=precision or "fp32_acc64",
                    desc="2D decaying turbulence 1024^2, k-epsilon tau_t, multi-D, 200 CFL steps, FP32 flux with "
                         "the state accumulated in IEEE double")
    if name == "turb2d_512":  # a smaller case of the same kernel for multi-pass captures
        spec = inputs.turbulence(512, 2, seed=SEED)
        return dict(spec=spec, kw=dict(gamma=1.4, mu=MU, turb_model="keps", C_mu=0.09, C_a=0.0, limiter="vanleer",
                                       expand="multid"), nsteps=NSTEPS, t_end=0.0,
                    precision=precision or "fp32_acc64",
                    desc="2D decaying turbulence 512^2, k-epsilon tau_t, multi-D, 200 CFL steps")
    if name == "turb2d_1024_transport":
        spec = dict(workload_inputs())
        # k-omega transport from the same initial fields: omega = eps / (C_mu k), so that nu_t = k/omega
        # equals the k-epsilon C_mu k^2/eps of the default workload at t = 0
        spec["f2"] = spec["f2"] / (0.09 * spec["f1"])
        return dict(spec=spec, kw=dict(gamma=1.4, mu=MU, turb_model="komega_transport", beta_star=0.09, C_a=0.0,
                                       limiter="vanleer", expand="multid"), nsteps=NSTEPS, t_end=0.0,
                    precision=precision or "fp32", transport=True,
                    desc="2D decaying turbulence 1024^2 with k and omega transported (Wilcox 2006 k-omega), "
                         "multi-D, 200 CFL steps")
    if name == "sod1d_400":
        spec = inputs.sod_1d(400)
        return dict(spec=spec, kw=dict(gamma=1.4, mu=1e-5, C_a=1.0, limiter="vanleer", expand="directional"),
                    nsteps=0, t_end=0.2, precision=precision or "fp64",
                    desc="Sod shock tube, 400 cells, van Leer, C_a = 1, CFL 0.5, to t = 0.2")
    if name.startswith("shock_bl_"):  # 1024x384: the workload; 512x192: a smaller case for kernel captures
        nx, ny = (int(v) for v in name.split("_")[2].split("x"))
        spec = inputs.shock_boundary_layer(nx, ny)
        return dict(spec=spec, kw=dict(gamma=1.4, mu=spec["mu"], T_wall=spec["T_wall"], turb_model="komega",
                                       beta_star=0.09, C_a=0.5, limiter="vanleer", expand="multid"),
                    nsteps=5000, t_end=0.0, precision=precision or "fp32_acc64",
                    desc="Mach 2.85 boundary layer under a 24-degree shock, %dx%d wall-clustered, k-omega tau_t, "
                         "5000 CFL steps, FP32 flux with the state accumulated in IEEE double" % (nx, ny))
    if name.startswith("steady_corner_"):
        nx, ny = (int(v) for v in name.split("_")[2].split("x"))
        spec = inputs.compression_corner(nx, ny, alpha_deg=24.0)
        return dict(spec=spec, steady=True, levels=4, precision=precision or "fp32",
                    schedule=[(20, 1.0), (80, 4.0)],
                    desc="steady solver (local time steps, LU-SGS on cell tiles, 4-level FAS multigrid) on the "
                         "Mach 2.85 / 24-degree compression corner, body-fitted %dx%d wall-clustered grid, k-omega "
                         "tau_t, 100 cycles from the inflow state (20 at CFL 1, 80 at CFL 4), flux windows CFL 0.5"
                         % (nx, ny))
    if name in ("naca2d_608x160", "naca2d_608x160_transport", "steady_naca_608x160",
                "steady_naca_608x160_transport"):
        # the fine NACA 0012 C-grid size of the paper's Table 2: 2 x 112 wake + 384 surface cells, 160 rows
        spec = inputs.naca0012_case(112, 384, 160, mach=0.8, alpha_deg=2.26, Re=9.0e6, dy1=2e-4, ratio=1.05,
                                    R=10.0, x_out=10.0)
        if name == "steady_naca_608x160_transport":
            return dict(spec=spec, steady=True, levels=4, precision=precision or "fp32", transport=True,
                        schedule=[(20, 1.0), (80, 4.0)],
                        desc="steady solver (local time steps, LU-SGS on cell tiles, 4-level FAS multigrid) with "
                             "k and omega transported (one diagonal-implicit steady k-omega update per cycle) on a "
                             "NACA 0012 C-grid 608x160 with a wake cut, M 0.8, incidence 2.26 degrees, Re 9e6, "
                             "from free-stream k and omega, 100 cycles (20 at CFL 1, 80 at CFL 4)")
        if name.startswith("steady_"):
            return dict(spec=spec, steady=True, levels=4, precision=precision or "fp32",
                        schedule=[(20, 1.0), (80, 4.0)],
                        desc="steady solver (local time steps, LU-SGS on cell tiles, 4-level FAS multigrid) on a "
                             "NACA 0012 C-grid 608x160 with a wake cut, M 0.8, incidence 2.26 degrees, Re 9e6, "
                             "k-omega tau_t from free-stream fields, 100 cycles (20 at CFL 1, 80 at CFL 4)")
        if name.endswith("_transport"):
            return dict(spec=spec, kw=dict(gamma=1.4, mu=spec["mu"], T_wall=spec["T_wall"],
                                           turb_model="komega_transport", beta_star=0.09, C_a=0.5, limiter="vanleer",
                                           expand="directional", wake_cut=spec["wake_cut"]),
                        nsteps=2000, t_end=0.0, precision=precision or "fp32", nodes=spec["nodes"], transport=True,
                        desc="NACA 0012 C-grid 608x160 with a wake cut, M 0.8, incidence 2.26 degrees, Re 9e6, "
                             "k and omega transported from free-stream values (Wilcox 2006 k-omega), directional "
                             "expansion in each face's frame, 2000 CFL steps")
        return dict(spec=spec, kw=dict(gamma=1.4, mu=spec["mu"], T_wall=spec["T_wall"], turb_model="komega",
                                       beta_star=0.09, C_a=0.5, limiter="vanleer", expand="directional",
                                       wake_cut=spec["wake_cut"]),
                    nsteps=2000, t_end=0.0, precision=precision or "fp32", nodes=spec["nodes"],
                    desc="NACA 0012 C-grid 608x160 with a wake cut, M 0.8, incidence 2.26 degrees, Re 9e6, "
                         "k-omega tau_t, directional expansion in each face's frame, 2000 CFL steps")
    if name.startswith("corner2d_"):
        nx, ny = (int(v) for v in name.split("_")[1].split("x"))
        spec = inputs.compression_corner(nx, ny, alpha_deg=24.0)
        spec["dx"] = [np.full(nx, 1.0 / nx), np.full(ny, 1.0 / ny)]  # unused: the grid is body-fitted
        return dict(spec=spec, kw=dict(gamma=1.4, mu=spec["mu"], T_wall=spec["T_wall"], turb_model="komega",
                                       beta_star=0.09, C_a=0.5, limiter="vanleer", expand="directional"),
                    nsteps=2000, t_end=0.0, precision=precision or "fp32", nodes=spec["nodes"],
                    desc="Mach 2.85 boundary layer over a 24-degree compression corner on a body-fitted "
                         "%dx%d wall-clustered channel grid, k-omega tau_t, directional expansion in each "
                         "face's frame, 2000 CFL steps" % (nx, ny))
    if name.startswith("turb3d_"):  # 256: the workload; 160: a smaller case (still larger than L2) for captures
        n3 = int(name.split("_")[1])
        spec = inputs.turbulence(n3, 3, seed=2132)
        return dict(spec=spec, kw=dict(gamma=1.4, mu=MU, turb_model="keps", C_mu=0.09, C_a=0.0, limiter="vanleer",
                                       expand="multid"), nsteps=100, t_end=0.0, precision=precision or "fp32_acc64",
                    desc="3D decaying turbulence %d^3, k-epsilon tau_t, multi-D, 100 CFL steps, FP32 flux with the "
                         "state accumulated in IEEE double" % n3)
    raise ValueError(name)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the step kernel, taken from
# one ncu capture of the same kernel build, keyed by workload and tile variant; a combination that
# was not captured (or whose kernel changed since) reports null.
# The shock / boundary-layer kernels were captured before the flux's last two changes, so that workload
# reports null.
TRAFFIC_PER_LAUNCH = {("turb2d_1024_keps_multid_fp32_acc64", 3): 43.06e6,
                      # 160^3 capture of the same kernel scaled by cells (x 4.096): the state streams at both sizes
                      ("turb3d_256_fp32_acc64", 2): 1.3804e9}


def faces_of(n, bc=None):
    """Distinct faces of a grid: n_d + 1 per grid line along axis d, n_d on a periodic axis (the wrap
    face is one face)."""
    D = len(n)
    tot = 0
    for d in range(D):
        f = n[d] + (0 if bc is not None and bc[d][0] == 0 else 1)
        for e in range(D):
            if e != d:
                f *= n[e]
        tot += f
    return tot


def steady_faces_per_cycle(n, levels):
    """Face flux evaluations of one multigrid cycle by level: (faces, cells, evaluations) per level.
    The finest level evaluates its residual before and after smoothing, every coarser level that of
    the restricted state, before smoothing and (except the coarsest) after it."""
    out = []
    for l in range(levels):
        a, b = n[0] >> l, n[1] >> l
        evals = (2 if levels > 1 else 1) if l == 0 else (2 if l == levels - 1 else 3)
        out.append(((a + 1) * b + a * (b + 1), a * b, evals))
    return out


def run_steady(args, wl):
    import torch
    from paper_1302_2132_gb300 import build, gks
    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    gks.load()
    spec = wl["spec"]
    n = tuple(spec["n"])
    levels = wl["levels"]
    transport = wl.get("transport", False)
    s = gks.SteadySolver(n, spec["bc"], spec["nodes"], levels=levels, bc_data=spec["bc_prim"], gamma=1.4,
                         mu=spec["mu"], T_wall=spec["T_wall"], turb_model="komega_transport" if transport
                         else "komega", beta_star=0.09, C_a=0.5,
                         limiter="vanleer", precision=wl["precision"], lusgs_tile=args.lusgs_tile,
                         wake_cut=spec.get("wake_cut", 0), expand=args.expand or "directional",
                         rarefaction=args.rarefaction)
    prim_dev = torch.tensor(spec["prim"].ravel(), device=dev)
    f1_dev = torch.tensor(np.ravel(spec["f1"]), dtype=torch.float64, device=dev)
    f2_dev = torch.tensor(np.ravel(spec["f2"]), dtype=torch.float64, device=dev)
    if not transport:  # transported fields are set after each set_state
        s.set_turbulence(f1_dev, f2_dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sched = wl["schedule"]
    ncyc = sum(k for k, _ in sched)
    hist = None

    def one_step():
        nonlocal hist
        s.set_state(prim_dev, layout="soa_prim")
        if transport:
            s.set_turbulence(f1_dev, f2_dev)
        hist = np.concatenate([s.cycles(k, cfl=c, cfl_flux=0.5) for k, c in sched])

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush.fill_(1)
        s.stream.wait_stream(torch.cuda.current_stream())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        one_step()
        e1.record(s.stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    clock_info = clocks.stop() if clocks else None
    if world > 1:
        ms = max_over_ranks(ms, dev)
    e2e = None
    if not args.no_e2e:
        prim_host = torch.tensor(spec["prim"].ravel()).pin_memory()
        out_host = np.zeros(4 * n[0] * n[1])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f1_host = torch.tensor(np.ravel(spec["f1"]), dtype=torch.float64).pin_memory()
        f2_host = torch.tensor(np.ravel(spec["f2"]), dtype=torch.float64).pin_memory()
        for _ in range(args.steps):
            s.set_state(prim_host, layout="soa_prim")
            if transport:
                s.set_turbulence(f1_host, f2_host)
            for k, c in sched:
                s.cycles(k, cfl=c, cfl_flux=0.5)
            out_host = s.get_state()
        e2e_s = time.perf_counter() - t0
        assert np.isfinite(out_host).all()
    per_level = steady_faces_per_cycle(n, levels)
    faces_cycle = sum(f * e for f, _, e in per_level)
    if not args.no_e2e:
        e2e = {"value": faces_cycle * ncyc * args.steps * world / e2e_s, "unit": "face_flux_evals/s",
               "h2d_bytes_per_step": int((prim_host.numel() + (2 * n[0] * n[1] if transport else 0)) * 8),
               "d2h_bytes_per_step": int(out_host.size * 8)}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    secs = ms / 1e3
    value = faces_cycle * ncyc * args.steps * world / secs
    fo_face = sum(gks.face_op_count(2, False, False)[:3])
    so_face = sum(gks.face_op_count(2, False, True)[:3])
    per_cell = CELL_OPS + sum(gks.cell_op_count(2)[:3])
    ops_cycle = sum(e * (f * (so_face if l == 0 else fo_face) + c * per_cell) for l, (f, c, e) in enumerate(per_level))
    if transport:  # the k-omega update of the finest grid
        ops_cycle += per_level[0][1] * KOMEGA_CELL_OPS[2]
    achieved = ops_cycle * ncyc * args.steps / secs / 1e12
    fp64 = wl["precision"] == "fp64"
    lanes = 2 if fp64 else 128
    peak = 152 * lanes * 2 * 2.070e9 / 1e12
    line = {
        "metric": "interface flux evals/sec and cell-updates/sec (% roofline); serving solves/sec, p50/p99",
        "value": value,
        "unit": "face_flux_evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if fp64 else "f32",
        "data": "synthetic",
        "config": {"workload": "%s_%s" % (args.workload, wl["precision"]) + ("_multid" if args.expand == "multid"
                                                                             else "") +
                               ("_rarefaction_tauhat" if args.rarefaction != "dt" else ""),
                   "description": wl["desc"], "grid": list(n), "expand": args.expand or "directional",
                   "levels": levels, "lusgs_tile": args.lusgs_tile, "cycles_per_bench_step": ncyc,
                   "precision": wl["precision"],
                   "l2": "flushed between bench steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "cycles_per_s": ncyc * args.steps * world / secs,
        "residual_drop": float(hist[-1] / hist[0]),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None,
                     "kernel": "whole multigrid cycle (residual kernels, LU-SGS, transfers), operations of the "
                               "residual evaluations only",
                     "ops_per_cycle": ops_cycle,
                     "peak_basis": "152 SMs x %d %s lanes x 2 (FMA) x 2070 MHz (derived)" % (lanes, "FP64" if fp64
                                                                                            else "FP32")},
        # per bench step: state_in; per cycle and level the local steps, residual, face spectral radii
        # and LU-SGS, plus (above the coarsest) the residual after smoothing, restriction, coarse
        # residual and forcing; the prolongations and the residual store; per cycles() call the
        # physical-state check
        # (with k-omega transport: per cycle the two field conversions, their restrictions and the
        # update; per bench step the six conversions of set_turbulence and their restrictions)
        "gpu_launches": args.steps * (1 + ncyc * (sum(4 + (6 if l + 1 < levels else 0) for l in range(levels))
                                                  + (levels - 1) + 1
                                                  + ((2 + 2 * (levels - 1) + 1) if transport else 0))
                                      + len(sched) + ((6 + 2 * (levels - 1)) if transport else 0)),
        "clocks": clock_info,
        "e2e": e2e,
    }
    print(json.dumps(line))
    sys.stdout.flush()
    s.close()
    if world > 1:
        dist.destroy_process_group()


def run_ours(args):
    import torch
    if args.workload.startswith("steady_"):
        return run_steady(args, make_workload(args.workload, args.precision))
    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_1302_2132_gb300 import build, gks
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    gks.load()
    wl = make_workload(args.workload, args.precision)
    if args.expand and wl.get("nodes") is not None:
        wl["kw"]["expand"] = args.expand
    spec = wl["spec"]
    D = spec["dim"]
    n = tuple(spec["n"])
    faces_per_step = faces_of(n, spec["bc"] if wl.get("nodes") is None else None)
    cells = int(np.prod(n))
    solver = gks.Solver(D, n, spec["bc"], dx=spec["dx"], bc_data=spec.get("bc_prim"), precision=wl["precision"],
                        reconstruction=args.reconstruction, rarefaction=args.rarefaction, **wl["kw"])
    curv = wl.get("nodes") is not None
    if curv:
        solver.set_nodes(wl["nodes"])
    prim_dev = torch.tensor(spec["prim"].ravel(), device=dev)
    turb = wl["kw"].get("turb_model", "none") != "none"
    transport = wl.get("transport", False)
    if turb:
        f1 = torch.tensor(spec["f1"].ravel(), device=dev)
        f2 = torch.tensor(spec["f2"].ravel(), device=dev)
        if not transport:  # transported fields are set after each set_state
            solver.set_turbulence(f1, f2)
    if args.profile > 0:
        # a short run for kernel captures: state in, NSTEPS steps, nothing timed
        solver.set_state(prim_dev, layout="soa_prim")
        if transport:
            solver.set_turbulence(f1, f2)
        solver.step(nsteps=args.profile, cfl=CFL, t_end=wl["t_end"])
        torch.cuda.synchronize()
        solver.close()
        return
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = solver.stream
    nsteps = wl["nsteps"]
    if wl["t_end"] > 0.0:  # count the steps that reach t_end
        solver.set_state(prim_dev, layout="soa_prim")
        if transport:
            solver.set_turbulence(f1, f2)
        nsteps = 0
        while solver.time()[0] < wl["t_end"]:
            solver.step(nsteps=1, cfl=CFL, t_end=wl["t_end"])
            nsteps += 1

    def one_step(mid=None):
        solver.set_state(prim_dev, layout="soa_prim")
        if transport:
            solver.set_turbulence(f1, f2)
        if mid is not None:
            mid.record(stream)
        solver.step(nsteps=nsteps, cfl=CFL, t_end=wl["t_end"])

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    # ---- timed region: K bench steps, each bracketed by events on the library stream ----------
    # A third event after the state copy-in marks the start of the time steps: the step kernels are
    # timed as the bench runs them, inside the captured graphs.
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush.fill_(1)
        stream.wait_stream(torch.cuda.current_stream())
        e0, em, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        one_step(em)
        e1.record(stream)
        evs.append((e0, em, e1))
        torch.cuda.current_stream().wait_stream(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = sum(a.elapsed_time(c) for a, _, c in evs)
    # the time steps of each bench step (step kernels in their graphs; with a separate transport
    # kernel, both), per time step
    kms = sum(b.elapsed_time(c) for _, b, c in evs)
    klaunch = nsteps * args.steps
    clock_info = clocks.stop() if clocks else None
    # sanity of the result: finite state, conservation monitor
    _, _, total = solver.residual()
    t_end, _ = solver.time()
    if world > 1:
        ms = max_over_ranks(ms, dev)
    # ---- end to end through the C ABI from pinned host memory ----------------------------------
    e2e = None
    if not args.no_e2e:
        prim_host = torch.tensor(spec["prim"].ravel()).pin_memory()
        f1_host = torch.tensor(spec["f1"].ravel()).pin_memory() if turb else None
        f2_host = torch.tensor(spec["f2"].ravel()).pin_memory() if turb else None
        out_host = torch.empty((D + 2) * cells, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            solver.set_state(prim_host, layout="soa_prim")
            if turb:
                solver.set_turbulence(f1_host, f2_host)
            solver.step(nsteps=nsteps, cfl=CFL, t_end=wl["t_end"])
            solver.get_state(out=out_host)
        t1 = time.perf_counter()
        assert torch.isfinite(out_host).all()
        e2e_s = (t1 - t0)
        e2e = {"value": faces_per_step * nsteps * args.steps * world / e2e_s, "unit": "face_flux_evals/s",
               "h2d_bytes_per_step": int(prim_host.numel() * 8 + (2 * cells * 8 if turb else 0)),
               "d2h_bytes_per_step": int(out_host.numel() * 8)}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    secs = ms / 1e3
    value = faces_per_step * nsteps * args.steps * world / secs
    # roofline of the fused step kernel (ALU bound): algorithmic operations per launch
    multid = wl["kw"].get("expand") == "multid" and D > 1
    counts = gks.face_op_count(D, multid, args.reconstruction == "muscl2")
    per_face = sum(counts[:3]) + sum(gks.recon_op_count(D, args.reconstruction)[:3])
    per_cell = CELL_OPS + sum(gks.cell_op_count(D)[:3]) + (KOMEGA_CELL_OPS[D] if transport else 0)
    ops_per_launch = faces_per_step * per_face + cells * per_cell
    avg_launch_s = kms / 1e3 / max(klaunch, 1)
    achieved = ops_per_launch / avg_launch_s / 1e12
    fp64 = wl["precision"] == "fp64"
    prec_name = {"fp64": "PREC_F64", "fp32": "PREC_F32", "fp32_acc64": "PREC_F32D"}[wl["precision"]]
    lanes = 2 if fp64 else 128  # FP64 runs at 1/64 of the FP32 rate on this part
    peak = 152 * lanes * 2 * 2.070e9 / 1e12
    workload_name = (WORKLOAD if args.workload == "turb2d_1024" and wl["precision"] == "fp32_acc64"
                     else "%s_%s" % (args.workload, wl["precision"]))
    if args.reconstruction != "muscl2":
        workload_name += "_" + args.reconstruction
    if args.expand == "multid" and curv:
        workload_name += "_multid"
    if args.rarefaction != "dt":
        workload_name += "_rarefaction_tauhat"
    tile = solver.tile_shape()
    # on body-fitted grids the MUSCL-2 step in FP64 or the FP32 float-pair form carries the transport
    fused_tr = transport and curv and args.reconstruction == "muscl2" and wl["precision"] in ("fp32", "fp64")
    tile_info = {"variant": tile[0], "cells": list(tile[1:1 + D]), "chosen_by": "autotuner"}
    line = {
        "metric": "interface flux evals/sec and cell-updates/sec (% roofline); serving solves/sec, p50/p99",
        "value": value,
        "unit": "face_flux_evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if fp64 else "f32",
        "data": "synthetic",
        "config": {"workload": workload_name,
                   "description": wl["desc"], "grid": list(n), "time_steps_per_bench_step": nsteps, "cfl": CFL,
                   "expand": "multid" if multid else "directional", "reconstruction": args.reconstruction,
                   "precision": wl["precision"], "state_accumulation": {"fp32": "float pair (hi+lo)",
                                                                        "fp32_acc64": "IEEE double",
                                                                        "fp64": "IEEE double"}[wl["precision"]],
                   "l2": "flushed between bench steps (256 MiB write)", "parallelism": "replicas" if world > 1 else "single"},
        "cell_updates_per_s": cells * nsteps * args.steps * world / secs,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": TRAFFIC_PER_LAUNCH.get((workload_name, tile_info.get("variant"))),
                     "kernel": (("step_kernel<%d, %s, %s>%s" % (D, prec_name, "multid" if multid else "directional",
                                                                 " + komega_kernel (timed together)" if transport
                                                                 else "")) if not curv else
                                "curv_step_kernel<%s, variant %d>%s" % (prec_name, tile[0],
                                                                         (" with the k-omega transport fused in"
                                                                          if fused_tr else
                                                                          " + curv_komega_kernel (timed together)")
                                                                         if transport else "")),
                     "avg_launch_us": avg_launch_s * 1e6,
                     "ops_per_face": per_face, "ops_per_cell": per_cell,
                     "peak_basis": "152 SMs x %d %s lanes x 2 (FMA) x 2070 MHz (derived)" % (lanes, "FP64" if fp64
                                                                                            else "FP32")},
        # per bench step: state_in + rate kernels, one step kernel per time step (plus, with k-omega
        # transport, the four field conversions of set_turbulence and, unless it is fused into the
        # body-fitted step, one transport kernel per time step)
        "gpu_launches": args.steps * (((nsteps if fused_tr else 2 * nsteps) + 2 + 4) if transport else (nsteps + 3)),
        "clocks": clock_info,
        "e2e": e2e,
        "final_time": t_end,
        "total_mass": float(total[0]),
    }
    line["config"]["tile"] = tile_info
    if (args.workload in ("turb2d_1024", "shock_bl_1024x384", "turb3d_256") and args.precision is None
            and args.reconstruction == "muscl2" and args.rarefaction == "dt"):
        # the float-pair form of the same workload, timed the same way: a second, labelled figure
        line["float_pair_form"] = time_other_form(args, wl, "fp32", faces_per_step, nsteps, ops_per_launch, peak,
                                                  dev, flush)
    if not args.no_cpu_baseline and args.workload == "turb2d_1024":
        line["cpu_baseline"] = cpu_baseline(budget_s=15.0)
    if not args.no_serving and args.workload == "turb2d_1024":
        try:
            line["serving"] = serving_summary(args.requests)
        except Exception as exc:  # the serving figures are reported beside the main metric
            line["serving"] = {"error": repr(exc)}
    print(json.dumps(line))
    sys.stdout.flush()
    if world > 1:
        dist.destroy_process_group()


def time_other_form(args, wl, precision, faces_per_step, nsteps, ops_per_launch, peak, dev, flush):
    """The same workload in another arithmetic form, timed as the headline is (K bench steps after W
    warm-up steps, events on the library stream, L2 flushed between bench steps)."""
    import torch
    from paper_1302_2132_gb300 import gks
    spec = wl["spec"]
    s = gks.Solver(spec["dim"], tuple(spec["n"]), spec["bc"], dx=spec["dx"], bc_data=spec.get("bc_prim"),
                   precision=precision, **wl["kw"])
    prim = torch.tensor(spec["prim"].ravel(), device=dev)
    f1 = torch.tensor(spec["f1"].ravel(), device=dev)
    f2 = torch.tensor(spec["f2"].ravel(), device=dev)
    s.set_turbulence(f1, f2)
    st = s.stream
    for _ in range(args.warmup):
        s.set_state(prim, layout="soa_prim")
        s.step(nsteps=nsteps, cfl=CFL)
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush.fill_(1)
        st.wait_stream(torch.cuda.current_stream())
        e0, em, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        s.set_state(prim, layout="soa_prim")
        em.record(st)
        s.step(nsteps=nsteps, cfl=CFL)
        e1.record(st)
        evs.append((e0, em, e1))
        torch.cuda.current_stream().wait_stream(st)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(c) for a, _, c in evs)
    kus = sum(b.elapsed_time(c) for _, b, c in evs) * 1e3 / (nsteps * args.steps)
    tile = s.tile_shape()
    s.close()
    return {"precision": precision, "state_accumulation": "float pair (hi+lo), about 48 significant bits",
            "value": faces_per_step * nsteps * args.steps / (ms / 1e3), "unit": "face_flux_evals/s",
            "ms_per_step": ms / args.steps, "avg_launch_us": kus,
            "roofline_frac": ops_per_launch / (kus * 1e-6) / 1e12 / peak,
            "kernel": "step_kernel<%d, PREC_F32, multid>" % spec["dim"],
            "tile": {"variant": tile[0], "cells": list(tile[1:1 + spec["dim"]])}}


# per-cell operations of the k-omega transport step (hand count of the kernel: per axis about 190 --
# k and omega of five cells, two limited-slope triples, two half-time face values with diffusion,
# gradients; sources about 100)
KOMEGA_CELL_OPS = {1: 290, 2: 480, 3: 670}

# per-cell operations of the fused step besides the faces and the reconstruction slopes (counted by
# gks_cell_op_count): turbulent relaxation time (velocity gradient, strain rate, k-epsilon formula:
# about 60), update (nv x (2 x 3)), CFL rate (about 12) -- a hand count
CELL_OPS = 60 + 4 * 6 + 12


def flop_counts(multid=True):
    from paper_1302_2132_gb300 import gks
    return list(gks.face_op_count(2, multid, True))


def oracle_sample(n_crop, nthreads):
    """One FP64 oracle time step on an n_crop^2 crop of the workload: (faces evaluated, seconds)."""
    import oracle
    spec = workload_inputs()
    prim = spec["prim"][:, :n_crop, :n_crop]
    h = 2 * math.pi / N
    c = oracle.Case(2, (n_crop, n_crop), [np.full(n_crop, h)] * 2, [[0, 0], [0, 0]], gamma=1.4, mu=MU,
                    turb_model=oracle.TURB_KEPS, C_mu=0.09, C_a=0.0, limiter=oracle.LIM_VANLEER, multid=1)
    W = c.prim_to_cons(np.ascontiguousarray(prim).ravel())
    f1 = np.ascontiguousarray(spec["f1"][:n_crop, :n_crop]).ravel()
    f2 = np.ascontiguousarray(spec["f2"][:n_crop, :n_crop]).ravel()
    dt = c.compute_dt(W, CFL)
    t0 = time.perf_counter()
    c.step(W, dt, f1=f1, f2=f2, nthreads=nthreads)
    return 2 * n_crop * n_crop, time.perf_counter() - t0


def cpu_baseline(budget_s=15.0):
    cores = os.cpu_count() or 1
    n_crop = 128
    faces, secs = oracle_sample(n_crop, cores)
    # grow the crop to spend about budget_s of wall time
    scale = max(1.0, math.sqrt(budget_s / max(secs, 1e-3)))
    n_crop = int(min(N, 16 * round(n_crop * scale / 16)))
    faces, secs = oracle_sample(n_crop, cores)
    return {"value": faces / secs, "unit": "face_flux_evals/s", "cores": cores, "kind": "oracle",
            "sample": "one FP64 time step of a %dx%d crop of the 1024^2 workload (OpenMP over faces, %d threads)"
                      % (n_crop, n_crop, cores)}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    n_crop = 160
    for _ in range(args.warmup):
        oracle_sample(64, cores)
    total_f, total_s = 0, 0.0
    for _ in range(args.steps):
        f, s = oracle_sample(n_crop, cores)
        total_f += f
        total_s += s
    value = total_f / total_s
    line = {"impl": "reference",
            "metric": "interface flux evals/sec and cell-updates/sec (% roofline); serving solves/sec, p50/p99",
            "value": value, "unit": "face_flux_evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [N, N], "sample_crop": [n_crop, n_crop]},
            "cpu_baseline": {"value": value, "unit": "face_flux_evals/s", "cores": cores, "kind": "oracle",
                             "sample": "each step: one FP64 time step of a %dx%d crop of the 1024^2 workload"
                                       % (n_crop, n_crop)},
            "e2e": {"value": value, "unit": "face_flux_evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _gen_request(args):
    from paper_1302_2132_gb300 import inputs
    return inputs.serving_request(*args)


def serving_requests(count, seed=4000):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_gen_request, [(i, seed) for i in range(count)], chunksize=16)


SERVE_KW = dict(gamma=1.4, mu=1e-4, C_a=0.5, cfl=0.5, limiter="vanleer", expand="multid")


def serve_stream(reqs, rate, seed, arena=16 << 30):
    """Submit reqs at Poisson arrival times (rate per second; 0 = all at once) and wait for all."""
    from paper_1302_2132_gb300 import inputs, serve
    srv = serve.Server(precision="fp32", arena_bytes=arena, max_cells=512 * 512, chunk_steps=24)
    tiles = srv.tile_variants()
    arrivals = inputs.poisson_arrivals(len(reqs), rate, seed) if rate > 0 else np.zeros(len(reqs))
    t0 = time.perf_counter()
    for r, ta in zip(reqs, arrivals):
        wait = t0 + ta - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        srv.submit(r, **SERVE_KW)
    srv.wait_all(3600)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    st["wall_s"] = wall
    st["offered_rate"] = rate
    st["tile_variants"] = tiles
    return st


def fp64_loop(reqs):
    """The plain FP64 per-solve loop on the same GPU: one solver per request, run to completion."""
    import torch
    from paper_1302_2132_gb300 import gks
    t0 = time.perf_counter()
    lat = []
    for r in reqs:
        ts = time.perf_counter()
        s = gks.Solver(r["dim"], r["n"], r["bc"], dx=r["dx"], gamma=1.4, mu=SERVE_KW["mu"], C_a=SERVE_KW["C_a"],
                       limiter="vanleer", expand="multid", precision="fp64")
        s.set_state(r["prim"].ravel(), layout="soa_prim")
        s.step(nsteps=r["nsteps"], cfl=SERVE_KW["cfl"])
        s.get_state()
        s.close()
        lat.append(time.perf_counter() - ts)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return {"solves_per_s": len(reqs) / wall, "requests": len(reqs), "p50_s": float(np.median(lat)),
            "p99_s": float(np.percentile(lat, 99))}


def serving_summary(count):
    """Serving form on the seeded stream: capacity (burst of 400), a Poisson stream at 0.8x capacity,
    a 2x overload of 1000 requests, and the plain FP64 per-solve loop on the first 400 requests."""
    reqs = serving_requests(count)
    # capacity with the first tile shape of every group, then with the shapes the server tunes
    os.environ["GKS_BATCH_TILES"] = "0,0,0"
    burst0 = serve_stream(reqs[:400], 0.0, 1)
    del os.environ["GKS_BATCH_TILES"]
    burst = serve_stream(reqs[:400], 0.0, 1)
    capacity = burst["completed"] / burst["wall_s"]
    steady = serve_stream(reqs, 0.8 * capacity, 2)
    over = serve_stream(reqs[:1000], 2.0 * capacity, 3)
    base = fp64_loop(reqs[:400])
    return {"metric": "serving solves/sec, p50/p99", "unit": "solves/s", "requests": len(reqs),
            "solves_per_s": steady["solves_per_s"], "p50_s": steady["p50_s"], "p99_s": steady["p99_s"],
            "offered_rate": steady["offered_rate"], "capacity_solves_per_s": capacity,
            "batch_tiles": {"tuned": burst["tile_variants"],
                            "capacity_with_first_shapes": burst0["completed"] / burst0["wall_s"]},
            "overload_2x": {k: over[k] for k in ("solves_per_s", "p50_s", "p99_s", "completed")},
            "fp64_per_solve_loop_solves_per_s": base["solves_per_s"], "fp64_per_solve_loop_requests": base["requests"],
            "batched_fp32_over_fp64_loop": capacity / base["solves_per_s"],
            "mix": "50% 1D (256-4096 cells), 50% 2D (64^2-512^2); Sod, Riemann quadrant, periodic turbulence; "
                   "50-500 steps; seed 4000; Poisson arrivals"}


def run_accuracy(args):
    """L1(rho) of the FP32 forms against the FP64 oracle after a run, on small instances of each
    configuration (the oracle runs them in seconds on the host cores)."""
    import torch
    import oracle
    from paper_1302_2132_gb300 import build, gks, inputs
    torch.cuda.init()
    build.build()
    oracle.build()
    gks.load()
    cores = os.cpu_count() or 1
    cases = []
    s = inputs.sod_1d(400)
    cases.append(("sod1d_400_to_t0.2", s, dict(mu=1e-5, C_a=1.0, limiter="vanleer", expand="directional"),
                  dict(mu=1e-5, C_a=1.0, limiter=oracle.LIM_VANLEER, multid=0), 0, 0.2))
    s = inputs.turbulence(64, 2, seed=1302)
    cases.append(("turb2d_64_200steps", s, dict(mu=MU, turb_model="keps", expand="multid"),
                  dict(mu=MU, turb_model=oracle.TURB_KEPS, multid=1), 200, 0.0))
    s = inputs.shock_boundary_layer(96, 48)
    cases.append(("shock_bl_96x48_300steps", s, dict(mu=s["mu"], T_wall=s["T_wall"], turb_model="komega", C_a=0.5,
                                                   expand="multid"),
                  dict(mu=s["mu"], T_wall=s["T_wall"], turb_model=oracle.TURB_KOMEGA, C_a=0.5, multid=1), 300, 0.0))
    s = inputs.turbulence(24, 3, seed=2132)
    cases.append(("turb3d_24_30steps", s, dict(mu=MU, turb_model="keps", expand="multid"),
                  dict(mu=MU, turb_model=oracle.TURB_KEPS, multid=1), 30, 0.0))
    out = {}
    for name, spec, gkw, okw, nsteps, t_end in cases:
        c = oracle.Case(spec["dim"], spec["n"], spec["dx"], spec["bc"], gamma=1.4, bc_prim=spec.get("bc_prim"), **okw)
        W0 = c.prim_to_cons(spec["prim"].ravel())
        f1 = spec.get("f1")
        f2 = spec.get("f2")
        f1 = None if f1 is None else f1.ravel()
        f2 = None if f2 is None else f2.ravel()
        Wo, to, no, st = c.run(W0, nsteps if nsteps else 100000, cfl=CFL, t_end=t_end, f1=f1, f2=f2, nthreads=cores)
        rho_o = Wo.reshape(spec["dim"] + 2, -1)[0]
        res = {"oracle_steps": no}
        for prec in ("fp32", "fp32_acc64", "fp64"):
            sol = gks.Solver(spec["dim"], spec["n"], spec["bc"], dx=spec["dx"], bc_data=spec.get("bc_prim"),
                             gamma=1.4, precision=prec, **gkw)
            sol.set_state(spec["prim"].ravel(), layout="soa_prim")
            if f1 is not None:
                sol.set_turbulence(f1, f2)
            sol.step(nsteps=nsteps if nsteps else no, cfl=CFL, t_end=t_end)
            rho = sol.get_state().reshape(spec["dim"] + 2, -1)[0]
            res[prec + "_L1_rho_rel"] = float(np.sum(np.abs(rho - rho_o)) / np.sum(np.abs(rho_o)))
            sol.close()
        out[name] = res
    print(json.dumps({"metric": "L1(rho) relative error against the FP64 oracle after the run", "cases": out}))


def run_serving(args):
    import torch
    from paper_1302_2132_gb300 import build, gks
    torch.cuda.init()
    reqs = serving_requests(args.requests)  # spawned workers, before the first kernel
    build.build()
    gks.load()
    cells = [int(np.prod(r["n"])) * r["nsteps"] for r in reqs]
    os.environ["GKS_BATCH_TILES"] = "0,0,0"
    burst0 = serve_stream(reqs[:400], 0.0, 1)
    del os.environ["GKS_BATCH_TILES"]
    burst = serve_stream(reqs[:400], 0.0, 1)
    capacity = burst["completed"] / burst["wall_s"]
    steady = serve_stream(reqs, 0.8 * capacity, 2)
    over = serve_stream(reqs[:1000], 2.0 * capacity, 3)
    sample = reqs[:400]
    base = fp64_loop(sample)
    line = {"metric": "serving solves/sec, p50/p99", "value": steady["solves_per_s"], "unit": "solves/s",
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving_stream_4000", "requests": len(reqs), "seed": 4000,
                       "mix": "50% 1D (256-4096 cells), 50% 2D (64^2-512^2); Sod, Riemann quadrant, periodic "
                              "turbulence; 50-500 steps; FP32 flux, float-pair state",
                       "cell_steps_total": int(sum(cells))},
            "capacity_solves_per_s": capacity, "burst": burst, "steady_0p8": steady, "overload_2x": over,
            "capacity_with_first_tile_shapes": burst0["completed"] / burst0["wall_s"],
            "fp64_per_solve_loop": base,
            "batched_vs_fp64_loop": capacity / base["solves_per_s"]}
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.serving:
        run_serving(a)
    elif a.accuracy:
        run_accuracy(a)
    else:
        run_ours(a)
