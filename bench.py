"""Benchmark of the ParO hot path on one GB300 (or N independent replicas).

A step is one ParO outer iteration (Step 3: N shifted source problems by
batched PCG with float64 refinement; Step 4: Rayleigh-Ritz; Step 5: the
|delta lambda| test) over the 3-D harmonic-oscillator workload: V = r^2/2 on
[-8, 8]^3, 64^3 Q1 cells (250 047 interior nodes), N = 20 orbitals, sigma = 0,
seeded Gaussian initial orbitals.  The metric unit is one interior node of one
orbital updated by one outer iteration (DOF.orbital updates/s).

Lines printed (rank 0, one JSON line):
  value        device-resident throughput (inputs in HBM; CUDA events on the
               library's stream; L2 flushed between steps, outside the events)
  e2e          the same through the C ABI with host buffers: H2D of U, the
               call, D2H of U and lambda inside the timed region
  roofline     the CG operator kernel (q = A p), timed per launch with CUDA
               events inside the timed steps, algorithmic bytes / duration
  time_to_converge  mixed vs plain float64 GPU ParO from the initial guess to
               max |lambda - lambda_discrete| < 1e-6 Ha (discrete values stored
               under tests/golden, written from the CPU oracle by shift-invert)
  cpu_baseline the CPU FP64 oracle, one outer iteration of the same workload
``--impl reference`` times the oracle alone on the same workload.
Multi-GPU (torchrun): independent replicas, one per rank, no collective on the
data path; value = all ranks' units / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ParO dof·orbital updates/s & time-to-converge at 1e-6 Ha vs plain FP64 GPU"
UNIT = "dof*orbital updates/s"
NC, L, NORB, SIGMA = 64, 8.0, 20, 0.0
WORKLOAD = "harmonic oscillator V=r^2/2, [-8,8]^3, 64^3 Q1 cells (250047 dofs), N=20, sigma=0"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# what the mixed path computes in: float32 CG; float-float (two float32, ~48-bit)
# refinement residuals, b = (lambda + sigma) M u, H X, M X and the rotation;
# tensor-core Grams from inputs rounded to 24 bits (exact BF16-digit products);
# float64 Cholesky and small eigensolve
DTYPE = "f32 CG; f32x2 (float-float) residual, HX, MX and eigensolve; bf16-digit tcgen05 Grams and rotation"


def effective_inner_tol(inner_tol, solve_tol):
    """The library's inner tolerance: the given one, else sqrt(solve_tol) clamped to [1e-6, 1e-3]."""
    return inner_tol if inner_tol > 0 else min(1e-3, max(1e-6, solve_tol ** 0.5))
GOLD = os.path.join(ROOT, "tests", "golden", "discrete_spectra.json")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, dist, device):
    """The largest of every rank's value (the slowest replica sets the job's time);
    dist None: a single process."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, ws, t_max_ms):
    """Whole-job throughput of ws independent replicas: all ranks' units over the slowest time."""
    return units_per_rank * ws / (t_max_ms * 1e-3)


def problem(rank):
    from paper_1405_0260_gb300 import workloads as W

    return W.harmonic(nc=NC, L=L, N=NORB, seed=2000 + rank, sigma=SIGMA)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) over the bytes the
# single-pass CG kernel streams, from one ncu capture of the current kernel on
# this workload (the autotuner's 9-pass launch of the geometry the bench keeps,
# 32 x 4 tiles with two nodes a thread, every orbital active: 1.731 GB of DRAM
# traffic for 1.641 GB streamed); None when no capture of the current kernel
# exists.  The bench's traffic per launch is this ratio times the bytes its
# launches stream.
K_CG2_DRAM_OVER_STREAMED = 1.055


def peaks():
    try:
        with open(PEAKS) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def flush_l2(buf):
    buf.add_(1.0)  # 256 MiB write: larger than the 129 MB L2


def run_ours(args, ws, rank, local):
    import torch

    from paper_1405_0260_gb300 import binding as B

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    p = problem(rank)
    nI, N = p.n_interior, p.N
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED, stream=stream)
    with torch.cuda.stream(stream):
        Vq = torch.from_numpy(p.Vq).cuda()
        m.set_potential(Vq, p.sigma)
        U = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
        X = torch.empty_like(U)
    lam, _ = m.rayleigh_ritz(U, X)
    U.copy_(X)
    torch.cuda.synchronize()
    params = B.paro_default_params(fixed_outer=1, solve_tol=1e-10, inner_tol=args.inner_tol)
    for _ in range(args.warmup):
        _, lam, _ = m.iterate(U, lam, params)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush_l2(flush)
            stream.synchronize()
            ev[i][0].record(stream)
            _, lam, st = m.iterate(U, lam, params)
            ev[i][1].record(stream)
            launches += st.kernel_launches
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    # Second timed region, same workload: CUDA events on the library's stream
    # around every launch of the persistent CG kernel (profile = 1: one launch per
    # float32 correction solve), for the kernel's roofline.
    prof = B.paro_default_params(fixed_outer=1, solve_tol=1e-10, inner_tol=args.inner_tol, profile=1)
    prof_ms = 0.0
    prof_n = 0
    prof_units = 0
    prof_nodes = 0
    prof_act = 0
    for i in range(max(1, min(args.steps, 3))):
        with torch.cuda.stream(stream):
            flush_l2(flush)
        stream.synchronize()
        _, lam, st = m.iterate(U, lam, prof)
        prof_ms += st.prof_ms
        prof_n += st.prof_launches
        prof_units += st.prof_dof_orb
        prof_nodes += st.prof_node_passes
        prof_act += st.prof_dof_orb_active
    if dist is not None:
        dist.barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    t_max = max_over_ranks(ms, dist, "cuda")
    value = replica_throughput(nI * N * args.steps, ws, t_max)

    # roofline of the single-pass CG kernel (the whole float32 CG loop of a
    # correction solve in one cooperative launch, one pass per iteration).
    # Algorithmic bytes in the method's unit: per active (node, orbital) and
    # iteration 32 B (r, p, x read and written, q written and read back), per node
    # and orbital-block pass 36 B (V_q 32 B and D^-1 4 B of the potential term).
    # The kernel itself streams 32 B for every orbital of a group still iterating
    # and 116 B of operator per node pass (27 stored float32 weights, one pad, and
    # D^-1): the "streamed" figures.
    peak, peak_kind = peaks()
    roof = None
    if prof_n > 0 and prof_ms > 0:
        alg_bytes = 32.0 * prof_act + 36.0 * prof_nodes
        streamed = 32.0 * prof_units + 116.0 * prof_nodes
        achieved = alg_bytes / (prof_ms * 1e-3) / 1e9
        passes = prof_nodes / nI / prof_n  # one orbital block (N <= 32)
        roof = {"kernel": "k_cg2 (single-pass Jacobi PCG: TMA-tiled r, q, p with halo, 27-point stencil, "
                          "one cross-CTA reduction a pass)",
                "bound": "hbm",
                "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": (round(K_CG2_DRAM_OVER_STREAMED * streamed / prof_n) if K_CG2_DRAM_OVER_STREAMED else None),
                "alg_bytes_formula": "32 B x active (node, orbital) iterations + 36 B x node passes",
                "launches": prof_n, "avg_launch_us": round(1e3 * prof_ms / prof_n, 2),
                "alg_bytes_per_launch": round(alg_bytes / prof_n),
                "streamed_bytes_per_launch": round(streamed / prof_n),
                "streamed_gbs": round(streamed / (prof_ms * 1e-3) / 1e9, 1),
                "passes_per_launch": round(passes, 2),
                # active orbitals over the orbitals of the groups the kernel streamed
                "active_fraction": round(prof_act / prof_units, 4) if prof_units else None,
                # the per-PCG-iteration form of the metric
                "dof_orbital_cg_iterations_per_s": round(prof_act / (prof_ms * 1e-3))}

    # end to end through the C ABI with host buffers
    Uh = torch.empty((nI, N), dtype=torch.float64, pin_memory=True)
    Uh.copy_(U.cpu())
    e2e_ms = 0.0
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush_l2(flush)
        stream.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        with torch.cuda.stream(stream):
            U.copy_(Uh, non_blocking=True)
        _, lam, _ = m.iterate(U, lam, params)
        with torch.cuda.stream(stream):
            Uh.copy_(U, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
    e2e = {"value": nI * N * args.steps / (e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": nI * N * 8, "d2h_bytes_per_step": nI * N * 8 + N * 8}

    ttc = None
    if not args.skip_converge and rank == 0:
        ttc = time_to_converge(B, torch, p, stream, args.inner_tol)
    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        cpu = cpu_baseline(p, args.warmup, min(args.steps, 3))
    m.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE,
            "data": "synthetic (seeded Gaussian initial orbitals, analytic potential)",
            "config": {"workload": WORKLOAD, "precision": "mixed", "parallelism": f"replicas x{ws}",
                       "l2": "flushed (256 MiB write) between steps, outside the timed events",
                       "step": "one ParO outer iteration (source problems to 1e-10 + Rayleigh-Ritz)",
                       "solve_tol": 1e-10, "inner_tol": effective_inner_tol(args.inner_tol, 1e-10)},
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "clocks": clk.summary(),
            "cpu_baseline": cpu, "time_to_converge": ttc, "wall_s_timed_region": wall,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def shell_angles(B, torch, m, U, modes):
    """Largest M-principal angle, per oscillator shell, between the orbitals U and
    the exact discrete eigenvectors.  The eigenvectors come from the stored 1-D
    modes (tests/golden, written from the oracle's separable construction) as
    Kronecker products; M U from the library's float64 mass apply; only
    N x N products are formed here (cosines: resolves angles down to ~1e-8)."""
    v1 = np.array(modes["v1d"]).T
    V = np.stack([np.kron(v1[:, c], np.kron(v1[:, b], v1[:, a])) for a, b, c in modes["triples"]], axis=1)
    MU = torch.empty_like(U)
    m.apply(B.PARO_OP_M, U, MU)
    torch.cuda.synchronize()
    u, mu = U.cpu().numpy(), MU.cpu().numpy()
    out = []
    for a, b in modes["clusters"]:
        G = u[:, a:b].T @ mu[:, a:b]
        Cm = V[:, a:b].T @ mu[:, a:b]  # V^T M U (M symmetric)
        Li = np.linalg.inv(np.linalg.cholesky(0.5 * (G + G.T)))
        K = Li @ (Cm.T @ Cm) @ Li.T
        s2 = np.clip(1.0 - np.linalg.eigvalsh(0.5 * (K + K.T)), 0.0, 1.0)
        out.append(float(np.max(np.arcsin(np.sqrt(s2)))))
    return out


def time_to_converge(B, torch, p, stream, inner_tol, max_outer=400):
    """Device time from the initial guess until max |lambda - lambda_discrete| < 1e-6 Ha
    (one outer iteration per call, as the bench steps), the orbitals' angles there,
    and the device time of one call to a tight stop (|delta lambda| < 1e-12) with
    its angles."""
    try:
        with open(GOLD) as f:
            g = json.load(f)
        gold = np.array(g["harmonic_64_L8"]["values"][: p.N])
        modes = g["harmonic_64_L8_modes"]
    except Exception as e:  # stored values missing
        return {"error": f"no discrete reference values: {e}"}
    out = {"target": "max_i |lambda_i - lambda_i(discrete, shift-invert Lanczos)| < 1e-6 Ha",
           "angles": "largest M-principal angle per oscillator shell against the exact discrete eigenvectors"}
    for name, prec, params in (
        ("mixed", B.PARO_MIXED, B.paro_default_params(fixed_outer=1, solve_tol=1e-10, inner_tol=inner_tol)),
        ("fp64", B.PARO_FP64, B.paro_default_params(fixed_outer=1, solve_tol=1e-10)),
        ("mixed_mg", B.PARO_MIXED, B.paro_default_params(fixed_outer=1, solve_tol=1e-10, inner_tol=inner_tol,
                                                         precond=B.PARO_PRECOND_MG)),
    ):
        m = B.Mesh(p.n, p.lo, p.hi, prec, stream=stream)
        with torch.cuda.stream(stream):
            Vq = torch.from_numpy(p.Vq).cuda()
            m.set_potential(Vq, p.sigma)
            U = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        t0 = time.perf_counter()
        lam = None
        outer = 0
        err = float("inf")
        while outer < max_outer:
            _, lam, _ = m.iterate(U, lam, params)
            outer += 1
            err = float(np.max(np.abs(lam - gold)))
            if err < 1e-6:
                break
        b.record(stream)
        b.synchronize()
        out[name] = {"seconds": a.elapsed_time(b) * 1e-3, "wall_s": time.perf_counter() - t0,
                     "outer_iters": outer, "final_err_ha": err, "reached": err < 1e-6,
                     "max_shell_angle": max(shell_angles(B, torch, m, U, modes))}
        if name != "mixed_mg":
            # one call to |delta lambda| < 1e-12 (the mixed loop switches to float-float Grams near the end)
            with torch.cuda.stream(stream):
                U = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
            torch.cuda.synchronize()
            a.record(stream)
            rc, lam, st = m.iterate(U, None, B.paro_default_params(tol=1e-12, max_outer=max_outer, solve_tol=1e-11,
                                                                   inner_tol=inner_tol if prec == B.PARO_MIXED else 0.0),
                                    allow=(-4,))
            b.record(stream)
            b.synchronize()
            ang = shell_angles(B, torch, m, U, modes)
            out[name]["tight"] = {"seconds": a.elapsed_time(b) * 1e-3, "rc": rc, "outer_iters": st.outer_iters,
                                  "final_err_ha": float(np.max(np.abs(lam - gold))),
                                  "max_shell_angle": max(ang), "shell_angles": ang}
        m.close()
    if out["mixed"]["reached"] and out["fp64"]["reached"]:
        out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
        out["speedup_tight_mixed_vs_fp64"] = out["fp64"]["tight"]["seconds"] / out["mixed"]["tight"]["seconds"]
    if out["mixed_mg"]["reached"] and out["fp64"]["reached"]:
        out["speedup_mixed_mg_vs_fp64"] = out["fp64"]["seconds"] / out["mixed_mg"]["seconds"]
    return out


def oracle_outer_step(ops, U, lam):
    from oracle import paro as O

    sol = O.source_problems(ops, U, lam, 1e-10, 5000)
    rr = O.rayleigh_ritz(ops, sol.X)
    return rr.U, rr.lam


def cores_used(cpu_s, wall_s):
    """Host cores a timed region kept busy: process CPU time (all threads) over wall time."""
    return round(cpu_s / wall_s, 2) if wall_s > 0 else None


def host_cpu():
    """The host's logical CPU count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return os.cpu_count(), model


def oracle_sample(p, warmup, steps):
    """The oracle, as it stands, on the same workload: the initial Rayleigh-Ritz
    and `warmup` outer iterations untimed, then `steps` timed outer iterations
    (the GPU arm times its steps after the same number of warm-up iterations)."""
    from oracle import paro as O

    ops = O.assemble(O.Mesh(p.n, p.lo, p.hi), p.Vq, p.sigma)
    rr = O.rayleigh_ritz(ops, p.U0)
    U, lam = rr.U, rr.lam
    for _ in range(warmup):
        U, lam = oracle_outer_step(ops, U, lam)
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(steps):
        U, lam = oracle_outer_step(ops, U, lam)
    return time.perf_counter() - t0, time.process_time() - c0


def cpu_record(value, dt, cpu, what):
    ncpu, model = host_cpu()
    return {"value": value, "unit": UNIT, "kind": "oracle", "cores": cores_used(cpu, dt),
            "host_cpus": ncpu, "cpu_model": model,
            "sample": f"{what} ({dt:.1f} s wall, {cpu:.1f} s CPU): the single-threaded float64 oracle "
                      f"(scipy sparse products on one thread, the small dense products in the BLAS), not a "
                      f"multi-core CPU ParO; cores = CPU time / wall time"}


def cpu_baseline(p, warmup, steps):
    """A bounded sample of the reference arm: the oracle after the same warm-up."""
    dt, cpu = oracle_sample(p, warmup, steps)
    return cpu_record(p.n_interior * p.N * steps / dt, dt, cpu,
                      f"outer iterations {warmup + 1}-{warmup + steps} of the full workload after the initial "
                      f"Rayleigh-Ritz, as the GPU arm's timed steps")


def run_reference(args, ws, rank):
    if rank != 0:
        return
    p = problem(0)
    dt, cpu = oracle_sample(p, args.warmup, args.steps)
    v = p.n_interior * p.N * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64 (CPU oracle)", "parallelism": "host cores"},
            "cpu_baseline": cpu_record(v, dt, cpu, f"each step one full outer iteration of the workload, "
                                                   f"iterations {args.warmup + 1}-{args.warmup + args.steps}"),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_peaks(args):
    """The SIMT float32 and float64 FMA rates of this GPU (the roofline denominators
    of the float-float and float64 kernels), through paro_peak_fma."""
    import torch

    from paper_1405_0260_gb300 import binding as B

    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    out = {"workload": "peaks", "sms": nsm}
    for name, dt, tdt in (("fp32_tflops", B.PARO_F32, torch.float32), ("fp64_tflops", B.PARO_F64, torch.float64)):
        buf = torch.empty(8 * nsm * 256, dtype=tdt, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        iters = 4096 if dt == B.PARO_F32 else 256
        vals = [B.paro_peak_fma(dt, iters, buf.data_ptr(), stream) for _ in range(5)]
        out[name] = max(vals)
        out[name + "_runs"] = [round(v, 2) for v in vals]
    with Clocks(0) as clk:
        buf = torch.empty(8 * nsm * 256, dtype=torch.float32, device="cuda")
        B.paro_peak_fma(B.PARO_F32, 16384, buf.data_ptr(), torch.cuda.current_stream().cuda_stream)
    out["clocks"] = clk.summary()
    print(json.dumps(out), flush=True)


def run_batch(args):
    """Batched independent systems (not the headline line): every system's handle
    on its own stream, all advanced by paro_batch_iterate in mixed precision --
    batched (the correction solves of all systems in one launch per refinement
    sweep) and as a pool of host threads -- against the mixed and plain float64
    per-system loops; each runs the initial Rayleigh-Ritz and `steps` outer
    iterations per system."""
    import math

    import torch

    from paper_1405_0260_gb300 import binding as B
    from paper_1405_0260_gb300 import workloads as W

    systems = W.batch_systems(count=args.systems)
    units = sum(p.n_interior * p.N for p in systems) * args.steps
    params = B.paro_default_params(fixed_outer=args.steps, solve_tol=1e-10,
                                   precond=B.PARO_PRECOND_MG if args.precond == "mg" else B.PARO_PRECOND_JACOBI)
    # sigma per system: 1 - (lowest initial Ritz value), rounded up to 0.5 Ha, but at
    # least 0.5 - min V: the Ritz value of poor guesses can sit far above lambda_1,
    # while min V (Gauss points) bounds the spectrum from below (K/2 >= 0), so
    # H + sigma M stays positive definite
    meshes, keep = [], []
    for p in systems:
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED, stream=stream)
            vq = torch.from_numpy(np.ascontiguousarray(p.Vq)).cuda()
            m.set_potential(vq, 0.0)
            X = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
            lam0, _ = m.rayleigh_ritz(X, torch.empty_like(X))
            p.sigma = math.ceil(max(1.0 - lam0[0], 0.5 - float(np.min(p.Vq))) / 0.5) * 0.5
            m.set_potential(vq, p.sigma)
        meshes.append(m)
        keep.append((vq, X, stream))
    torch.cuda.synchronize()

    def run(fused, warm):
        """paro_batch_iterate over every system from U0; warm: one untimed call
        first (the batched plan and its autotuning are made on the first call)."""
        batch = B.Batch(workers=args.workers, fused=fused)
        for m, (vq, X, stream) in zip(meshes, keep):
            batch.add(m, X, None, params)
        if warm:
            for p, (vq, X, stream) in zip(systems, keep):
                X.copy_(torch.from_numpy(np.ascontiguousarray(p.U0)))
            torch.cuda.synchronize()
            batch.iterate()
        for p, (vq, X, stream) in zip(systems, keep):
            X.copy_(torch.from_numpy(np.ascontiguousarray(p.U0)))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rcs, _, stats = batch.iterate()
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        launches = batch.fused_launches()
        batch.close()
        return t, rcs, stats, launches

    t_mixed, rcs, stats, nfused = run(True, True)
    t_pool, rcs_pool, _, _ = run(False, False)
    for m in meshes:
        m.close()
    del keep
    torch.cuda.empty_cache()
    # one system after the other (handles made outside the clock): mixed precision
    # (the batching gain) and plain float64 (the reference loop)
    def loop(precision):
        t = 0.0
        for p in systems:
            m = B.Mesh(p.n, p.lo, p.hi, precision)
            vq = torch.from_numpy(np.ascontiguousarray(p.Vq)).cuda()
            m.set_potential(vq, p.sigma)
            U = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m.iterate(U, None, params)
            torch.cuda.synchronize()
            t += time.perf_counter() - t0
            m.close()
        return t

    t_mloop = loop(B.PARO_MIXED)
    t_fp64 = loop(B.PARO_FP64)
    sizes = collections_count(p.n[0] for p in systems)
    line = {"metric": "batched ParO throughput, independent systems (mixed batch vs float64 per-system loop)",
            "unit": UNIT, "systems": len(systems), "precond": args.precond, "outer_iters_per_system": args.steps,
            "mesh_counts": sizes, "N_range": [min(p.N for p in systems), max(p.N for p in systems)],
            "mixed_batch": {"value": units / t_mixed, "seconds": t_mixed,
                            "form": "one host thread per system; the correction solves of all systems in one "
                                    "batched cooperative launch per refinement sweep",
                            "batched_launches": nfused,
                            "ok": sum(1 for rc in rcs if rc == 0),
                            "rr_tc_steps": int(sum(st.rr_tc_steps for st in stats))},
            "mixed_pool": {"value": units / t_pool, "seconds": t_pool, "workers": args.workers,
                           "form": "pool of host threads, each system's own launches on its own stream",
                           "ok": sum(1 for rc in rcs_pool if rc == 0)},
            "mixed_loop": {"value": units / t_mloop, "seconds": t_mloop},
            "fp64_loop": {"value": units / t_fp64, "seconds": t_fp64},
            "speedup": t_fp64 / t_mixed, "batching_gain": t_mloop / t_mixed, "batched_vs_pool": t_pool / t_mixed,
            "data": "synthetic (seeded nuclei and Gaussian orbitals)"}
    print(json.dumps(line), flush=True)


def run_large(args):
    """The large fixed-potential workload (192^3 cells, 40 nuclei, N = 256, mixed
    precision): the initial Rayleigh-Ritz and one outer iteration untimed, then
    `steps` outer iterations timed (not the headline line)."""
    import math

    import torch

    from paper_1405_0260_gb300 import binding as B
    from paper_1405_0260_gb300 import workloads as W

    t0 = time.perf_counter()
    p = W.large_cluster(nc=args.large_nc)
    t_gen = time.perf_counter() - t0
    sigma = math.ceil((0.5 - float(np.min(p.Vq))) / 0.5) * 0.5  # min V bounds the spectrum from below
    free0, total = torch.cuda.mem_get_info()
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED)
    vq = torch.from_numpy(np.ascontiguousarray(p.Vq)).cuda()
    m.set_potential(vq, sigma)
    N, nI = p.N, p.n_interior
    U = torch.from_numpy(p.U0).cuda()
    p.U0 = None  # release the host copy
    t0 = time.perf_counter()
    pc = B.PARO_PRECOND_MG if args.precond == "mg" else B.PARO_PRECOND_JACOBI
    rc, lam, st0 = m.iterate(U, None, B.paro_default_params(fixed_outer=1, solve_tol=1e-10, precond=pc))
    torch.cuda.synchronize()
    t_first = time.perf_counter() - t0
    free1, _ = torch.cuda.mem_get_info()
    params = B.paro_default_params(fixed_outer=args.steps, solve_tol=1e-10, precond=pc)
    t0 = time.perf_counter()
    rc, lam, st = m.iterate(U, lam, params)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    units = nI * N * args.steps
    line = {"metric": "ParO outer iterations on the large workload (mixed precision)", "unit": UNIT,
            "value": units / dt, "seconds_per_outer": dt / args.steps, "outer_iters": args.steps,
            "workload": f"{len(p.nuclei)} softened-Coulomb nuclei, [-20,20]^3, {p.n[0]}^3 cells "
                        f"({nI} dofs), N={N}, sigma={sigma}", "precond": args.precond,
            "device_memory_gb": round((free0 - free1) / 1e9, 1), "device_total_gb": round(total / 1e9, 1),
            "first_call_s": round(t_first, 2), "generate_s": round(t_gen, 1),
            "stats": {"cg_iters_f32": st.cg_iters_f32, "cg_iters_max": st.cg_iters_max,
                      "refine_sweeps": st.refine_sweeps, "ms_solve": st.ms_solve, "ms_rr": st.ms_rr,
                      "rr_tc_steps": st.rr_tc_steps, "max_dlambda": st.max_dlambda},
            "lambda_1_4": [float(v) for v in lam[:4]], "data": "synthetic (seeded nuclei, random initial block)"}
    print(json.dumps(line), flush=True)
    m.close()


def run_ks(args):
    """The Kohn-Sham cluster (8 softened nuclei, 128^3 cells, mixed precision):
    SCF ParO with linear mixing 0.3, stopped at max |delta lambda| < 1e-6 over the
    occupied orbitals (the 8 extra orbitals are the Algorithm 3.2 buffer) or after
    --ks-max-outer SCF iterations, then the total energy (not the headline line).
    Reports the time per SCF iteration and the state reached."""
    import math

    import torch

    from oracle import ks as KS  # occupations only (a two-line rule), no method arithmetic
    from paper_1405_0260_gb300 import binding as B
    from paper_1405_0260_gb300 import workloads as W

    p = W.cluster(nc=args.ks_nc)
    N = p.U0.shape[1]
    n_el = int(round(float(p.nuclei[:, 3].sum())))
    occ = KS.occupations(N, n_el)
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED)
    vq = torch.from_numpy(np.ascontiguousarray(p.Vq)).cuda()
    m.set_potential(vq, 0.0)
    X = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
    # shift: first a safe one (min V bounds the spectrum from below) for a few ParO
    # iterations on V_ext alone, then 1 - theta_1 rounded up (theta_1 their lowest Ritz
    # value, an upper bound close to lambda_1).  The Hartree potential of 16 electrons
    # raises the spectrum by more than Slater exchange lowers it; a shift that still
    # leaves H + sigma M indefinite ends the solve with PARO_ERR_NOT_SPD.  A large shift
    # slows every source-problem step ((lambda_i + s)/(lambda_N+1 + s) -> 1).
    safe = math.ceil((0.5 - float(np.min(p.Vq))) / 0.5) * 0.5
    m.set_potential(vq, safe)
    U = X.clone()
    _, lam0, _ = m.iterate(U, None, B.paro_default_params(tol=1e-2, max_outer=100, solve_tol=1e-8), allow=(-4,))
    sigma = math.ceil((1.0 - lam0[0]) / 0.5) * 0.5
    m.set_potential(vq, sigma)
    pc = B.PARO_PRECOND_MG if args.precond == "mg" else B.PARO_PRECOND_JACOBI
    params = B.paro_default_params(tol=1e-6, max_outer=args.ks_max_outer, solve_tol=1e-10, n_check=p.n_occ,
                                   precond=pc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, lam, st = m.scf_iterate(U, occ, vq, args.ks_mix, params, allow=(-4,))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    energy = m.ks_energy(U, occ, lam, B.paro_default_params(solve_tol=1e-10))
    # the pieces of one SCF iteration outside the source problems and Rayleigh-Ritz,
    # each timed alone (device time, 3 calls): the potential set-up (operator
    # weights), the density, and the Kohn-Sham potential (Hartree solve + Slater)
    rho = torch.empty_like(vq)
    veff = torch.empty_like(vq)
    m.density(U, occ, rho)
    m.ks_potential(rho, vq, veff, None, params)

    def dev_ms(fn, reps=3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps

    pieces = {"set_potential_ms": dev_ms(lambda: m.set_potential(veff, sigma)),
              "density_ms": dev_ms(lambda: m.density(U, occ, rho)),
              "ks_potential_warm_ms": dev_ms(lambda: m.ks_potential(rho, vq, veff, None, params))}
    line = {"metric": "Kohn-Sham SCF ParO to max |delta lambda| < 1e-6 Ha on the occupied orbitals (mixed)",
            "workload": f"{len(p.nuclei)} softened nuclei, [-12,12]^3, {p.n[0]}^3 cells ({p.n_interior} dofs), "
                        f"{n_el} electrons, N={N} ({p.n_occ} occupied + buffer), sigma={sigma}, mixing {args.ks_mix}",
            "converged": rc == 0, "outer_iters": st.outer_iters, "seconds": dt,
            "ms_per_outer": 1e3 * dt / max(st.outer_iters, 1), "max_dlambda": st.max_dlambda,
            "poisson_cg_iters": st.poisson_cg_iters, "cg_iters_f32": st.cg_iters_f32,
            "rr_tc_steps": st.rr_tc_steps, "energy_ha": energy, "precond": args.precond,
            "ms_orbital_solves": st.ms_solve, "ms_rayleigh_ritz": st.ms_rr,
            "ms_hartree_density_potential": 1e3 * dt - st.ms_solve - st.ms_rr, "pieces": pieces,
            "lambda_occupied": [float(v) for v in lam[:p.n_occ]], "data": "synthetic (seeded nuclei)"}
    print(json.dumps(line), flush=True)
    m.close()


def run_clusters(args):
    """Cluster-separated Rayleigh-Ritz (Section 3): N = 256 orbitals on a 24^3 mesh (so
    that the small eigenproblem dominates the step), mixed precision, 3 outer iterations
    timed with one eigenvalue cluster, 4 of 64 and 16 of 16 (not the headline line)."""
    import torch

    from paper_1405_0260_gb300 import binding as B
    from paper_1405_0260_gb300 import workloads as W

    N = 256
    p = W.harmonic(nc=24, L=8.0, N=4, seed=8100, sigma=0.0)
    m = B.Mesh(p.n, p.lo, p.hi, B.PARO_MIXED)
    vq = torch.from_numpy(np.ascontiguousarray(p.Vq)).cuda()
    m.set_potential(vq, 2.0)
    U0 = torch.from_numpy(W.random_block(p.n, N, seed=8101)).cuda()
    out = {}
    for name, sizes in (("1x256", None), ("4x64", [64] * 4), ("16x16", [16] * 16)):
        U = U0.clone()
        _, lam, _ = m.iterate(U, None, B.paro_default_params(fixed_outer=1, solve_tol=1e-8))
        prm = B.paro_default_params(fixed_outer=3, solve_tol=1e-8)
        if sizes:
            prm.set_clusters(sizes)
        rc, lam, st = m.iterate(U, lam, prm)
        torch.cuda.synchronize()
        out[name] = {"rc": rc, "ms_rayleigh_ritz_per_outer": st.ms_rr / 3, "ms_source_problems_per_outer": st.ms_solve / 3}
    line = {"metric": "cluster-separated Rayleigh-Ritz time per outer iteration", "unit": "ms",
            "workload": f"harmonic V=r^2/2, [-8,8]^3, 24^3 cells ({p.n_interior} dofs), N={N}, sigma=2, mixed",
            "clusters": out, "data": "synthetic (seeded unit-variance block)"}
    print(json.dumps(line), flush=True)
    m.close()


def collections_count(values):
    out = {}
    for v in values:
        out[str(v)] = out.get(str(v), 0) + 1
    return out


def run_adapt(args):
    """The adaptive loop of Section 2.1 (not the headline line): a hydrogen-like
    nucleus off the nodes of a coarse uniform mesh; each step solves with
    paro_iterate (mixed precision, source problems to 1e-10, |delta lambda| <
    1e-9), estimates (paro_estimate), marks with Doerfler's strategy (theta
    0.5), refines the marked cells' axis intervals and moves the orbitals to the
    new mesh (paro_transfer).  Beside it, uniform meshes with about the same
    unknowns: the ground level a graded mesh reaches for its unknowns."""
    import math

    import torch

    from paper_1405_0260_gb300 import binding as B
    from paper_1405_0260_gb300 import workloads as W

    L, nc0, N, R = 10.0, args.adapt_nc, 5, (0.31, -0.23, 0.17)
    params = B.paro_default_params(tol=1e-9, max_outer=400, solve_tol=1e-10)

    def coulomb(n, coords):
        x, y, z = W.gauss_point_coords(n, None, None, coords)
        return np.ascontiguousarray((-1.0 / np.sqrt((x - R[0]) ** 2 + (y - R[1]) ** 2 + (z - R[2]) ** 2)).ravel())

    def handle(coords):
        n = tuple(len(c) - 1 for c in coords)
        m = B.Mesh(n, None, None, B.PARO_MIXED, coords=coords)
        Vd = torch.from_numpy(coulomb(n, coords)).cuda()
        m.set_potential(Vd, 2.0)
        return m, Vd

    def solve(m, U0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, lam, st = m.iterate(U0, None, params, allow=(-4,))
        torch.cuda.synchronize()
        return rc, lam, st, time.perf_counter() - t0

    ax = np.linspace(-L, L, nc0 + 1)
    coords = (ax, ax, ax)
    p = W.hydrogen(nc=nc0, L=L, N=N, seed=8700, sigma=2.0)
    U = torch.from_numpy(np.ascontiguousarray(p.U0)).cuda()
    steps, prev = [], None
    for k in range(args.adapt_steps):
        n = tuple(len(c) - 1 for c in coords)
        m, Vd = handle(coords)
        if prev is not None:
            Un = torch.empty(((n[0] - 1) * (n[1] - 1) * (n[2] - 1), N), dtype=torch.float64, device="cuda")
            prev.transfer_to(m, U, Un)
            prev.close()
            U = Un
        rc, lam, st, t_solve = solve(m, U)
        eta2 = torch.empty(n[0] * n[1] * n[2], dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.estimate(U, lam, Vd, eta2)
        torch.cuda.synchronize()
        t_est = time.perf_counter() - t0
        e = eta2.cpu().numpy().reshape(n[2], n[1], n[0])
        marked = B.mark(e, B.PARO_MARK_DORFLER, 0.5)
        steps.append({"cells": list(n), "unknowns": int((n[0] - 1) * (n[1] - 1) * (n[2] - 1)), "rc": int(rc),
                      "lambda": [float(v) for v in lam], "outer_iters": int(st.outer_iters),
                      "solve_s": t_solve, "estimate_s": t_est, "eta": float(np.sqrt(e.sum())),
                      "marked": int(marked.sum())})
        coords = B.refine_coords(n, coords, marked)
        prev = m
    prev.close()
    uniform = []
    for nc in sorted({int(round(math.pow(s["unknowns"], 1.0 / 3.0))) + 1 for s in steps[-2:]}):
        ax = np.linspace(-L, L, nc + 1)
        q = W.hydrogen(nc=nc, L=L, N=N, seed=8700, sigma=2.0)
        m, _ = handle((ax, ax, ax))
        rc, lam, st, t = solve(m, torch.from_numpy(np.ascontiguousarray(q.U0)).cuda())
        uniform.append({"cells": nc, "unknowns": (nc - 1) ** 3, "rc": int(rc), "lambda": [float(v) for v in lam],
                        "solve_s": t})
        m.close()
    print(json.dumps({"metric": "adaptive loop (Solve -> Estimate -> Mark -> Refine) on tensor-product meshes",
                      "workload": f"hydrogen-like Z=1 at {list(R)}, [-{L},{L}]^3, {nc0}^3 start, N={N}, sigma=2, "
                                  "mixed precision, Doerfler theta=0.5",
                      "steps": steps, "uniform": uniform,
                      "data": "synthetic (seeded Gaussian initial orbitals, analytic potential)"}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-cpu", action="store_true", help="omit the cpu_baseline leg")
    ap.add_argument("--skip-converge", action="store_true", help="omit the time-to-converge leg")
    ap.add_argument("--workload", default="harmonic64",
                    choices=["harmonic64", "batch", "large", "ks", "clusters", "peaks", "adapt"],
                    help="batch: independent systems (meshes 32-96^3, N 4-48) through paro_batch_iterate; "
                         "large: 192^3 cells, N = 256; ks: the Kohn-Sham cluster SCF; "
                         "clusters: cluster-separated Rayleigh-Ritz at N = 256; "
                         "peaks: the SIMT float32 and float64 FMA rates; "
                         "adapt: the adaptive loop on a hydrogen-like problem")
    ap.add_argument("--ks-nc", type=int, default=128, help="ks workload: cells per axis")
    ap.add_argument("--ks-max-outer", type=int, default=1500, help="ks workload: SCF iteration limit")
    ap.add_argument("--ks-mix", type=float, default=0.3, help="ks workload: linear density mixing")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="mixed path: relative tolerance of each float32 correction solve "
                         "(0: the library's choice, sqrt(solve_tol) = 1e-5 here)")
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "mg"],
                    help="ks, large, batch workloads: preconditioner of the float32 correction solves")
    ap.add_argument("--large-nc", type=int, default=192, help="large workload: cells per axis")
    ap.add_argument("--systems", type=int, default=64, help="batch workload: number of systems")
    ap.add_argument("--workers", type=int, default=8, help="batch workload: host worker threads")
    ap.add_argument("--adapt-nc", type=int, default=16, help="adapt workload: cells per axis of the first mesh")
    ap.add_argument("--adapt-steps", type=int, default=5, help="adapt workload: adaptive steps")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if args.workload in ("batch", "large", "ks", "clusters", "peaks", "adapt"):
        if rank == 0 and args.impl == "ours":
            {"batch": run_batch, "large": run_large, "ks": run_ks, "clusters": run_clusters,
             "peaks": run_peaks, "adapt": run_adapt}[args.workload](args)
        return
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
