"""Benchmark of the NEP hot path on GB300.

Headline: NVE molecular dynamics with the FP32 NEP force path on the
125,000-atom diamond workload (25^3 cells, 32-30-1 network, 300 K start,
dt = 1 fs, 1 A skin), in atom-steps per second.  One bench step is one MD
step: kick + drift, skin check (and list rebuild when due), site energies
and partial forces, force/virial assembly with the second kick, heat current
and FP64 reductions.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the only reference this paper
has: it publishes no code) on the host cores, on bounded samples of the same
workload.  Under torchrun (N > 1) every rank runs an independent replica
(the path has no exchange step) and rank 0 prints one JSON line.
"""
from __future__ import annotations

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

from paper_2107_08119_gb300 import inputs  # noqa: E402

METRIC = "NEP MD atom-step/s at 125k atoms; SNES generation/s (pop 50) vs plain FP32"
UNIT = "atom-step/s"
WORKLOAD = "NVE MD, 125,000-atom Si-like diamond (25^3 cells), NEP 32-30-1 FP32, dt 1 fs, skin 1 A"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------- flop model
def flops_per_atom(m_r: float, m_a: float, n_neu: int = 30) -> float:
    """Algorithmic FP32 flops (FMA = 2) of one atom's site + partial-force pass
    in the O(M) harmonic form: per radial pair 134 (g_n, g_n' for 8 orders,
    accumulation, contraction), per angular pair 1500 (g_n, g_n' for 6 orders,
    24 harmonics and gradients, 144 accumulations, 2 x 144 contractions,
    r-hat and gradient terms), per atom 288 for q_nl plus 2 x 2 x n_neu x 32
    for the network and its input gradient and 10 per tanh."""
    return 134.0 * m_r + 1500.0 * m_a + 288.0 + 4.0 * n_neu * 32 + 10.0 * n_neu


SITE_SOURCES = ("paper_2107_08119_gb300/csrc/nep_site.cuh", "paper_2107_08119_gb300/csrc/nep_force.cu",
                "paper_2107_08119_gb300/csrc/nep_internal.cuh")
SITE_PROFILE = os.path.join(ROOT, "profiles", "k_site_md_125k.json")


def sources_digest(paths) -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def site_dram_traffic():
    """DRAM bytes (read + write) of one k_site launch on this workload, from
    the committed ncu summary, or None when the kernel sources changed since
    those counters were taken."""
    try:
        prof = json.load(open(SITE_PROFILE))
    except (OSError, ValueError):
        return None
    if prof.get("sources_sha256") != sources_digest(SITE_SOURCES):
        return None
    return prof.get("dram_bytes_per_launch")


def fp32_peak_tflops(sm_mhz: float) -> float:
    """152 SMs x 128 FP32 lanes x 2 flops per FMA x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# --------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- CPU oracle
def cpu_oracle_md(seconds: float = 15.0, cells: int = 8, max_steps: int | None = None):
    """Oracle MD on an 8^3-cell (4,096-atom) block of the same lattice, model,
    displacements and temperature; atom-steps/s on the host cores."""
    import oracle
    pos, vel, box, z = inputs.config2(n_cells=cells)
    h = oracle.NepHyper()
    z = np.asarray(z, np.float32).astype(np.float64)
    n = len(pos)
    t0 = time.perf_counter()
    pos, vel, _, _ = oracle.md(h, z, pos, vel, box, inputs.MASS_SI, 1.0, 1)
    per = time.perf_counter() - t0
    steps = max(1, int(seconds / max(per, 1e-3)))
    if max_steps is not None:
        steps = min(steps, max_steps)
    t0 = time.perf_counter()
    oracle.md(h, z, pos, vel, box, inputs.MASS_SI, 1.0, steps)
    dt = time.perf_counter() - t0
    return {"value": n * steps / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{steps} velocity-Verlet steps (+1 startup force call excluded) of the FP64 oracle on a "
                      f"{n}-atom {cells}^3-cell block of the same workload (same model, sigma, 300 K)"}


def max_over_ranks(vals, dist=None, device="cpu"):
    """Each value's maximum over the ranks of the process group: the slowest
    rank sets the whole job's time.  Without a group, the values themselves."""
    if dist is None:
        return [float(x) for x in vals]
    import torch
    t = torch.tensor([float(x) for x in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_throughput(world: int, units_per_rank: int, steps: int, t_max_ms: float) -> float:
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return world * units_per_rank * steps / (t_max_ms / 1e3)


def run_reference(args, rank, world):
    """The oracle as the reference arm: W + K MD steps on the 4,096-atom sample."""
    if rank != 0:
        return 0
    import oracle
    pos, vel, box, z = inputs.config2(n_cells=8)
    h = oracle.NepHyper()
    z = np.asarray(z, np.float32).astype(np.float64)
    n = len(pos)
    if args.warmup > 0:
        pos, vel, _, _ = oracle.md(h, z, pos, vel, box, inputs.MASS_SI, 1.0, args.warmup)
    t0 = time.perf_counter()
    oracle.md(h, z, pos, vel, box, inputs.MASS_SI, 1.0, args.steps)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{n}-atom 8^3-cell block per step", "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"each step: one oracle MD step on a {n}-atom 8^3-cell block of the workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world, local):
    import torch
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep as N

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    pos, vel, box, z = inputs.config2()
    n = len(pos)
    hyper = N.Hyper()
    model = N.NEP(np.asarray(z, np.float32), hyper)

    # average neighbour counts within r_c^R and r_c^A (flop model of the site
    # pass), of the starting state and again of the final state
    p0 = torch.tensor(pos.T.copy(), dtype=torch.float64, device="cuda")
    m_r0, m_a0 = neighbour_counts(model, p0, box, hyper)

    md = N.MD(model, n, box, inputs.MASS_SI)
    p = torch.tensor(pos.T.copy(), dtype=torch.float64, device="cuda")
    v = torch.tensor(vel.T.copy(), dtype=torch.float64, device="cuda")
    K, W = args.steps, args.warmup
    thermo = torch.zeros(max(K, W, 1), N.THERMO_COLS, dtype=torch.float64, device="cuda")
    heat = torch.zeros(max(K, W, 1), 3, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    md.step(p, v, W, 1.0, thermo, heat)
    md.sync_status()
    rebuilds0 = md.rebuild_count()
    p_w, v_w = p.clone(), v.clone()   # the state after warm-up, for the phase-timing pass

    # the timed steps: no phase timing, so each step replays the captured step
    # graph (the list rebuild behind a conditional node)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("md_timed")  # names the timed launches for profiler filters (ncu --nvtx)
    e0.record(stream)
    md.step(p, v, K, 1.0, thermo, heat)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    md.sync_status()
    ms = e0.elapsed_time(e1)
    rebuilds = md.rebuild_count() - rebuilds0

    # the same K steps again from the same state with CUDA events around each
    # phase (launched one by one): the per-phase split and the k_site duration
    md2 = N.MD(model, n, box, inputs.MASS_SI)
    p2, v2 = p_w.clone(), v_w.clone()
    th2 = torch.zeros_like(thermo)
    md2.step(p2, v2, 0, 1.0)     # starting forces of the fresh handle, outside the timed phases
    torch.cuda.synchronize()
    model.profile_read()
    model.profile(True)          # events around each force-pass launch, on the launching stream
    torch.cuda.nvtx.range_push("md_phases")  # launched one by one: the pass profilers can take apart
    md2.step(p2, v2, K, 1.0, th2, None)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    model.profile(False)
    prof = model.profile_read()
    site_ms = prof["site"][0] / max(1, prof["site"][1])
    rebuilds_phase = md2.rebuild_count()
    md2.close()
    th = thermo[:K].cpu().numpy()
    etot = th[:, 0] + th[:, 1]
    m_r1, m_a1 = neighbour_counts(model, p, box, hyper)
    m_r, m_a = 0.5 * (m_r0 + m_r1), 0.5 * (m_a0 + m_a1)

    if args.only == "md":
        if rank == 0:
            print(json.dumps({"md_ms_per_step": ms / K, "phase_ms_per_step": {k: v[0] / K for k, v in prof.items()},
                              "list_rebuilds_timed": rebuilds, "clocks": clocks}), flush=True)
        md.close()
        model.close()
        if dist:
            dist.destroy_process_group()
        return 0

    # end to end through the C ABI with host buffers: per step, the state goes
    # host -> device from pinned memory and comes back with the thermo row.
    # The same K steps from the same warmed-up state as the timed region (a
    # fresh handle, starting forces outside the timing), so that both cover
    # one trajectory and its list rebuilds: the random-weight potential melts
    # the crystal, and later stretches of the run rebuild more often.
    # The state lives in one (6, n) buffer on each side (positions in rows
    # 0-2, velocities in rows 3-5: each a contiguous [3][n] block, as the
    # library takes them), so it crosses the host link as one copy each way.
    md3 = N.MD(model, n, box, inputs.MASS_SI)
    state = torch.cat([p_w, v_w])
    p3, v3 = state[0:3], state[3:6]
    md3.step(p3, v3, 0, 1.0)
    hstate = torch.empty_like(state, device="cpu").pin_memory()
    hth = torch.empty(N.THERMO_COLS, dtype=torch.float64).pin_memory()
    hstate.copy_(state)
    Ke = K
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Ke):
        state.copy_(hstate, non_blocking=True)
        md3.step(p3, v3, 1, 1.0, thermo, None)
        hstate.copy_(state, non_blocking=True)
        hth.copy_(thermo[0], non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    md3.sync_status()
    md3.close()

    # steady state of the melting run: after the timed window, skip ahead
    # and time a later window of the same trajectory (the random-weight
    # potential heats the crystal, and the list is rebuilt more often)
    steady = None
    if args.steady_steps > 0:
        md.step(p, v, args.steady_skip, 1.0)
        r_s0 = md.rebuild_count()
        torch.cuda.synchronize()
        e0.record(stream)
        md.step(p, v, args.steady_steps, 1.0)
        e1.record(stream)
        torch.cuda.synchronize()
        md.sync_status()
        ms_s = e0.elapsed_time(e1) / args.steady_steps
        rb_s = md.rebuild_count() - r_s0
        steady = {"first_step": W + K + args.steady_skip, "steps": args.steady_steps, "ms_per_step": ms_s,
                  "atom_steps_per_s": n / (ms_s / 1e3), "list_rebuilds": rb_s,
                  "rebuilds_per_step": rb_s / args.steady_steps}
        # the cost of one rebuild on the molten state: a phase-timed stretch
        # (kernels launched one by one), its list time net of the gated list
        # launches of the steps without a rebuild (their cost per step taken
        # from the crystal phase pass when that had no rebuild)
        model.profile_read()
        model.profile(True)
        r_p0 = md.rebuild_count()
        md.step(p, v, args.steady_phase_steps, 1.0)
        torch.cuda.synchronize()
        model.profile(False)
        prof_m = model.profile_read()
        rb_p = md.rebuild_count() - r_p0
        steady["phase_ms_per_step"] = {k: v_[0] / args.steady_phase_steps for k, v_ in prof_m.items()}
        steady["phase_steps"] = args.steady_phase_steps
        steady["phase_list_rebuilds"] = rb_p
        if rebuilds_phase == 0 and rb_p > 0:
            gate = prof["neighbor"][0] / K
            steady["list_gate_ms_per_step"] = gate
            steady["list_ms_per_rebuild"] = (prof_m["neighbor"][0] - gate * (args.steady_phase_steps - rb_p)) / rb_p

    t_max, e2e_s = max_over_ranks([ms, e2e_s], dist, "cuda")
    value = job_throughput(world, n, K, t_max)

    flops_atom = flops_per_atom(m_r, m_a, hyper.n_neu)
    achieved = flops_atom * n / (site_ms / 1e3) / 1e12
    peak = fp32_peak_tflops(2070.0)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "atoms": n, "md_steps_timed": K, "list_rebuilds_timed": rebuilds,
                       "l2": "inputs larger than L2 (per-step working set: positions, velocities, 96-slot "
                             "neighbour list, reverse index and partial forces ~340 MB > 129 MB)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "mean_neighbors_rcR": m_r, "mean_neighbors_rcA": m_a,
                       "mean_neighbors_start_end": [[m_r0, m_a0], [m_r1, m_a1]],
                       "phase_ms_per_step": {k: v[0] / K for k, v in prof.items()},
                       "list_rebuilds_phase_pass": rebuilds_phase,
                       "energy_drift_eV_per_atom": float(np.abs(etot - etot[0]).max() / n)},
            "steady_state": steady,
            "roofline": {"kernel": "k_site (descriptors + network + partial forces)", "bound": "alu",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": site_dram_traffic(), "traffic_unit": "bytes per launch (ncu dram read + write)",
                         "flops_per_atom": flops_atom, "kernel_ms": site_ms,
                         "kernel_share_of_step": prof["site"][0] / t_max if t_max > 0 else None,
                         "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop/FMA x 2070 MHz (fp32 pipe, derived)"},
            "clocks": clocks,
            "e2e": {"value": world * n * Ke / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(state.numel() * 8),
                    "d2h_bytes_per_step": int(state.numel() * 8 + N.THERMO_COLS * 8),
                    "steps": Ke},
            # per replayed step: kick-drift (with the rebuild decision), site,
            # assembly, finish; per rebuild the six list kernels of the
            # conditional body (bin, scan, scatter, half-shell search, row
            # sort, reverse index)
            "gpu_launches": 4 * K + 6 * rebuilds,
            "measured_peaks": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")} if peaks else None,
        }
        line["force_eval_vs_plain_fp32"] = force_eval_comparison(N, model, p0, box)
        line["md_step_vs_plain_fp32"] = md_vs_plain(N, model, p_w, v_w, box)
        line["config1_latency"] = config1_latency(N)
        line["config3_heat_transport_md"] = config3_md(N)
        line["pbte_split_model"] = pbte_split_model(N)
        v0 = torch.tensor(vel.T.copy(), dtype=torch.float64, device="cuda")
        line["md_nvt_hnemd"] = md_nvt_hnemd(N, model, p0, v0, box)
        adj = adjoint_gradients(N)
        line["snes"] = {"fp32": snes_generations(N, N.PREC_FP32), "bf16": snes_generations(N, N.PREC_BF16),
                        "unit": "generation/s",
                        "workload": "200 periodic structures of 32-256 atoms, population 50, 32-30-1 NEP"}
        adj["vs_one_fp32_generation"] = adj["ms_per_gradient"] / line["snes"]["fp32"]["ms_per_generation"]
        line["adjoint"] = adj
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_oracle_md(seconds=args.cpu_seconds)
        print(json.dumps(line), flush=True)
    md.close()
    model.close()
    if dist:
        dist.destroy_process_group()
    return 0


def md_nvt_hnemd(N, model, pos, vel, box, steps: int = 200, warm: int = 5):
    """The same 125k-atom state under a Berendsen thermostat (300 K, tau =
    100 fs) with HNEMD driving F_e = (1e-4, 0, 0) /A, heat current every
    step: atom-step/s of the heat-transport variant of the MD step."""
    import torch
    n = pos.shape[1]
    md = N.MD(model, n, box, inputs.MASS_SI)
    md.set_thermostat(300.0, 100.0)
    md.set_hnemd([1e-4, 0.0, 0.0])
    p, v = pos.clone(), vel.clone()
    thermo = torch.zeros(max(steps, warm), N.THERMO_COLS, dtype=torch.float64, device="cuda")
    heat = torch.zeros(max(steps, warm), 3, dtype=torch.float64, device="cuda")
    md.step(p, v, warm, 1.0, thermo, heat)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    md.step(p, v, steps, 1.0, thermo, heat)
    e1.record(stream)
    torch.cuda.synchronize()
    md.sync_status()
    ms = e0.elapsed_time(e1) / steps
    th = thermo[:steps].cpu().numpy()
    T = 2 * th[:, 1] / ((3 * n - 3) * inputs.KB_EV)
    md.close()
    return {"atom_steps_per_s": n / (ms / 1e3), "ms_per_step": ms, "steps_timed": steps,
            "temperature_K_last": float(T[-1]), "mean_heat_current_x": float(heat[:steps, 0].mean().item())}


def neighbour_counts(model, pos, box, hyper):
    """Mean number of neighbours within r_c^R and r_c^A per atom of the state
    `pos` (CUDA (3, n) FP64), from the list the library builds for it."""
    import torch
    n = pos.shape[1]
    model.compute(pos, box)
    cnt, nbr = model.neighbors(n)
    j = (nbr & 0xFFFFFF).long()
    code = (nbr >> 24).long()
    valid = torch.arange(nbr.shape[0], device="cuda")[:, None] < cnt[None, :]
    L = torch.tensor(np.diag(box), device="cuda")
    wrapped = pos - L[:, None] * torch.floor(pos / L[:, None])
    shifts = torch.stack([code // 25 - 2, (code // 5) % 5 - 2, code % 5 - 2]).double() * L[:, None, None]
    jj = j.clamp(max=n - 1)
    r = wrapped[:, jj] + shifts - wrapped[:, None, :]
    d = torch.linalg.norm(r, dim=0)
    m_r = float(((d < hyper.rc_R) & valid).sum()) / n
    m_a = float(((d < hyper.rc_A) & valid).sum()) / n
    return m_r, m_a


def force_eval_comparison(N, model, pos, box, reps: int = 10):
    """One force evaluation (list build, site pass, assembly, reductions) of
    the 125k-atom state through nep_compute_efv and through the plain FP32
    comparator nep_compute_efv_plain (literal O(M^2) angular sum, unfused,
    uncompensated), CUDA events on the current stream."""
    import torch
    stream = torch.cuda.current_stream()
    out = {}
    for name, plain in (("optimised", False), ("plain_fp32", True)):
        for _ in range(2):
            model.compute(pos, box, plain=plain, sync=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            model.compute(pos, box, plain=plain, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        model.sync_status()
        out[name] = e0.elapsed_time(e1) / reps
    n = pos.shape[1]
    return {"unit": "ms per force evaluation", "atoms": n, "optimised_ms": out["optimised"],
            "plain_fp32_ms": out["plain_fp32"], "speedup_vs_plain": out["plain_fp32"] / out["optimised"],
            "evaluations_timed": reps}


def md_vs_plain(N, model, pos, vel, box, steps: int = 100, warm: int = 3):
    """MD steps of the 125k-atom workload from the same warmed-up state with
    the optimised force pass and with the plain FP32 comparator
    (nep_md_set_force_form): list, assembly, integrator and heat current are
    shared, only the site pass differs.  CUDA events on the current stream;
    each form's handle replays its own captured step graph."""
    import torch
    n = pos.shape[1]
    stream = torch.cuda.current_stream()
    out = {"unit": "ms per MD step", "atoms": n, "steps_timed": steps}
    for name, plain in (("optimised", False), ("plain_fp32", True)):
        md = N.MD(model, n, box, inputs.MASS_SI)
        md.set_force_form(plain)
        p, v = pos.clone(), vel.clone()
        heat = torch.zeros(max(steps, warm), 3, dtype=torch.float64, device="cuda")
        md.step(p, v, warm, 1.0, None, heat)
        r0 = md.rebuild_count()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        md.step(p, v, steps, 1.0, None, heat)
        e1.record(stream)
        torch.cuda.synchronize()
        md.sync_status()
        ms = e0.elapsed_time(e1) / steps
        out[f"{name}_ms_per_step"] = ms
        out[f"{name}_atom_steps_per_s"] = n / (ms / 1e3)
        out[f"{name}_list_rebuilds"] = md.rebuild_count() - r0
        md.close()
    out["speedup_vs_plain"] = out["plain_fp32_ms_per_step"] / out["optimised_ms_per_step"]
    return out


def config3_md(N, steps: int = 50, warm: int = 5):
    """The heat-transport workload: 921,600 atoms (40 x 40 x 80 diamond cells,
    10 % vacancies, sigma = 0.15 A, 300 K), NVE with the heat current
    J = sum_i W_i . v_i accumulated in FP64 every step; a bounded window of
    `steps` steps after `warm`, from the captured step graph.  Device memory
    of the MD handle from cudaMemGetInfo around its creation and first steps
    (the state tensors are allocated before)."""
    import torch
    pos, vel, box, z = inputs.config3()
    n = len(pos)
    model = N.NEP(np.asarray(z, np.float32))
    p = torch.tensor(pos.T.copy(), dtype=torch.float64, device="cuda")
    v = torch.tensor(vel.T.copy(), dtype=torch.float64, device="cuda")
    thermo = torch.zeros(max(steps, warm), N.THERMO_COLS, dtype=torch.float64, device="cuda")
    heat = torch.zeros(max(steps, warm), 3, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    md = N.MD(model, n, box, inputs.MASS_SI)
    md.step(p, v, warm, 1.0, thermo, heat)
    torch.cuda.synchronize()
    lib_bytes = free0 - torch.cuda.mem_get_info()[0]
    r0 = md.rebuild_count()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("md_config3_timed")
    e0.record(stream)
    md.step(p, v, steps, 1.0, thermo, heat)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    md.sync_status()
    ms = e0.elapsed_time(e1) / steps
    J = heat[:steps].cpu().numpy()
    m_cap = N.Hyper().max_neighbors
    out = {"workload": "heat-transport NVE MD, 921,600 atoms (40x40x80 diamond cells, 10% vacancies, "
                       "sigma 0.15 A, 300 K), J = sum W_i . v_i every step in FP64, dt 1 fs",
           "atoms": n, "atom_steps_per_s": n / (ms / 1e3), "ms_per_step": ms, "steps_timed": steps,
           "warmup": warm, "list_rebuilds_timed": md.rebuild_count() - r0, "heat_current_finite": bool(np.isfinite(J).all()),
           "device_bytes": int(lib_bytes), "device_bytes_per_atom": lib_bytes / n,
           "paper_memory_model_bytes_per_atom": 36 * m_cap + 2000,
           "paper_memory_model": "12 N M + 24 N M + 2000 N bytes (Sec. III.C), with M = this build's 96 slots"}
    md.close()
    model.close()
    return out


def pbte_split_model(N, reps: int = 10, md_steps: int = 50, warm: int = 3):
    """The split-hyperparameter model of the paper's PbTe potential (r_c^R = 8 A,
    n_max^R = 12; r_c^A = 4 A, n_max^A = 6; l_max = 4; 41-40-1 network) on a
    two-species rocksalt box of 25^3 cells (125,000 atoms, a = 6.46 A, sigma =
    0.1 A, weights sqrt(Z_i Z_j) with Z = 82, 52): one force evaluation
    through nep_compute_efv (list, site pass, assembly, reductions) and NVE MD
    steps (one mass, 1 A skin), CUDA events on the current stream."""
    import torch
    pos, vel, box, z, Z = inputs.config_pbte((25, 25, 25))
    n = len(pos)
    hyper = N.Hyper(max_neighbors=128, **inputs.PBTE_HYPER)
    model = N.NEP(np.asarray(z, np.float32), hyper)
    model.set_species(Z)
    p = torch.tensor(pos.T.copy(), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        model.compute(p, box, sync=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        model.compute(p, box, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    model.sync_status()
    ms_eval = e0.elapsed_time(e1) / reps
    model.close()
    hyper_md = N.Hyper(max_neighbors=160, **inputs.PBTE_HYPER)
    model = N.NEP(np.asarray(z, np.float32), hyper_md)
    model.set_species(Z)
    md = N.MD(model, n, box, inputs.MASS_PBTE)
    v = torch.tensor(vel.T.copy(), dtype=torch.float64, device="cuda")
    p = torch.tensor(pos.T.copy(), dtype=torch.float64, device="cuda")
    md.step(p, v, warm, 1.0)
    r0 = md.rebuild_count()
    torch.cuda.synchronize()
    e0.record(stream)
    md.step(p, v, md_steps, 1.0)
    e1.record(stream)
    torch.cuda.synchronize()
    md.sync_status()
    ms_md = e0.elapsed_time(e1) / md_steps
    out = {"workload": "PbTe-like rocksalt, 125,000 atoms (25^3 cells, a 6.46 A, sigma 0.1 A), two species "
                       "weighted sqrt(Z_i Z_j), NEP 41-40-1 (r_c^R 8 A, n_max^R 12; r_c^A 4 A, n_max^A 6)",
           "atoms": n, "force_eval_ms": ms_eval, "force_evals_per_s": 1e3 / ms_eval,
           "md_ms_per_step": ms_md, "md_atom_steps_per_s": n / (ms_md / 1e3), "md_steps_timed": md_steps,
           "md_list_rebuilds": md.rebuild_count() - r0}
    md.close()
    model.close()
    return out


def config1_latency(N, reps: int = 200, warm: int = 10):
    """One call of nep_compute_efv on the 512-atom configuration (4^3 diamond
    cells, sigma = 0.1 A): list build, site pass, assembly and reductions.
    Device time per call (CUDA events over back-to-back calls), host time per
    call with a synchronize after each (what a caller waiting for every result
    sees), and end to end with the positions copied in from pinned host memory
    and energy and forces copied back every call."""
    import torch
    pos, box, z = inputs.config1()
    n = len(pos)
    model = N.NEP(np.asarray(z, np.float32))
    p = torch.tensor(pos.T.copy(), dtype=torch.float64, device="cuda")
    outs = [torch.empty(1, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.float64, device="cuda"),
            torch.empty(3, n, dtype=torch.float32, device="cuda"), torch.empty(9, n, dtype=torch.float32, device="cuda"),
            torch.empty(9, dtype=torch.float64, device="cuda")]
    _, bp = N._box9(box)
    stream = torch.cuda.current_stream()
    args = (model._h, n, bp, N._ptr(p), *[N._ptr(t) for t in outs], N._vp(stream.cuda_stream))

    def call():
        rc = N._lib.nep_compute_efv(*args)
        if rc != 0:
            raise RuntimeError(f"nep_compute_efv failed: {rc}")
    for _ in range(warm):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    dev_us = 1e3 * e0.elapsed_time(e1) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        call()
        torch.cuda.synchronize()
    host_us = 1e6 * (time.perf_counter() - t0) / reps
    hp = p.cpu().pin_memory()
    he = torch.empty(1, dtype=torch.float64).pin_memory()
    hf = torch.empty(3, n, dtype=torch.float32).pin_memory()
    t0 = time.perf_counter()
    for _ in range(reps):
        p.copy_(hp, non_blocking=True)
        call()
        he.copy_(outs[0], non_blocking=True)
        hf.copy_(outs[2], non_blocking=True)
        torch.cuda.synchronize()
    e2e_us = 1e6 * (time.perf_counter() - t0) / reps
    model.sync_status()
    model.close()
    return {"workload": "512-atom diamond (4^3 cells, sigma 0.1 A), one energy + force + virial call", "atoms": n,
            "device_us_per_call": dev_us, "host_us_per_call_synchronised": host_us,
            "e2e_us_per_call": e2e_us, "e2e_h2d_bytes": int(p.numel() * 8),
            "e2e_d2h_bytes": int(8 + outs[2].numel() * 4), "calls_timed": reps}


def training_set(N):
    """The 200-structure training workload on the device, labelled by the CUDA
    force path with the teacher (a timing input, not a checked value)."""
    import torch
    structures, teacher, pop = inputs.config4()
    model = N.NEP(np.asarray(teacher, np.float32))
    E, F, W = [], [], []
    for s in structures:
        out = model.compute(torch.tensor(s["pos"].T.copy(), dtype=torch.float64, device="cuda"), s["box"])
        wt = out["virial_total"].cpu().numpy().reshape(3, 3)
        E.append(out["e_total"].item())
        F.append(out["force"].cpu().numpy().T)
        W.append([wt[0, 0], wt[1, 1], wt[2, 2], wt[0, 1], wt[1, 2], wt[2, 0]])
    ds = N.Dataset(model, structures, np.array(E), np.concatenate(F), np.array(W))
    return model, ds, structures, pop


def adjoint_gradients(N, reps: int = 20, warm: int = 3):
    """Force-loss gradient of one parameter vector on the same training set:
    nep_force_loss + nep_force_loss_backward (descriptors recomputed in both),
    CUDA events on the current stream."""
    import torch
    model, ds, structures, pop = training_set(N)
    z = torch.tensor(np.asarray(pop[0], np.float32), device="cuda")
    for _ in range(warm):
        ds.force_loss(z)
        ds.force_loss_backward()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("adjoint_timed")
    e0.record(stream)
    for _ in range(reps):
        ds.force_loss(z)
        ds.force_loss_backward()
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    model.sync_status()
    ms = e0.elapsed_time(e1) / reps
    ds.close()
    model.close()
    return {"ms_per_gradient": ms, "gradients_per_s": 1e3 / ms, "n_par": model.hyper.n_par,
            "gradients_timed": reps}


def snes_generations(N, precision: int, gens: int = 20, warm: int = 3, shape=None):
    """SNES on the 200-structure training workload, population 50: one
    generation = draws + population evaluation + update, on the device.  The
    launch shape is picked by the library's autotuner, or given (`shape`, a
    dict of Dataset.SHAPE_KEYS: profiler captures use a fixed one); the timed
    loop is snes_run (one captured generation replayed), with the eager
    snes_step loop timed beside it."""
    import torch
    model, ds, structures, pop = training_set(N)
    info = ds.info()
    if shape is None:
        shape, tune_ms = ds.tune(50, precision, reps=3)
    else:
        ds.set_shape(**shape)
        shape, tune_ms = ds.shape(), None
    snes = N.SNES(model, 50, np.zeros(model.hyper.n_par), np.full(model.hyper.n_par, 0.1), seed=2107081194)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, label):
        fn(warm)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(label)
        e0.record(stream)
        fn(gens)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / gens

    tag = "bf16" if precision == N.PREC_BF16 else "fp32"
    counts = ds.counts()
    ms = timed(lambda n: snes.run(ds, n, precision), f"snes_{tag}_graph")

    def eager(n):
        for _ in range(n):
            snes.step(ds, precision)
    ms_eager = timed(eager, f"snes_{tag}_eager")
    snes.close()
    ds.close()
    model.close()
    return {"generations_per_s": 1e3 / ms, "ms_per_generation": ms, "ms_per_generation_eager": ms_eager,
            "shape": shape, "tuned_ms_per_evaluation": tune_ms, "atoms": info["atoms"], "pairs": info["pairs"],
            "angular_pairs": counts["angular_pairs"], "population": 50, "structures": len(structures),
            "generations_timed": gens,
            "roofline": snes_roofline(counts, 50, model.hyper.n_neu, precision == N.PREC_BF16, ms, tag)}


SNES_SOURCES = ("paper_2107_08119_gb300/csrc/nep_train.cu", "paper_2107_08119_gb300/csrc/nep_pop_tc.cu",
                "paper_2107_08119_gb300/csrc/nep_tc.cuh", "paper_2107_08119_gb300/csrc/nep_dataset.cuh",
                "paper_2107_08119_gb300/csrc/nep_internal.cuh", "paper_2107_08119_gb300/csrc/nep_recv.cuh",
                "paper_2107_08119_gb300/csrc/nep_philox.cuh")
SNES_PROFILE = os.path.join(ROOT, "profiles", "snes_generation_dram_200structs.json")


def snes_roofline(c, P: int, n_neu: int, tensor: bool, ms: float, tag: str):
    """Roofline of one SNES generation (population evaluation; the draws,
    ranking and update are O(P N_par) and left out).  Two phases, each bound
    by its own roof, t_roof = sum over phases of max(flops / pipe peak,
    algorithmic bytes / HBM bandwidth):
      network     4 N P 32 N_neu flops (H = Q W1^T and G = D W1, 2 flops per
                  multiply-add) on the BF16 tensor pipe (FP32 pipe in FP32
                  mode); bytes: descriptors in (N 32 x 2 B), parameters in,
                  G out at 2 B per value, U out (N P x 8 B);
      contraction P (31 n_pairs + 144 n_ang + 192 N) flops on the FP32 pipe
                  (per pair: 8 radial multiply-adds, 3 products, 6 virial
                  multiply-adds; per angular pair 72 multiply-adds; per atom
                  the own term, 96); bytes: the Jacobian records (48 B per
                  pair, 288 B per angular pair, 384 B per atom), G and U in,
                  targets and pair indices.
    `achieved_fraction` = t_roof / the measured generation time.  `traffic`:
    DRAM bytes (read + write) of one generation's kernels from the committed
    ncu capture, while the digest of the sources matches."""
    N, npairs, nang = c["atoms"], c["pairs"], c["angular_pairs"]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs") or 6800.0) * 1e9
    bf16_peak = float(peaks.get("bf16_tflops") or 1900.0) * 1e12
    fp32 = fp32_peak_tflops(2070.0) * 1e12
    n_par = (32 + 2) * n_neu + 1
    f_net = 4.0 * N * P * 32 * n_neu
    b_net = N * 32 * 2 + P * n_par * 4 + N * 32 * P * 2 + N * P * 8
    f_con = P * (31.0 * npairs + 144.0 * nang + 192.0 * N)
    b_con = 48 * npairs + 288 * nang + 384 * N + N * 32 * P * 2 + N * P * 8 + 12 * N + 12 * npairs + 8 * N
    t_net = max(f_net / (bf16_peak if tensor else fp32), b_net / hbm)
    t_con = max(f_con / fp32, b_con / hbm)
    t_roof = t_net + t_con
    traffic = None
    try:
        prof = json.load(open(SNES_PROFILE))
        if prof.get("sources_sha256") == sources_digest(SNES_SOURCES):
            traffic = prof.get("dram_bytes_per_generation", {}).get(tag)
    except (OSError, ValueError):
        pass
    return {"bound": "tensor+alu" if tensor else "alu", "t_roof_us": 1e6 * t_roof,
            "achieved_fraction": t_roof / (ms / 1e3),
            "network": {"flops": f_net, "bytes": b_net, "roof_us": 1e6 * t_net,
                        "peak": "bf16 tensor (measured burst)" if tensor else "fp32 pipe (derived)"},
            "contraction": {"flops": f_con, "bytes": b_con, "roof_us": 1e6 * t_con, "peak": "fp32 pipe (derived)"},
            "algorithmic_bytes": b_net + b_con, "traffic": traffic,
            "traffic_over_algorithmic": traffic / (b_net + b_con) if traffic else None,
            "peaks": {"hbm_gbs": hbm / 1e9, "bf16_tflops": bf16_peak / 1e12, "fp32_tflops": fp32 / 1e12}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--steady-skip", type=int, default=500,
                    help="MD steps after the timed window before the steady-state window")
    ap.add_argument("--steady-steps", type=int, default=200, help="MD steps of the steady-state window (0: none)")
    ap.add_argument("--steady-phase-steps", type=int, default=30,
                    help="phase-timed MD steps after the steady-state window (the cost of one rebuild)")
    ap.add_argument("--only", default="all", choices=["all", "md", "snes"],
                    help="md: the timed MD steps alone (no e2e, SNES or CPU legs); snes: the SNES legs alone. "
                         "Small single-purpose runs for profiler captures.")
    ap.add_argument("--snes-shape", default=None,
                    help="with --only snes: a fixed launch shape as JSON (Dataset.SHAPE_KEYS) instead of the "
                         "autotuner's, so that profiler captures run one known shape")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.only == "snes":
        return run_snes_only(json.loads(args.snes_shape) if args.snes_shape else None)
    return run_gpu(args, rank, world, local)


def run_snes_only(shape=None):
    import torch  # noqa: F401
    from paper_2107_08119_gb300 import build
    build.build()
    from paper_2107_08119_gb300 import nep as N
    out = {"fp32": snes_generations(N, N.PREC_FP32, shape=shape), "bf16": snes_generations(N, N.PREC_BF16, shape=shape)}
    adj = adjoint_gradients(N)
    print(json.dumps({"snes": out, "adjoint": adj}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
