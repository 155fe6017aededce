#!/usr/bin/env python
"""Benchmark of the FAS multigrid hot path on one B300 (or N replicas).

Workload (one "step" = one FAS V-cycle over the whole hierarchy, Alg. 2): the
large curvilinear run, Poisson on [0,1]^3 with Dirichlet conditions, 64^3
trilinear elements with interior vertices perturbed by +-0.15h, p = 7
(134M DoF), seeded 16-mode right-hand side; p-multigrid 7 -> 3 -> 1 with the
Schwarz-preconditioned CG smoother (Alg. 6, V(2,2), n_sc = 4) and an FP64 SCG
root solve at p = 1.  Headline: mixed precision plus learned surrogate -- the
smoother in correction form on FP32 vectors with the fast-diagonalization
mode products on the tensor cores (BF16 operands, FP32 accumulation), the
learned MLP surrogate on the p = 7 and p = 3 levels, the V-cycle replayed as a
CUDA graph -- with FP64 residual, tau, restriction and root.  Beside it: the
plain FP64 GPU path and the geometric surrogate (DoF/s per V-cycle and time
to 1e-10), the graded curvilinear, uniform Cartesian and locally refined
workloads, and the FP64 oracle on the host cores.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead
(on a bounded sample of the same workload).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2608_14123_b300 import workloads as wl  # noqa: E402

METRIC = "DoF/s per FAS V-cycle and time-to-1e-10 residual, mixed+learned vs FP64, 1 B300"
UNIT = "DoF/s"
L2_BYTES = 126 * 2 ** 20


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return dict(hbm=float(d.get("hbm_gbs", 6400.0)), src="measured", raw=d)
    return dict(hbm=6400.0, src="fallback", raw=None)


def apply_flops_per_dof(N, box=True):
    """Algorithmic FP64 flops per DoF of the SIP apply (Eq. (2)) as the kernels
    evaluate it.  Box elements (Kronecker form): volume 3 N FMA plus 5
    operations per node; faces: 6 N^2 face nodes per element, each with the own
    and the neighbour's normal derivative and the lifting along the normal
    line (3 N FMA) and about 12 operations of flux.  Curvilinear elements:
    gradient and transposed gradient (6 N FMA) and the 3 x 3 metric."""
    if box:
        vol = 2 * 3 * N + 5
    else:
        vol = 2 * 6 * N + 18
    face = 6 * N * N * (2 * 3 * N + 12) / N ** 3
    return vol + face


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel, from one ncu capture of the current kernels on a 16^3,
# p = 7 curvilinear case (2,097,152 DoF, vectors and geometry larger than L2:
# k_curv_grad 155.2 + 45.4 MB, k_curv_div 142.9 + 4.5 MB), scaled by the DoF
# of the 64^3 level (x 64; the per-element data grow in proportion); to be
# retaken whenever the kernels change
NCU_TRAFFIC = {"residual_fp64": int((155234560 + 45440768 + 142932480 + 4498688) * 64)}


def fd_flops_per_dof(N, m):
    ns = N + 2 * m
    return 12.0 * ns ** 4 / N ** 3


class _CtypesNvml:
    """The four NVML queries the clock sampler needs, through ctypes on the
    driver's libnvidia-ml (read-only queries; nothing is set)."""

    def __init__(self):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        rc = self.lib.nvmlInit_v2()
        if rc != 0:
            raise RuntimeError(f"nvmlInit_v2 returned {rc}")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def _handle(self, fn, arg):
        h = self.ct.c_void_p()
        rc = fn(arg, self.ct.byref(h))
        if rc != 0:
            raise RuntimeError(f"NVML handle lookup returned {rc}")
        return h

    def handle_by_uuid(self, uuid):
        return self._handle(self.lib.nvmlDeviceGetHandleByUUID, uuid.encode())

    def handle_by_index(self, i):
        return self._handle(self.lib.nvmlDeviceGetHandleByIndex_v2, self.ct.c_uint(i))

    def _clock(self, fn, h):
        v = self.ct.c_uint()
        rc = fn(h, self.ct.c_int(1), self.ct.byref(v))   # NVML_CLOCK_SM = 1
        if rc != 0:
            raise RuntimeError(f"NVML clock query returned {rc}")
        return v.value

    def sm_clock(self, h):
        return self._clock(self.lib.nvmlDeviceGetClockInfo, h)

    def max_sm_clock(self, h):
        return self._clock(self.lib.nvmlDeviceGetMaxClockInfo, h)

    def event_reasons(self, h):
        v = self.ct.c_ulonglong()
        rc = self.reasons_fn(h, self.ct.byref(v))
        if rc != 0:
            raise RuntimeError(f"NVML reasons query returned {rc}")
        return v.value


class ClockSampler:
    """SM clocks and clock-event reasons sampled DURING the timed region.

    NVML is polled from a background thread every 5 ms (the timed region of the
    default run is well under a second, too short for nvidia-smi's loop);
    nvidia-smi is the fallback when the NVML library cannot be loaded."""
    # clock-event reason bits (nvml.h): sw power cap, hw slowdown,
    # sw thermal slowdown, hw thermal slowdown
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
            "hw_thermal_slowdown": 0x40}

    def __init__(self, device):
        self.sm, self.mx, self.reasons = [], [], set()
        self.stop_ev = threading.Event()
        self.thread = self.proc = self.fh = None
        self.err = None
        try:
            self.nv = _CtypesNvml()
            import torch
            try:
                uuid = str(torch.cuda.get_device_properties(device).uuid)
                self.h = self.nv.handle_by_uuid(uuid if uuid.startswith("GPU-") else "GPU-" + uuid)
            except Exception:   # noqa: BLE001 - fall back to the ordinal
                self.h = self.nv.handle_by_index(device)
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
        except Exception as ex:   # noqa: BLE001 - any NVML failure falls back to nvidia-smi
            self.nv = None
            self.err = f"{type(ex).__name__}: {ex}"[:200]
            self._start_smi(device)

    def _poll(self):
        nv = self.nv
        mx = nv.max_sm_clock(self.h)
        while not self.stop_ev.is_set():
            try:
                self.sm.append(float(nv.sm_clock(self.h)))
                self.mx.append(float(mx))
                bits = nv.event_reasons(self.h)
                for nm, b in self.BITS.items():
                    if bits & b:
                        self.reasons.add(nm)
            except Exception:   # noqa: BLE001 - a failed sample is skipped
                pass
            self.stop_ev.wait(0.005)

    def _start_smi(self, device):
        try:
            self.fh = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            self.dev = device
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_ev.set()
            self.thread.join(timeout=2)
            src = "nvml (ctypes), 5 ms"
        elif self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.flush()
            self.fh.seek(0)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for line in self.fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9 or parts[0] != str(self.dev):
                    continue
                try:
                    self.sm.append(float(parts[1]))
                    self.mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        self.reasons.add(nm)
            os.unlink(self.fh.name)
            src = "nvidia-smi, 100 ms"
        else:
            return None
        if not self.sm:
            return None
        out = dict(sm_mhz=float(np.median(self.sm)), sm_max_mhz=float(max(self.mx)),
                   reasons=sorted(self.reasons), samples=len(self.sm), source=src)
        if self.err:
            out["nvml_error"] = self.err
        return out


def level_rhs(S, cfg, torch):
    """Each level's own assembled right-hand side (the FMG inputs)."""
    out = []
    for l in range(S.n_levels):
        xyz = S.node_coords(l)
        fn = torch.from_numpy(wl.eval_f(cfg["rhs"], xyz.cpu().numpy())).to(xyz.device)
        bl = torch.empty_like(fn)
        S.dgfas_assemble_rhs_level(l, fn, None, bl)
        out.append(bl)
        del xyz, fn
    return out


def max_over_ranks(value, device):
    """The largest per-rank value (the job's time is the slowest rank's)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ CPU oracle arm
def oracle_sample_rate(n_sample=8, cycles=1):
    """DoF/s per V-cycle of the FP64 oracle on a bounded sample of the headline
    workload: the same degree, perturbation, p-hierarchy (7 -> 3 -> 1), SCG
    smoother and SCG root on n_sample^3 elements (the oracle is never tuned)."""
    from oracle import fas, sip
    rng = np.random.default_rng(wl.SEED_BASE + 5)
    V = wl.perturbed_vertices(n_sample, 0.15, rng)
    levels = wl.hierarchy(V, [7, 3, 1])
    spec = wl.modes_rhs_spec(rng)
    H = fas.Hierarchy(levels, 5.0, 0.08, 2, 2, 4, smoother="scg", coarse="scg", root_rtol=1e-3,
                      root_steps=64)
    top = H.ops[-1]
    X = top.geo["x"]
    b = sip.rhs(top, wl.eval_f(spec, X), np.zeros(X.shape[:-1])).reshape(-1)
    u = H.zero_levels(wl.random_start(rng, top.ndof))
    t0 = time.perf_counter()
    for _ in range(cycles):
        u, _ = H.fas_vcycle(u, b)
    dt = time.perf_counter() - t0
    return top.ndof * cycles / dt, dt, top.ndof


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    n_sample = 8
    rates = []
    t_all = time.perf_counter()
    for _ in range(args.warmup):
        oracle_sample_rate(n_sample=n_sample)
    for _ in range(args.steps):
        r, dt, ndof = oracle_sample_rate(n_sample=n_sample)
        rates.append(r)
    value = float(np.mean(rates))
    threads = int(os.environ.get("OMP_NUM_THREADS", host_cores()))
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ndof / value * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "curvilinear-64^3-p7 (trilinear, +-0.15h perturbation), 16-mode "
                               "RHS, Dirichlet Poisson (sampled at 8^3 elements)",
                   "global_batch": 1, "seq_len": 0, "parallelism": "replicas",
                   "sample_dof": ndof},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"one FP64 oracle V-cycle (SCG smoother and root) on "
                                   f"{n_sample}^3 elements p=7 ({ndof} DoF) per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t_all,
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ helpers of the GPU arm
SURR_SET = 100000
GOLD = os.path.join(ROOT, "tests", "golden")


def train_surrogates(torch, degrees=(7, 3), epochs=80):
    """The learned surrogate per degree: the MLP trained on the GPU by the
    library's kernels on the 10^5 oracle Kronecker-sum fits (stored targets;
    inputs regenerated from the seeded training elements by the library)."""
    from paper_2608_14123_b300 import learned
    out, info = {}, {}
    for p in degrees:
        d = np.load(os.path.join(GOLD, f"surrogate_fits_p{p}_n{SURR_SET}.npz"))
        cr = wl.surrogate_training_set(SURR_SET, p)[d["ok"]]
        X = learned.inputs(cr)
        Y = torch.from_numpy(d["Y"]).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        th, loss = learned.train(X, Y, epochs=epochs, batch=256, lr=2e-3, seed=11)
        torch.cuda.synchronize()
        out[p] = th
        info[p] = {"samples": int(X.shape[0]), "epochs": epochs, "seconds": time.perf_counter() - t0,
                   "loss_first": float(loss[0]), "loss_last": float(loss[-1])}
        del X, Y
    return out, info


def build_solver(dgfas, cfg, prec, smoother, surr=None):
    """Solver of workload cfg (set-up); surr: {degree: trained params} replaces
    the geometric surrogate on the levels of those degrees."""
    pr = cfg["params"]
    kw = {}
    if pr.get("coarse") == "scg":
        kw = dict(coarse=dgfas.DGFAS_COARSE_SCG, root_rtol=pr["root_rtol"],
                  root_steps=pr["root_steps"])
    S = dgfas.Solver(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"],
                     precision=prec, smoother=smoother, **kw)
    fallback = {}
    if surr:
        for l in range(1, S.n_levels):
            p = cfg["levels"][l]["p"]
            if p in surr:
                fallback[l] = S.dgfas_learned_surrogate(l, surr[p])
    return S, fallback


def top_rhs(S, cfg, torch, dev):
    xyz = S.node_coords(-1)
    f = torch.from_numpy(wl.eval_f(cfg["rhs"], xyz.cpu().numpy())).to(dev)
    del xyz
    b = torch.empty_like(f)
    S.dgfas_assemble_rhs(f, None, b)
    del f
    return b


def time_vcycles(S, u, b, steps, warmup, torch, dgfas, ws=1, dev=None, clocks=False):
    """ms per FAS V-cycle over `steps` cycles after `warmup` (CUDA events on the
    current stream, which the library's graph replays are ordered on)."""
    for _ in range(warmup):
        S.dgfas_fas_vcycle(u, b, want_norm=False)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = ClockSampler(dev.index if dev is not None else 0) if clocks else None
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    k0 = dgfas.dgfas_kernel_launches()
    torch.cuda.nvtx.range_push("timed")
    e0.record()
    for _ in range(steps):
        S.dgfas_fas_vcycle(u, b, want_norm=False)
    e1.record()
    torch.cuda.nvtx.range_pop()
    launches = dgfas.dgfas_kernel_launches() - k0
    torch.cuda.synchronize()
    ck = clk.stop() if clk else None
    return e0.elapsed_time(e1) / steps, launches, ck


def solve_record(S, u, b, torch, rtol=1e-10, max_cycles=40):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = S.dgfas_solve(u, b, rtol, max_cycles, raise_on_fail=False)
    torch.cuda.synchronize()
    if info["code"] != 0:
        print(f"bench: solve stopped with code {info['code']} after {info['cycles']} cycles "
              f"(relative residual {info['r_final'] / info['r0']:.3e})", file=sys.stderr)
    return {"seconds": time.perf_counter() - t0, "cycles": info["cycles"],
            "rel_residual": info["r_final"] / info["r0"], "code": info["code"],
            "history": [h / info["history"][0] for h in info["history"][1:]]}


def e2e_record(S, u0_host, b, torch, steps):
    """The metric end to end through the C ABI with host buffers: every step
    uploads u and f from pinned host memory and reads u back; two device
    buffer pairs and two copy streams overlap step k+1's upload and step
    k-1's download with step k's V-cycle (one captured graph per pair)."""
    u_host = u0_host.pin_memory()
    b_host = b.cpu().pin_memory()
    u_back = [torch.empty_like(u_host).pin_memory() for _ in range(2)]
    ud = [torch.empty_like(b) for _ in range(2)]
    bd = [torch.empty_like(b) for _ in range(2)]
    comp = torch.cuda.current_stream()
    s_h2d, s_d2h = torch.cuda.Stream(), torch.cuda.Stream()
    h2d_done = [torch.cuda.Event() for _ in range(2)]
    comp_done = [torch.cuda.Event() for _ in range(2)]
    d2h_done = [torch.cuda.Event() for _ in range(2)]

    def run(n):
        for k in range(n):
            i = k % 2
            with torch.cuda.stream(s_h2d):
                if k >= 2:
                    s_h2d.wait_event(d2h_done[i])
                ud[i].copy_(u_host, non_blocking=True)
                bd[i].copy_(b_host, non_blocking=True)
                h2d_done[i].record(s_h2d)
            comp.wait_event(h2d_done[i])
            S.dgfas_fas_vcycle(ud[i], bd[i], want_norm=False)
            comp_done[i].record(comp)
            with torch.cuda.stream(s_d2h):
                s_d2h.wait_event(comp_done[i])
                u_back[i].copy_(ud[i], non_blocking=True)
                d2h_done[i].record(s_d2h)

    run(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run(steps)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    n = b.numel()
    out = {"seconds_per_step": dt, "h2d_bytes_per_step": 2 * n * 8, "d2h_bytes_per_step": n * 8,
           "overlap": "double-buffered, 2 copy streams", "steps": steps}
    del ud, bd, u_back, u_host, b_host
    return out


# ------------------------------------------------------------------ other workloads
def config4_record(dgfas, torch):
    """Time to 1e-10 on the locally refined front (FP32 smoother vs FP64)."""
    c4 = wl.config4()
    pr = c4["params"]
    leaf = sum(int(np.sum(lv["cls"] == 0)) * (lv["p"] + 1) ** 3 for lv in c4["levels"])
    rec = {"leaf_dof": leaf, "levels": len(c4["levels"])}
    for name, prec in (("mixed_fp32", dgfas.DGFAS_FP32), ("fp64", dgfas.DGFAS_FP64)):
        S = dgfas.Solver(c4["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"],
                         precision=prec)
        L = S.n_levels - 1
        for l in range(S.n_levels):
            xyz = S.node_coords(l).cpu().numpy()
            fn = torch.from_numpy(wl.eval_front_f(c4["rhs"], xyz)).cuda()
            un = torch.from_numpy(wl.eval_front_u(c4["rhs"], xyz)).cuda()
            b = torch.empty_like(fn)
            S.dgfas_assemble_rhs_level(l, fn, un, b)
            if l < L:
                S.dgfas_set_level_rhs(l, b)
        rec[name] = solve_record(S, torch.from_numpy(c4["u0"]).cuda(), b, torch)
        S.close()
    return rec


def curvilinear_records(dgfas, torch, dev, cid, surr, arms):
    """Per arm (name, precision, surrogate) on workload cid: ms per V-cycle
    (3 graph replays) and time to 1e-10 from the random start."""
    cfg = wl.config(cid)
    pr = cfg["params"]
    rec = {"dof": int(cfg["u0"].size), "levels": [lv["p"] for lv in cfg["levels"]],
           "smoother": f"SCG (Alg. 6) ({pr['s1']}, {pr['s2']}, {pr['sc']}), mu_star = {pr['mu_star']}",
           "root": "p = 1 h-coarsened to 4^3, exact"}
    for name, prec, use in arms:
        S, fb = build_solver(dgfas, cfg, prec, dgfas.DGFAS_SCG, surr if use else None)
        S.dgfas_use_graph(True)
        b = top_rhs(S, cfg, torch, dev)
        u0 = torch.from_numpy(cfg["u0"]).to(dev)
        u = u0.clone()
        ms, _, _ = time_vcycles(S, u, b, 3, 1, torch, dgfas)
        r = solve_record(S, u0.clone(), b, torch, max_cycles=80)
        r["ms_per_vcycle"] = ms
        r["dof_per_s_per_vcycle"] = rec["dof"] / (ms * 1e-3)
        if use:
            r["fallback_elements"] = fb
        rec[name] = r
        S.close()
        del b, u, u0
        torch.cuda.empty_cache()
    return rec


def cartesian_record(dgfas, torch, dev, args):
    """The uniform Cartesian workload (32^3, p = 8, WAS, BF16 tensor-core
    smoother): ms per V-cycle, roofline of its FP64 residual, time to 1e-10."""
    cfg = wl.config(2)
    pr = cfg["params"]
    S = dgfas.Solver(cfg["levels"], pr["mu_star"], pr["delta"], pr["s1"], pr["s2"], pr["sc"],
                     precision=dgfas.DGFAS_BF16)
    S.dgfas_use_graph(True)
    if not args.no_autotune:
        S.dgfas_autotune(reps=5)
    b = top_rhs(S, cfg, torch, dev)
    u0 = torch.from_numpy(cfg["u0"]).to(dev)
    ms, _, _ = time_vcycles(S, u0.clone(), b, 10, 3, torch, dgfas)
    ndof = S.ndof(-1)
    N = cfg["levels"][-1]["p"] + 1
    prof = S.dgfas_profile_sweep(S.n_levels - 1, u0.clone(), b, 5)
    fp64_tf, _ = dgfas.dgfas_fma_peak()
    fl = (6 * N + 30) * ndof
    rec = {"dof": ndof, "ms_per_vcycle": ms, "dof_per_s_per_vcycle": ndof / (ms * 1e-3),
           "kernel_ms": prof,
           "residual_fp64_roofline": {"bound": "alu", "flops_per_dof": 6 * N + 30,
                                      "achieved_tflops": fl / (prof["residual_fp64"] * 1e-3) / 1e12,
                                      "peak_tflops": fp64_tf,
                                      "frac": fl / (prof["residual_fp64"] * 1e-3) / 1e12 / fp64_tf}}
    rec["time_to_1e-10_bf16"] = solve_record(S, u0.clone(), b, torch)
    S.close()
    return rec


# ------------------------------------------------------------------ GPU arm
def kernel_table(prof, ndof, N, ns, fp64_tf, hbm, counts):
    """Per-kernel algorithmic work, bound and measured time of one SCG step on
    the top curvilinear level (p = 7, n_s = 12), and per V-cycle counts.
    Algorithmic work per DoF (stated in the design notes):
      FP64 residual    12 N + 60 flop (FP64 pipe)
      FP32 operator    44 B: u, out, 6 metric factors, face factors (HBM)
      FD (BF16 tc)     4 B in + 4 (n_s / N)^3 B patch out (HBM)
      combine          4 (n_s / N)^3 B patch in + 4 B out (HBM)
      z.r + direction  24 B; p.q + update 36 B (FP32 vectors, HBM)."""
    patch = 4.0 * (ns / N) ** 3
    rows = {
        "residual_fp64": dict(ms=prof["residual_fp64"], bound="alu", work=(12 * N + 60) * ndof,
                              peak=fp64_tf, unit="TFLOP/s", scale=1e12),
        "apply_fp32": dict(ms=prof["apply_smoother"], bound="hbm", work=44.0 * ndof, peak=hbm,
                           unit="GB/s", scale=1e9),
        "fd_tc": dict(ms=prof["fd"], bound="hbm", work=(4.0 + patch) * ndof, peak=hbm,
                      unit="GB/s", scale=1e9),
        "combine": dict(ms=prof["combine"], bound="hbm", work=(patch + 4.0) * ndof, peak=hbm,
                        unit="GB/s", scale=1e9),
        "scg_zr_dir": dict(ms=prof["zr_dir"], bound="hbm", work=24.0 * ndof, peak=hbm,
                           unit="GB/s", scale=1e9),
        "scg_pq_update": dict(ms=prof["pq_update"], bound="hbm", work=36.0 * ndof, peak=hbm,
                              unit="GB/s", scale=1e9),
    }
    for k, v in rows.items():
        v["count_per_vcycle"] = counts.get(k, 0)
        v["achieved"] = v["work"] / (v["ms"] * 1e-3) / v["scale"]
        v["frac"] = v["achieved"] / v["peak"]
    return rows


def run_gpu(args):
    import torch
    from paper_2608_14123_b300 import dgfas

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t_start = time.perf_counter()

    # ---- set-up (outside every timed region): the learned surrogate trained on
    # the GPU from the oracle's 10^5 fits, the solver, the right-hand side
    surr, train_info = train_surrogates(torch)
    cfg = wl.config(5)
    levels = cfg["levels"]
    top = levels[-1]
    N = top["p"] + 1
    prec = {"fp32": dgfas.DGFAS_FP32, "bf16": dgfas.DGFAS_BF16, "fp64": dgfas.DGFAS_FP64}[args.precision]
    t0 = time.perf_counter()
    S, fallback = build_solver(dgfas, cfg, prec, dgfas.DGFAS_SCG, None if args.geometric else surr)
    setup_s = time.perf_counter() - t0
    S.dgfas_use_graph(True)
    tuning = [] if args.no_autotune else S.dgfas_autotune(reps=3)
    ndof = S.ndof(-1)
    b = top_rhs(S, cfg, torch, dev)
    u0 = torch.from_numpy(cfg["u0"]).to(dev)

    # ---- headline: ms per FAS V-cycle (graph replays), inputs resident in HBM
    ms, gpu_launches, clocks = time_vcycles(S, u0.clone(), b, args.steps, args.warmup, torch, dgfas,
                                            ws, dev, clocks=True)
    if ws > 1:
        ms = max_over_ranks(ms, dev)
        torch.distributed.barrier()
    value = ndof * ws / (ms * 1e-3)

    # ---- end to end through the C ABI with host buffers
    e2e_raw = e2e_record(S, torch.from_numpy(cfg["u0"]), b, torch, max(3, min(args.steps, 6)))
    e2e = {"value": ndof / e2e_raw["seconds_per_step"], "unit": UNIT,
           "h2d_bytes_per_step": e2e_raw["h2d_bytes_per_step"],
           "d2h_bytes_per_step": e2e_raw["d2h_bytes_per_step"], "overlap": e2e_raw["overlap"]}

    # ---- per-kernel timing of one SCG step on the top level and the roofline
    prof = S.dgfas_profile_scg(S.n_levels - 1, u0.clone(), b, 5)
    fp64_tf, fp32_tf = dgfas.dgfas_fma_peak()
    pk = peaks()
    m = 2
    ns = N + 2 * m
    smooth = cfg["params"]["s1"] + cfg["params"]["s2"]
    # per V-cycle on the top level: one FP64 residual (the cycle's start, the
    # two kernels of the two-pass form), the s1 + s2 SCG steps, and one more
    # smoother-precision operator (the start of post-smoothing, r - A d; the
    # residual after pre-smoothing is SCG's recursive one)
    counts = {"residual_fp64": 1, "apply_fp32": smooth + 1, "fd_tc": smooth, "combine": smooth,
              "scg_zr_dir": smooth, "scg_pq_update": smooth}
    kt = kernel_table(prof, ndof, N, ns, fp64_tf, pk["hbm"], counts)
    dom = max(kt, key=lambda k: kt[k]["count_per_vcycle"] * kt[k]["ms"])
    kd = kt[dom]
    roofline = {"bound": kd["bound"], "kernel": dom, "achieved": kd["achieved"], "peak": kd["peak"],
                "unit": kd["unit"], "frac": kd["frac"],
                "traffic": NCU_TRAFFIC.get(dom),
                "peak_source": ("measured FP64 FMA microbenchmark (dgfas_fma_peak)"
                                if kd["bound"] == "alu" else f"{pk['src']} HBM copy (MEASURED_PEAKS.json)")}

    # ---- time to 1e-10: the headline arm, then the plain FP64 GPU path
    head = "mixed_learned" if not args.geometric else "mixed_geometric"
    tts = {head: solve_record(S, u0.clone(), b, torch)}
    tts[head]["ms_per_vcycle"] = ms
    if not args.skip_fmg:
        # the same target (1e-10 of the random start's residual) from the full
        # multigrid start value (Alg. 4); the per-level right-hand sides are
        # problem set-up, outside the timing
        rr = torch.empty_like(b)
        S.dgfas_apply_op(-1, u0, b, rr)
        r_rand = S.dgfas_norm(-1, rr)
        f_lv = level_rhs(S, cfg, torch)
        uf = torch.zeros_like(u0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.dgfas_fmg(f_lv, uf)
        S.dgfas_apply_op(-1, uf, b, rr)
        r_fmg = S.dgfas_norm(-1, rr)
        info = S.dgfas_solve(uf, b, 1e-10 * r_rand / r_fmg, 40, raise_on_fail=False)
        torch.cuda.synchronize()
        tts[head + "_fmg"] = {"seconds": time.perf_counter() - t0, "cycles": info["cycles"],
                              "rel_residual": info["r_final"] / r_rand, "code": info["code"],
                              "fmg_start_rel_residual": r_fmg / r_rand}
        del f_lv, uf, rr
    S.close()
    torch.cuda.empty_cache()
    arms = []
    if not args.skip_fp64:
        arms.append(("fp64_geometric", dgfas.DGFAS_FP64, None, cfg))
    if not args.geometric and not args.skip_geometric:
        arms.append(("mixed_geometric", prec, None, cfg))
    if not args.skip_geometric:
        # the p-multigrid hierarchy 7 -> 3 -> 1 with the SCG root at p = 1
        arms.append(("mixed_learned_scg_root_p1", prec, None if args.geometric else surr,
                     wl.config(5, root="p1")))
    for name, pm, sur, cf in arms:
        S2, _ = build_solver(dgfas, cf, pm, dgfas.DGFAS_SCG, sur)
        S2.dgfas_use_graph(True)
        ms2, _, _ = time_vcycles(S2, u0.clone(), b, 3, 1, torch, dgfas)
        r = solve_record(S2, u0.clone(), b, torch)
        r["ms_per_vcycle"] = ms2
        r["dof_per_s_per_vcycle"] = ndof / (ms2 * 1e-3)
        tts[name] = r
        S2.close()
        torch.cuda.empty_cache()

    # ---- the other workloads
    others = {}
    if not args.skip_others:
        others["curvilinear16_graded_p7"] = curvilinear_records(
            dgfas, torch, dev, 3, surr,
            [("mixed_learned", prec, True), ("mixed_geometric", prec, False),
             ("fp64_geometric", dgfas.DGFAS_FP64, False)])
        others["cartesian32_p8"] = cartesian_record(dgfas, torch, dev, args)
        others["front_local_refinement_p3"] = config4_record(dgfas, torch)

    # ---- CPU baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        rate, dt, sdof = oracle_sample_rate(n_sample=8)
        cpu = {"value": rate, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS",
                                                                          host_cores())),
               "kind": "oracle",
               "sample": f"one FP64 oracle V-cycle (SCG smoother, SCG root) on the same "
                         f"workload at 8^3 elements, p = 7 ({sdof} DoF), {dt:.1f} s"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f64", 1: "f32+f64", 2: "bf16(tc)+f32+f64"}[prec], "data": "synthetic",
            "config": {"workload": "curvilinear-64^3-p7 (trilinear, +-0.15h perturbation), "
                                   "16-mode RHS, Dirichlet Poisson",
                       "elements": top["corners"].shape[0], "p": top["p"], "dof": ndof,
                       "levels": [lv["p"] for lv in levels],
                       "smoother": "SCG (Alg. 6) V(2,2), n_sc = 4, delta = 0.08",
                       "root": "p = 1 h-coarsened to 4^3 (every other vertex), exact dense root",
                       "surrogate": "geometric" if args.geometric else "learned MLP (24-64-64-6)",
                       "precision": args.precision, "graph": True,
                       "global_batch": 1, "seq_len": 0,
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "inputs larger than L2 (top vector 1.07 GB > 126 MB)"},
            "gpu_launches": gpu_launches,
            "setup": {"solver_seconds": setup_s, "surrogate_training": train_info,
                      "surrogate_fallback_elements": fallback,
                      "autotune_changed": [{k: (round(v, 4) if isinstance(v, float) else v)
                                            for k, v in t.items()} for t in tuning if t["value"] != 0]},
            "roofline": roofline,
            "kernels_top_level_scg_step": {k: {kk: (round(vv, 5) if isinstance(vv, float) else vv)
                                               for kk, vv in v.items()} for k, v in kt.items()},
            "peaks": {"fp64_tflops": fp64_tf, "fp32_tflops": fp32_tf, "hbm_gbs": pk["hbm"],
                      "hbm_source": pk["src"]},
            "time_to_1e-10": tts,
            "other_workloads": others,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "wall_s": time.perf_counter() - t_start,
        }
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()




def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dgfas", choices=["dgfas", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp64"])
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-others", action="store_true")
    ap.add_argument("--skip-geometric", action="store_true")
    ap.add_argument("--skip-fmg", action="store_true")
    ap.add_argument("--geometric", action="store_true",
                    help="headline with the geometric instead of the learned surrogate")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in launch shapes instead of the autotuner's")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
