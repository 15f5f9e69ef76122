"""Benchmark: Laplace-Beltrami solve throughput on one GB300 (or N replicas).

Workload (the default, and the one every number below refers to): the
ellipsoid with semi-axes (1, 1.5, 2), an icosahedron subdivided three times
into 1280 curved triangular patches of order 8 (45 nodes each, N = 57,600),
right-hand side f = a seeded sum of 8 Gaussian bumps exp(-|x - c_i|^2 / 0.1)
centred on surface nodes, synthetic data.

One step = one mean-zero Laplace-Beltrami solve Delta_Gamma u = f through the
A3 formulation to relative residual 1e-10: float32 far-field pair sums inside
float64 GMRES and float64 iterative refinement, near-field corrections built
once before timing (the setup time t_q is reported separately).  The metric
is far-field pair interactions evaluated per second during the solve
(Ginteractions/s, every evaluated pair counted, float32 and float64 alike),
next to the time to solve.

Timing: W untimed warm-up solves, then K solves, each bracketed by CUDA
events on the library's stream, with a 512 MB write between steps to flush
the 129 MB L2; a barrier and a device synchronise bracket the K steps, and
the maximum over ranks is reported.  Under torchrun every rank runs its own
replica of the workload on its own GPU (the solve has no exchange step).

After the timed region the same process times the plain float64 solve of
the same right-hand side (fp64_plain) and reports the refined solution's
error against a float64 solve to 1e-12 (err_vs_fp64).  cpu_baseline times
the FP64 CPU oracle on the host cores: one full A3 apply, one S apply and the
correction build of sampled rows, from which it estimates the oracle's time
to solve with and without t_q.  torus_batch records the batched form: the
18 right-hand sides of the torus (16 random f, 2 Hodge) solved in lockstep,
beside one plain float64 solve of its first right-hand side.

--impl reference times the FP64 CPU oracle (the tests' reference
implementation) on the host cores instead, one full A3 apply per step.
--gpus N outside torchrun starts N replicas under torch.distributed.run.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Layer-potential apply Ginteractions/s; time-to-solve at 1e-10 rel. residual"
UNIT = "Ginteractions/s"
WORKLOAD = ("ellipsoid (1,1.5,2), {P} order-8 patches (N={N:,}), f = 8 Gaussian bumps; "
            "A3 solve to 1e-10 rel. residual")
WORKLOAD_TORUS = ("torus R=2 r=0.75, {P} order-6 patches (N={N:,}), batch of 18 RHS: 16 random Legendre f "
                  "+ the 2 Hodge RHS div F, -div(n x F); A3 lockstep solve to 1e-10 rel. residual")

# far-field flops per evaluated pair, counting an FMA as two (kernel source in
# paper_2111_10743_gb300/csrc/far.cu): d (3), r^2 (5), then per kind
FLOPS_PER_PAIR = {"k1": 20, "kall": 45, "k2": 43, "k4": 21}
# batched kernels (csrc/far_batch.cu): flops per pair shared by the densities
# of a pass, and flops per pair and density
FLOPS_BATCH = {"k1": (10, 9), "k2": (35, 8)}
# double-float kernels (csrc/far_df.cu): float32 operations per pair, FMA = 2
# (TwoSum 6, FastTwoSum 3, pair add 8, pair product 7, square 6, rsqrt with
# Newton step 17, accumulate 8; d renormalised, 15)
DF_FLOPS_PER_PAIR = {"k1": 146, "kall": 329, "k2": 335, "k4": 159}
# symmetric kernels (A3 passes; far.cu k_far32_sym, far_df.cu k_far_df_sym):
# flops of one unordered pair, both directions, halved to a per-ordered-pair
# figure: float32 K1 28 / 2, K2 56 / 2; double-float K1 213 / 2, K2 396 / 2
SYM_FLOPS_PER_PAIR = {"k1": 14.0, "k2": 28.0}
DF_SYM_FLOPS_PER_PAIR = {"k1": 106.5, "k2": 198.0}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def worst_over_ranks(values, device="cpu"):
    """Elementwise maximum of per-rank timings over all ranks (every replica
    times its own solves; the slowest one sets the whole job's time)."""
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        # nvidia-smi's start-up (NVML initialisation) must not overlap the
        # timed region: wait for its first sample line (at most 5 s)
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < 5.0:
            if self.proc.poll() is not None or os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "power_w_max": max(power),
                "samples": len(sm), "reasons": sorted(reasons)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


def source_digest(name: str) -> str:
    """First 16 hex digits of the SHA-256 of a CUDA source file of the library."""
    src = os.path.join(ROOT, "paper_2111_10743_gb300", "csrc", name)
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def _traffic(kernel: str, n_nodes: int):
    """DRAM bytes per launch of `kernel` from profiles/traffic.json (an ncu
    capture of dram__bytes_read.sum + dram__bytes_write.sum), or None when the
    kernel's source has changed since.  The capture is on a smaller surface;
    the sources and targets stay in L2, so DRAM traffic grows with the node
    count N, not with the N^2 pairs, and is scaled by N."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        ent = json.load(open(path)).get(kernel)
    except (OSError, ValueError):
        return None
    if not ent or not ent.get("source") or ent.get("source_sha256") != source_digest(ent["source"]):
        return None
    return int(ent["dram_bytes_per_launch"] * n_nodes / ent["captured_n"])


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    g.build()
    import paper_2111_10743_gb300 as lb
    from workloads.configs import config

    if args.case == "small":   # same code path on 320 patches (N = 14,400), for profiler captures
        from workloads.configs import ellipsoid_gauss
        w = ellipsoid_gauss(2, 8, 1002)
    elif args.case == "torus_batch":
        w = config(3)
    elif args.case == "torus_small":   # the batch on a 16 x 16 torus (N = 14,336), for profiler captures
        from workloads.configs import torus_batch
        w = torus_batch(16, 16, 6, 16, 1003)
    else:
        w = config(2)
    s = w.surface
    prec = {"fp32_refined": lb.LB_FP32_REFINED, "fp64": lb.LB_FP64, "fp32": lb.LB_FP32}[args.precision]
    params = lb.default_params(eps_quad=1e-12, tol=1e-10, precision=prec, formulation=lb.LB_A3)
    stream = torch.cuda.current_stream()
    ctx = lb.Context(local, params, stream=stream)
    ctx.upload_surface(s)
    torch.cuda.synchronize()
    t0 = time.time()
    ctx.build_corrections()
    torch.cuda.synchronize()
    t_q = time.time() - t0
    fb = w.f
    if args.case in ("torus_batch", "torus_small"):   # right-hand sides of the two Hodge potentials (Section 5)
        n, _, _ = ctx.get_geometry()
        F = w.extra["F"]
        fb = np.concatenate([w.f, ctx.surface_div(F[None]), -ctx.surface_div(np.cross(n, F)[None])])
    f = torch.tensor(fb, device="cuda")
    u = torch.empty_like(f)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        _, info = ctx.solve_lb(f, out=u)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    pairs = 0
    infos = []
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ctx.set_profiling(True)
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            _, info = ctx.solve_lb(f, out=u)
            ev[k][1].record(stream)
            pairs += info["pairs"]
            infos.append(info)
        torch.cuda.synchronize()
        prof = ctx.get_profile()
        ctx.set_profiling(False)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    clocks = clk.summary()

    # end to end through the C ABI with pinned host buffers: copies inside
    fh = torch.tensor(fb).pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    ctx.solve_lb(fh, out=uh)   # untimed: first use of the host-staging buffers
    e2e_ms = []
    for k in range(max(1, min(args.steps, args.e2e_steps))):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info_e = ctx.solve_lb(fh, out=uh)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_pairs = info_e["pairs"]

    # the plain float64 form of the same solve on the same GPU, after the
    # timed region: its time, and the refined solution's error against a
    # float64 solve to 1e-12
    fp64_plain = None
    if args.precision == "fp32_refined" and not args.case.startswith("torus") and not args.no_fp64:
        u_ref = u.detach().clone()
        p64 = lb.default_params(eps_quad=1e-12, tol=1e-10, precision=lb.LB_FP64, formulation=lb.LB_A3)
        ctx.set_params(p64)
        u64 = torch.empty_like(f)
        ctx.solve_lb(f, out=u64)                      # warm-up (float64 kernels, workspaces)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        e0.record(stream)
        _, i64 = ctx.solve_lb(f, out=u64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        p64.tol = 1e-12
        ctx.set_params(p64)
        uex = torch.empty_like(f)
        _, iex = ctx.solve_lb(f, out=uex)
        torch.cuda.synchronize()
        ctx.set_params(params)
        nrm = float(torch.linalg.vector_norm(uex))
        fp64_plain = {
            "ms_per_step": round(ms64, 2), "iterations": i64["iterations"],
            "rel_residual": i64["rel_residual"], "tol": 1e-10,
            "value": round(i64["pairs"] / (ms64 * 1e-3) / 1e9, 3), "unit": UNIT,
            "err_vs_fp64_tol1e-12": {
                "refined_rel_l2": float(torch.linalg.vector_norm(u_ref - uex)) / nrm,
                "refined_max_rel": float((u_ref - uex).abs().max() / uex.abs().max()),
                "fp64_tol1e-10_rel_l2": float(torch.linalg.vector_norm(u64 - uex)) / nrm,
                "reference_iterations": iex["iterations"], "reference_rel_residual": iex["rel_residual"]},
        }

    # worst rank
    ms_max, e2e_max = worst_over_ranks([ms, sum(e2e_ms) / len(e2e_ms)], device="cuda")
    if rank != 0:
        return
    ms_step = ms_max / args.steps
    value = pairs * ws / (ms_max * 1e-3) / 1e9
    e2e_value = e2e_pairs * ws / (e2e_max * 1e-3) / 1e9

    # dominant far kernel: its flops per launch over its mean event-timed duration
    peaks = _peaks()
    sm_count = ctx.info()["sm_count"]
    clk_mhz = clocks.get("sm_mhz") or (peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 1440.0)
    cats = {k: v for k, v in prof.items() if isinstance(v, dict) and k.startswith("far")}
    tuning = ctx.get_tuning()
    dom = max(cats, key=lambda k: cats[k]["ms"]) if cats else None
    roofline = None
    nrhs = fb.shape[0]
    if dom:
        kind = dom.split("_")[1]
        per_launch_ms = cats[dom]["ms"] / cats[dom]["calls"]
        fp32_peak = sm_count * 128 * 2 * clk_mhz * 1e6 / 1e12
        fp32_note = "fp32 CUDA-core FMA peak: SMs x 128 lanes x 2 flops x median SM clock sampled under load"
        if dom.startswith("far32") and nrhs >= 2:
            # lockstep solves: chunks of 8 densities (fewer in the last chunk)
            per_launch_dens = cats[dom]["pairs"] / (s.N * s.N) / cats[dom]["calls"]
            sh, pd = FLOPS_BATCH[kind]
            flops = s.N * s.N * (sh + pd * per_launch_dens)
            peak, note, kname = fp32_peak, fp32_note, f"k_farb32<{dom}>"
        elif dom.startswith("far32"):
            sym = (tuning.get(f"far32_single_{kind}") or "").startswith("symmetric")
            flops = s.N * s.N * (SYM_FLOPS_PER_PAIR[kind] if sym else FLOPS_PER_PAIR[kind])
            peak, note = fp32_peak, fp32_note
            kname = f"k_far32_sym<{dom}>" if sym else f"k_far<{dom}>"
        elif dom.startswith("fardf"):
            sym = kind in DF_SYM_FLOPS_PER_PAIR
            flops = s.N * s.N * (DF_SYM_FLOPS_PER_PAIR[kind] if sym else DF_FLOPS_PER_PAIR[kind])
            peak, note = fp32_peak, fp32_note + " (double-float arithmetic in float32 operations)"
            kname = f"k_far_df_sym<{dom}>" if sym else f"k_far_df<{dom}>"
        else:
            flops = s.N * s.N * FLOPS_PER_PAIR[kind]
            peak = 1.25 * clk_mhz / 2070.0
            note = "fp64 nominal 1.25 TFLOP/s scaled by median SM clock / 2070 MHz"
            kname = f"k_far<{dom}>"
        achieved = flops / (per_launch_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": kname, "achieved": round(achieved, 3),
                    "peak": round(peak, 3), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                    "traffic": _traffic(kname, s.N), "peak_source": note,
                    "launch_ms": round(per_launch_ms, 4), "share_of_step": round(cats[dom]["ms"] / ms, 4)}
    kernels = {k: {"ms_per_step": round(v["ms"] / args.steps, 3), "calls_per_step": v["calls"] / args.steps,
                   **({"gpairs_per_step": round(v["pairs"] / args.steps / 1e9, 3)} if v.get("pairs") else {})}
               for k, v in prof.items() if isinstance(v, dict)}
    last = infos[-1]
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32_refined": "f32 + double-float pairs, f64 solve", "fp64": "f64",
                  "fp32": "f32 pairs, f64 solve"}[args.precision],
        "data": "synthetic", "time_to_solve_ms": round(ms_step, 3), "t_q_s": round(t_q, 2),
        "config": {"workload": (WORKLOAD_TORUS if args.case.startswith("torus") else WORKLOAD).format(
                       P=s.npatch, N=s.N), "N": s.N,
                   "patches": s.npatch, "order": s.order, "nrhs": int(nrhs),
                   "formulation": "A3", "precision": args.precision, "tol": 1e-10, "eps_quad": 1e-12,
                   "near_factor": 2.0, "l2": "512 MB write between timed steps",
                   "parallelism": f"replicas x{ws}"},
        "solve": {"iterations": last["iterations"], "refinements": last["refinements"],
                  "applies_fp32": last["applies_fp32"], "applies_fp64": last["applies_fp64"],
                  "rel_residual": last["rel_residual"], "pairs_per_step": last["pairs"]},
        "kernels": kernels,
        "roofline": roofline,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "ms_per_step": round(e2e_max, 3),
                "ms_each": [round(x, 3) for x in e2e_ms],
                "h2d_bytes_per_step": int(fh.numel() * 8), "d2h_bytes_per_step": int(uh.numel() * 8)},
        "gpu_launches": int(prof["launches"]),
        **({"fp64_plain": {**fp64_plain, "speedup_of_refined": round(fp64_plain["ms_per_step"] / ms_step, 2)},
            "err_vs_fp64": fp64_plain["err_vs_fp64_tol1e-12"]["refined_rel_l2"]} if fp64_plain else {}),
        "autotune": {k: v for k, v in ctx.get_tuning().items() if v},
        "clocks": clocks,
    }
    if ws == 1 and args.case == "full" and not args.no_batch:
        ctx.close()
        out["torus_batch"] = torus_batch_record(lb, torch, local, stream, flush)
    if ws == 1 and not args.no_cpu_baseline and not args.case.startswith("torus"):
        iters64 = fp64_plain["iterations"] if fp64_plain else None
        out["cpu_baseline"] = cpu_baseline(iters64)
    print(json.dumps(out))


def run_genus5(args):
    """Configuration 5 with direct far-field sums: the genus-5 surface (five
    blended tori, 36,272 order-6 patches, N = 1,015,616).  Corrections built
    on the GPU; the harmonic fields of six seeded tangential F (12 Hodge
    right-hand sides, the five of the configuration and one more so that the
    rank gap after 2g = 10 can show) and four of its random f, solved in
    lockstep with float32 pairs refined to 1e-9; the harmonic space's rank;
    far sums against the FP64 oracle on 2,048 sampled targets.  The octree FMM
    that the paper uses at this size is not built: every pass is a direct sum
    over N^2 pairs, and the timings say what that costs."""
    import torch
    _, _, local = _dist()
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    g.build()
    import paper_2111_10743_gb300 as lb
    from oracle import farsum
    from oracle.geometry import build_geometry, near_lists
    from workloads import rhs as R
    from workloads.configs import _centred, _tangential, config
    t0 = time.time()
    w = config(5)
    s = w.surface
    Xc, L = _centred(s)
    F = np.concatenate([w.extra["F"],
                        _tangential(s, R.legendre_field(Xc, np.random.default_rng(1105), 4, L, ncomp=3))[None]])
    t_mesh = time.time() - t0
    stream = torch.cuda.current_stream()
    params = lb.default_params(eps_quad=1e-12, tol=w.tol, precision=lb.LB_FP32_REFINED, formulation=lb.LB_A3)
    ctx = lb.Context(local, params, stream=stream)
    ctx.upload_surface(s)
    torch.cuda.synchronize()
    t0 = time.time()
    ctx.build_corrections()
    torch.cuda.synchronize()
    t_q = time.time() - t0
    Fd = torch.tensor(F, device="cuda")
    H = torch.empty((2 * F.shape[0],) + F.shape[1:], dtype=torch.float64, device="cuda")
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    _, info_h = ctx.harmonic_fields(Fd, out=H)
    e[1].record(stream)
    f = torch.tensor(w.f[:4], device="cuda")
    u = torch.empty_like(f)
    e[2].record(stream)
    _, info_f = ctx.solve_lb(f, out=u)
    e[3].record(stream)
    torch.cuda.synchronize()
    ms_h, ms_f = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
    n, wq, _ = ctx.get_geometry()
    Hh = H.cpu().numpy()
    M = (Hh * np.sqrt(wq)[None, :, None]).reshape(Hh.shape[0], -1)
    sv = np.sqrt(np.maximum(np.linalg.eigvalsh(M @ M.T)[::-1], 0.0))
    div = ctx.surface_div(Hh)
    divrel = max(float(np.sqrt(np.sum(wq * div[k] ** 2) / np.sum(wq * np.sum(Hh[k] ** 2, 1))))
                 for k in range(Hh.shape[0]))
    # far sums against the oracle on sampled targets (its own geometry and near lists)
    geo = build_geometry(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv)
    rng = np.random.default_rng(7)
    targets = np.sort(rng.choice(s.N, 2048, replace=False)).astype(np.int64)
    ptr, pl = near_lists_sampled(geo, targets, 2.0)
    sig = rng.standard_normal(s.N)
    ref = farsum.far_sums(geo, ptr, pl, sig, targets)[0]
    errs = {}
    for name, prec in (("fp32", lb.LB_FP32), ("df64", lb.LB_DF64)):
        got = ctx.far_sums(sig[None], precision=prec)[0][:, targets]
        errs[name] = max(float(np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max()) for k in range(4))
    pairs = info_h["pairs"] + info_f["pairs"]
    ctx.close()
    print(json.dumps({
        "metric": METRIC, "value": round(pairs / ((ms_h + ms_f) * 1e-3) / 1e9, 3), "unit": UNIT,
        "case": "genus5", "data": "synthetic", "dtype": "f32 + double-float pairs, f64 solve",
        "config": {"workload": f"genus-5 surface (5 blended tori), {s.npatch} order-6 patches (N={s.N:,}); "
                               f"12 Hodge RHS (6 tangential F) + 4 Legendre f; A3 lockstep solves to 1e-9",
                   "N": s.N, "patches": s.npatch, "order": s.order, "far_field": "direct sums (no FMM)"},
        "mesh_s": round(t_mesh, 1), "t_q_s": round(t_q, 1),
        "hodge": {"nrhs": 2 * F.shape[0], "ms": round(ms_h, 1), "iterations": info_h["iterations"],
                  "refinements": info_h["refinements"], "rel_residual": info_h["rel_residual"],
                  "converged": info_h["converged"]},
        "random_f": {"nrhs": 4, "ms": round(ms_f, 1), "iterations": info_f["iterations"],
                     "refinements": info_f["refinements"], "rel_residual": info_f["rel_residual"],
                     "converged": info_f["converged"]},
        "harmonic_space": {"fields": int(Hh.shape[0]), "sv_rel": [float(x / sv[0]) for x in sv],
                           "rank_2g": int(np.sum(sv > 1e-3 * sv[0])), "max_rel_div": divrel},
        "oracle_sampled_far_sums": {"targets": 2048, "max_rel_err": errs},
        "pairs": int(pairs),
    }))


def near_lists_sampled(geo, targets, eta):
    """Near lists by the oracle's rule for the sampled targets only, as a CSR
    over all N rows (rows outside the sample are empty)."""
    N = geo.N
    counts = np.zeros(N, dtype=np.int64)
    rows = []
    for i in targets:
        d = np.linalg.norm(geo.centroid - geo.X[i][None, :], axis=1)
        r = np.nonzero(d < eta * geo.radius)[0].astype(np.int32)
        rows.append(r)
        counts[i] = len(r)
    ptr = np.zeros(N + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(counts)
    return ptr, (np.concatenate(rows) if rows else np.zeros(0, dtype=np.int32))


def torus_batch_record(lb, torch, device, stream, flush, steps=3, warmup=3):
    """The batched form on the torus R = 2, r = 0.75 (2,048 order-6 patches,
    N = 57,344): 16 random Legendre f and the two Hodge right-hand sides
    solved together in lockstep (A3, fp32_refined, tol 1e-10), timed like the
    main line; beside it one plain float64 solve of its first right-hand side
    (the float64 form solves right-hand sides one at a time, so 18 of them
    cost 18 such solves) and that solution's error against the batch's."""
    from workloads.configs import config
    w = config(3)
    s = w.surface
    params = lb.default_params(eps_quad=1e-12, tol=1e-10, precision=lb.LB_FP32_REFINED, formulation=lb.LB_A3)
    ctx = lb.Context(device, params, stream=stream)
    ctx.upload_surface(s)
    torch.cuda.synchronize()
    t0 = time.time()
    ctx.build_corrections()
    torch.cuda.synchronize()
    t_q = time.time() - t0
    n, _, _ = ctx.get_geometry()
    F = w.extra["F"]
    fb = np.concatenate([w.f, ctx.surface_div(F[None]), -ctx.surface_div(np.cross(n, F)[None])])
    f = torch.tensor(fb, device="cuda")
    u = torch.empty_like(f)
    for _ in range(warmup):
        ctx.solve_lb(f, out=u)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    pairs = 0
    torch.cuda.synchronize()
    ctx.set_profiling(True)
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        _, info = ctx.solve_lb(f, out=u)
        ev[k][1].record(stream)
        pairs += info["pairs"]
    torch.cuda.synchronize()
    prof = ctx.get_profile()
    ctx.set_profiling(False)
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    cats = {k: v for k, v in prof.items() if isinstance(v, dict) and k.startswith("far")}
    tuning = ctx.get_tuning()
    dom = max(cats, key=lambda k: cats[k]["ms"])
    # one plain float64 solve of the first right-hand side, timed
    ctx.set_params(lb.default_params(eps_quad=1e-12, tol=1e-10, precision=lb.LB_FP64, formulation=lb.LB_A3))
    u64 = torch.empty_like(f[:1])
    ctx.solve_lb(f[:1], out=u64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, i64 = ctx.solve_lb(f[:1], out=u64)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    err = float(torch.linalg.vector_norm(u[:1] - u64) / torch.linalg.vector_norm(u64))
    ctx.close()
    return {
        "workload": WORKLOAD_TORUS.format(P=s.npatch, N=s.N), "nrhs": int(fb.shape[0]), "steps": steps,
        "ms_per_step": round(ms, 2), "value": round(pairs / steps / (ms * 1e-3) / 1e9, 3), "unit": UNIT,
        "t_q_s": round(t_q, 2), "iterations": info["iterations"], "refinements": info["refinements"],
        "rel_residual": info["rel_residual"], "graph_iterations": info["graph_iterations"],
        "dominant_kernel": {"name": dom, "ms_per_step": round(cats[dom]["ms"] / steps, 3),
                            "calls_per_step": cats[dom]["calls"] / steps},
        "fp64_plain_one_rhs_ms": round(ms64, 2), "fp64_plain_iterations": i64["iterations"],
        "fp64_plain_all_rhs_est_ms": round(ms64 * fb.shape[0], 1),
        "speedup_of_batch_est": round(ms64 * fb.shape[0] / ms, 2),
        "err_vs_fp64_first_rhs": err,
    }


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_setup():
    """The oracle's geometry and near lists of the benchmark surface, and a
    Discretisation whose correction blocks have the oracle's CSR structure and
    seeded values: the timed arithmetic (every far pair, every correction
    entry) is the oracle's own, and its cost does not depend on the values."""
    from oracle.geometry import build_geometry
    from oracle.layers import Discretisation
    from workloads.configs import config
    w = config(2)
    s = w.surface
    geo = build_geometry(s.order, s.uv, s.wref, s.X, s.Xu, s.Xv)
    # near lists by the oracle's rule, vectorised over targets in chunks
    N = geo.N
    rows = []
    for a in range(0, N, 4096):
        d = np.linalg.norm(geo.X[a:a + 4096, None, :] - geo.centroid[None, :, :], axis=2)
        rows += [np.nonzero(r < 2.0 * geo.radius)[0].astype(np.int32) for r in d]
    ptr = np.zeros(N + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([len(r) for r in rows])
    pl = np.concatenate(rows)
    vals = np.random.default_rng(8).standard_normal((len(pl), 4, geo.np_)) * 1e-3
    disc = Discretisation(geo, ptr, pl, vals, 2.0, 1e-12)
    return w, disc


def _oracle_apply(disc, seed):
    """One A3 apply by the oracle (far sums of 1 + 2 densities over all
    targets, correction sums, assembly); returns (seconds, far pairs)."""
    tau = np.random.default_rng(seed).standard_normal(disc.geo.N)
    t0 = time.perf_counter()
    disc.apply_A3(tau)
    return time.perf_counter() - t0, 3 * disc.geo.N * disc.geo.N


def _oracle_tq_sample(disc, nrows: int):
    """Oracle correction build for nrows sampled rows, all host cores;
    returns (seconds, blocks built)."""
    from oracle.quadrature import build_corrections
    g = disc.geo
    rows = np.random.default_rng(9).choice(g.N, nrows, replace=False)
    t0 = time.perf_counter()
    build_corrections(g, disc.near_ptr, disc.near_patch, eps_q=1e-12, rows=rows, workers=os.cpu_count() or 1)
    dt = time.perf_counter() - t0
    nblk = int(np.isin(np.repeat(np.arange(g.N), np.diff(disc.near_ptr)), rows).sum())
    return dt, nblk


def cpu_baseline(iters_fp64, tq_rows: int = 32):
    """The FP64 oracle on all host cores: one full A3 apply (the far sums in
    C/OpenMP, the correction sums in C/OpenMP, the assembly in numpy), one
    S apply, and the correction build of sampled rows.  Time to solve is
    estimated as k applies + 2 S applies (u = S[S[sigma]]), k the iteration
    count of the float64 GPU solve of the same system (the same operator and
    GMRES); t_q is the sampled rows' time scaled to every block."""
    w, disc = _oracle_setup()
    g = disc.geo
    t_apply, pairs = _oracle_apply(disc, 1)
    sig = np.random.default_rng(2).standard_normal(g.N)
    t0 = time.perf_counter()
    disc.S(sig)
    t_s = time.perf_counter() - t0
    t_smp, nblk = _oracle_tq_sample(disc, tq_rows)
    t_q = t_smp * len(disc.near_patch) / max(nblk, 1)
    k = iters_fp64
    out = {"value": round(pairs / t_apply / 1e9, 4), "unit": UNIT, "cores": os.cpu_count(),
           "cpu_model": cpu_model(), "kind": "oracle",
           "sample": (f"one full A3 apply (N = {g.N:,}: far sums of 1 + 2 densities, correction sums, assembly), "
                      f"one S apply, and the correction build of {tq_rows} sampled rows ({nblk} blocks) "
                      f"scaled to all {len(disc.near_patch):,} blocks; FP64 C/OpenMP + numpy oracle"),
           "apply_ms": round(t_apply * 1e3, 1), "s_apply_ms": round(t_s * 1e3, 1),
           "t_q_s": round(t_q, 1), "t_q_sample_s": round(t_smp, 2)}
    if k:
        ts = k * t_apply + 2 * t_s
        out["time_to_solve_ms"] = round(ts * 1e3, 1)
        out["time_to_solve_with_t_q_s"] = round(ts + t_q, 1)
        out["time_to_solve_basis"] = f"{k} applies (the float64 GPU solve's iterations) + 2 S applies"
    return out


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    w, disc = _oracle_setup()
    g = disc.geo
    for k in range(args.warmup):   # warm-up: the far sums of 64 targets
        from oracle import farsum
        farsum.far_sums(g, disc.near_ptr, disc.near_patch, np.ones(g.N), np.arange(64))
    tot, inter = 0.0, 0
    for k in range(args.steps):
        dt, n = _oracle_apply(disc, 100 + k)
        tot += dt
        inter += n
    value = inter / tot / 1e9
    cores = os.cpu_count()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot / args.steps * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD.format(P=g.npatch, N=g.N), "N": g.N,
                   "step": "one full A3 apply by the FP64 oracle (the unit each GMRES iteration repeats)"},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "cpu_model": cpu_model(),
                         "kind": "oracle",
                         "sample": f"{args.steps} full A3 applies (far sums of 1 + 2 densities over all "
                                   f"{g.N:,} targets, correction sums, assembly), FP64 C/OpenMP + numpy"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32_refined", choices=["fp32_refined", "fp64", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain float64 solve after the timed region")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched torus record of the default line")
    ap.add_argument("--case", default="full", choices=["full", "small", "torus_batch", "torus_small", "genus5"],
                    help="full: the benchmark surface; small: 320 patches of the same kind (profiling); "
                         "torus_batch: the torus with 18 right-hand sides solved in lockstep; "
                         "torus_small: the same batch on a 16 x 16 torus (profiling); genus5: configuration 5 "
                         "(N = 1,015,616) with direct far sums, one run")
    ap.add_argument("--e2e-steps", type=int, default=3)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: start the replicas under torch.distributed.run
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr", "127.0.0.1", "--master-port", str(29500 + os.getpid() % 1000),
               os.path.abspath(__file__), *sys.argv[1:]]
        sys.exit(subprocess.call(cmd))
    if ws != args.gpus:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE {ws}; timing {ws} replica(s)", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.case == "genus5":
        run_genus5(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
