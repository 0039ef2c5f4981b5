#!/usr/bin/env python
"""Throughput of the periodic FMM evaluation of u and the stretching term.

Workload (one "step" = the whole hot path once): 256^3 = 16,777,216 vortex particles on the
cell-centre lattice of [0, 2 pi)^3, seeded random-phase solenoidal field with
E(k) ~ k^4 exp(-2 k^2/k0^2), k0 = 4, unit energy, alpha = omega h^3, sigma = h; FMM order
p = 10, 27^3 periodic images (3 super-levels of the image lattice, S = 2).  A step is
vfmm_build_tree (wrap, Morton-free leaf keys, counting sort) + vfmm_eval_velocity_stretching
(P2M, M2M, FP64 root and lattice operator, M2L, L2L, L2P, P2P + un-permute).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead.
Multi-GPU (torchrun): every rank evaluates its own independent field (seed 1 + rank):
replicas, weak scaling, no data-path collective.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/s for u+stretching at 256³ (p=10), rel-L2 err vs FP64 direct sum"
PAPER_PARTICLES_PER_S = 0.84e6   # 256^3 / 20 s per step at p=10 on one C2070 (paper, Section 4.1)
FLOPS_PER_PAIR = 61              # FP32 operations of one smoothed P2P pair (FMA = 2), + 3 MUFU
FLOPS_PER_PAIR_SINGULAR = 42     # a pair of leaves >= 6.5 sigma apart (singular kernel), + 1 MUFU
ALGO_FLOPS_PER_PAIR = 70         # algorithmic work of one pair of Eqs. (biotsavart)+(stretching) with the
                                 # smoothed kernel: difference, r^2, K, F, two cross products, the
                                 # projection gamma_i . r and six accumulations (FMA = 2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="vfmm", choices=["vfmm", "reference"])
    ap.add_argument("--n", type=int, default=256, help="particles per side")
    ap.add_argument("--p", type=int, default=10)
    ap.add_argument("--k0", type=int, default=4)
    ap.add_argument("--m2l", default="bf16x3", choices=["fp32", "tf32x3", "bf16x3"])
    ap.add_argument("--periodic-levels", type=int, default=2)
    ap.add_argument("--depth", type=int, default=0, help="tree depth (0 = from the mean leaf occupancy)")
    ap.add_argument("--rho-cut", type=float, default=5.0,
                    help="pairs closer than rho_cut sigma take the smoothed kernel, farther ones the singular")
    ap.add_argument("--check", type=int, default=16, help="sampled targets for the oracle error (0 = off)")
    ap.add_argument("--cpu-targets", type=int, default=0, help="oracle targets for cpu_baseline (0 = one per host core)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--concurrent-far", type=int, default=-1,
                    help="1: far field on a side stream beside the P2P; 0: every phase in line; -1: library default")
    ap.add_argument("--peaks", type=int, default=1, help="measure the FP32/MUFU/FP64/TF32/BF16 peaks (probe kernels)")
    ap.add_argument("--workload", default="eval", choices=["eval", "timestep"],
                    help="eval: u + S per step (the metric); timestep: ten Heun steps + one reinitialisation")
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def combine_ranks(ms, particles, steps, device=None):
    """Max-over-ranks time (ms) and whole-job particles/s.

    Replicas: every rank evaluates its own field of ``particles`` particles, so the job
    processes world_size * particles * steps particles in the slowest rank's time."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, ws * particles * steps / (ms_max / 1e3)


def p2p_work(x, L, depth, R, sigma, Rc=0, rho_cut=6.0, half_cull=True):
    """Pairs the P2P visits, split as the kernel splits them: by the gap d between the target
    leaf's box and each source octant's box.  In the R near rings d < 6.5 sigma -> smoothed
    kernel (61 flops), d >= 6.5 sigma -> singular kernel (42 flops); in the rings R+1..Rc
    (Gaussian-tail correction of the far field) d < rho_cut sigma -> smoothed minus singular
    (61 flops), farther octants are skipped.  With half_cull the correction rings use the box
    of each half of a warp's targets (ranks 0-31 and 32-63 of each 64-target chunk of a leaf
    sorted by (octant, index)) instead of the leaf's box.  Returns (pairs, flops)."""
    import itertools
    import numpy as np
    ns = 1 << depth
    xf = np.mod(x, L).astype(np.float32).astype(np.float64)
    c = np.clip((xf / L * ns).astype(np.int64), 0, ns - 1)
    o = np.clip((xf / L * 2 * ns).astype(np.int64) - 2 * c, 0, 1)
    key = (c[:, 0] * ns + c[:, 1]) * ns + c[:, 2]
    okey = key * 8 + (o[:, 0] * 4 + o[:, 1] * 2 + o[:, 2])
    nleaf = ns ** 3

    def boxes(k, nk):
        cnt = np.bincount(k, minlength=nk).astype(np.float64)
        lo = np.full((nk, 3), 3e38)
        hi = np.full((nk, 3), -3e38)
        order = np.argsort(k, kind="stable")
        xs = xf[order]
        ne = cnt > 0
        starts = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.int64)[ne]
        lo[ne] = np.minimum.reduceat(xs, starts, axis=0)
        hi[ne] = np.maximum.reduceat(xs, starts, axis=0)
        return cnt, lo, hi

    cnt, lo, hi = boxes(key, nleaf)
    ocnt, olo, ohi = boxes(okey, 8 * nleaf)
    if half_cull:
        # rank of each particle in its leaf in the kernel's order (octant, caller index)
        order = np.lexsort((np.arange(len(key)), okey))
        first = np.searchsorted(key[order], key[order], side="left")
        rank = np.empty(len(key), np.int64)
        rank[order] = np.arange(len(key)) - first
        grp = (rank // 64) * 2 + (rank % 64) // 32
        G = int(grp.max()) + 1
        hcnt, hlo, hhi = boxes(key * G + grp, G * nleaf)
        hcnt = hcnt.reshape(ns, ns, ns, G)
        hlo = hlo.reshape(ns, ns, ns, G, 3)
        hhi = hhi.reshape(ns, ns, ns, G, 3)
    cnt = cnt.reshape(ns, ns, ns)
    lo = lo.reshape(ns, ns, ns, 3)
    hi = hi.reshape(ns, ns, ns, 3)
    ocnt = ocnt.reshape(ns, ns, ns, 8)
    olo = olo.reshape(ns, ns, ns, 8, 3)
    ohi = ohi.reshape(ns, ns, ns, 8, 3)
    g = np.arange(ns)
    C = np.meshgrid(g, g, g, indexing="ij")
    d2_sing = np.float32(42.25 * sigma * sigma)
    d2_cut = np.float32(rho_cut * rho_cut * sigma * sigma)
    p_s, p_g = 0.0, 0.0
    for t in itertools.product(range(-max(R, Rc), max(R, Rc) + 1), repeat=3):
        corr = max(abs(v) for v in t) > R
        nb = [C[d] + t[d] for d in range(3)]
        sh = [np.floor_divide(nb[d], ns) * L for d in range(3)]
        ix = [np.mod(nb[d], ns) for d in range(3)]
        cn = ocnt[ix[0], ix[1], ix[2]]                      # (ns,ns,ns,8)
        d2 = np.zeros_like(cn)
        for d in range(3):
            slo = olo[ix[0], ix[1], ix[2], :, d] + sh[d][..., None]
            shi = ohi[ix[0], ix[1], ix[2], :, d] + sh[d][..., None]
            gap = np.maximum(0.0, np.maximum(slo - hi[..., d][..., None], lo[..., d][..., None] - shi))
            d2 += gap * gap
        pairs = cnt[..., None] * cn
        if corr and half_cull:
            for gi in range(G):
                dh = np.zeros_like(cn)
                for d in range(3):
                    slo = olo[ix[0], ix[1], ix[2], :, d] + sh[d][..., None]
                    shi = ohi[ix[0], ix[1], ix[2], :, d] + sh[d][..., None]
                    gap = np.maximum(0.0, np.maximum(slo - hhi[..., gi, d][..., None], hlo[..., gi, d][..., None] - shi))
                    dh += gap * gap
                hp = hcnt[..., gi][..., None] * cn
                p_s += float(hp[dh < d2_cut].sum())
            continue
        if corr:
            p_s += float(pairs[d2 < d2_cut].sum())
            continue
        sing = d2 >= d2_sing
        p_g += float(pairs[sing].sum())
        p_s += float(pairs[~sing].sum())
    return p_s + p_g, FLOPS_PER_PAIR * p_s + FLOPS_PER_PAIR_SINGULAR * p_g


PROBE_REPS = {"fp32_ffma": 40000, "mufu_ex2": 5000, "mufu_rsqrt": 5000, "fp64_dfma": 600,
              "tf32_tcgen05": 400000, "bf16_tcgen05": 400000}


def measure_peaks(dev, stream, repeats=3):
    """Peak rates of the units the path uses, from the library's probe kernels (one launch each,
    CUDA events on the launching stream, best of ``repeats`` after one warm-up), with the SM
    clock sampled while they run.  Units: TFLOP/s (FMA and MMA: 2 flops each), Gop/s (MUFU)."""
    import torch
    from paper_1110_2921_gb300 import _native as nv
    kinds = {"fp32_ffma": nv.VFMM_PROBE_FFMA, "mufu_ex2": nv.VFMM_PROBE_EX2, "mufu_rsqrt": nv.VFMM_PROBE_RSQRT,
             "fp64_dfma": nv.VFMM_PROBE_DFMA, "tf32_tcgen05": nv.VFMM_PROBE_MMA_TF32,
             "bf16_tcgen05": nv.VFMM_PROBE_MMA_BF16}
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    sp = stream.cuda_stream
    clocks = ClockSampler(dev.index)
    out = {}
    for name, kind in kinds.items():
        reps = PROBE_REPS[name]
        nv.vfmm_probe_peak(kind, reps // 10, sp, err.data_ptr())
        best = None
        for _ in range(repeats):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ops = nv.vfmm_probe_peak(kind, reps, sp, err.data_ptr())
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        scale = 1e9 if name.startswith("mufu") else 1e12
        out[name] = ops / (best / 1e3) / scale
        out[name + "_ms"] = best
    clk = clocks.stop()
    if int(err.item()) != 0:
        raise RuntimeError("a tcgen05 probe reported a wait timeout")
    out["units"] = "TFLOP/s (fp32, fp64, tf32, bf16), Gop/s (mufu)"
    out["how"] = ("probe kernels of libvfmm (vfmm_probe_peak), one launch each timed with CUDA events, best of %d"
                  % repeats)
    out["clocks"] = clk
    return out


def source_hash(*names):
    h = hashlib.sha1()
    for nm in names:
        with open(os.path.join(ROOT, "paper_1110_2921_gb300", "csrc", nm), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def profiled_traffic(kernel, src, n_particles):
    """DRAM bytes per launch from a committed ncu capture, if the kernel source is unchanged,
    scaled from the captured case to n_particles (the kernel reads each sorted particle and
    writes each output once, so its traffic is proportional to the particle count)."""
    path = os.path.join(ROOT, "profiles", "counters.json")
    try:
        d = json.load(open(path))[kernel]
    except Exception:
        return None
    if d.get("source_hash") != source_hash(*src):
        return None
    measured, n_meas = d.get("measured_bytes"), d.get("measured_particles")
    if measured is None or not n_meas:
        return d.get("dram_bytes_per_launch")
    return measured * n_particles / n_meas


def load_golden(n, k0):
    """Stored oracle values at sampled targets of the 256^3, k0 = 4 benchmark field (written by
    tests/golden/make_field256.py from the oracle), or None for other workloads."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", "field256_k4_seed1.txt")
    if n != 256 or k0 != 4 or not os.path.exists(path):
        return None
    a = np.loadtxt(path)
    return {"index": a[:, 0].astype(np.int64), "face": a[:, 1] > 0.5, "u_near": a[:, 2:5],
            "S_near": a[:, 5:8], "u_far": a[:, 8:11], "S_far": a[:, 11:14]}


def oracle_rate(f, targets, K, nthreads=0):
    """FP64 oracle (as it stands) on a target sample: seconds and threads used."""
    import oracle
    t0 = time.perf_counter()
    oracle.direct(f["x"], f["alpha"], f["sigma"], K=K, targets=targets, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return dt, nthreads if nthreads > 0 else os.cpu_count()


def cpu_baseline(f, ntargets, single_core=True):
    """Oracle particles/s for the workload's definition (27^3 image boxes), from a timed
    sample of targets with the central 27 boxes; the 27^3-box cost is the same loop over
    729 times as many (target, source, box) triples."""
    import workload as wl
    N = len(f["x"])
    tid = wl.target_subset(N, ntargets, seed=11)
    dt, cores = oracle_rate(f, tid, K=1)
    cores = min(cores, ntargets)
    boxes_full = (2 * 13 + 1) ** 3
    value = ntargets / dt * 27.0 / boxes_full
    sample = ("%d targets of the %d-particle field, direct FP64 sum over the central 27 image boxes in %.1f s; "
              "scaled by 27/%d to the 27^3-box sum" % (ntargets, N, dt, boxes_full))
    out = {"value": value, "unit": "particles/s", "cores": cores, "kind": "oracle", "sample": sample,
           "seconds": dt}
    if single_core:  # the same loop on one core, one target
        dt1, _ = oracle_rate(f, tid[:1], K=1, nthreads=1)
        out["single_core"] = {"value": 1.0 / dt1 * 27.0 / boxes_full, "cores": 1, "seconds": dt1,
                              "sample": "1 target, central 27 boxes, scaled by 27/%d" % boxes_full}
    return out


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    import workload as wl
    n = args.n
    f = wl.make_vortex_lattice(n, args.k0, 1)
    nt = args.cpu_targets or os.cpu_count()
    for _ in range(args.warmup):
        cpu_baseline(f, nt, single_core=False)
    vals, secs = [], 0.0
    for _ in range(args.steps):
        cb = cpu_baseline(f, nt, single_core=False)
        vals.append(cb["value"])
        secs += cb["seconds"]
    value = len(vals) * nt / secs * 27.0 / (27 ** 3)
    cb["value"] = value
    cb["sample"] = "%d steps of %d targets each; " % (args.steps, nt) + cb["sample"].split("; ", 1)[0] + \
        "; scaled by 27/19683 to the 27^3-box sum"
    out = {"metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": value / PAPER_PARTICLES_PER_S, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": "vortex lattice %d^3, k0=%d, sigma=h, 27^3 periodic images" % (n, args.k0),
                      "n_particles": n ** 3, "direct_sum": "FP64 CPU oracle"},
           "cpu_baseline": cb,
           "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_timestep(args):
    """Ten Heun steps (dt = 0.01, core spreading with nu for Re_lambda = 100) and one
    reinitialisation onto the 256^3 lattice (20 iterations), mixed precision and plain FP32 M2L."""
    import numpy as np
    import torch
    import workload as wl
    import paper_1110_2921_gb300 as vf
    from paper_1110_2921_gb300 import build
    build.build()
    n = args.n
    N = n ** 3
    f = wl.make_vortex_lattice(n, args.k0, 1)
    nu = wl.viscosity_for_re_lambda(n, args.k0, 1, 100.0)
    out = {"metric": "Heun step and reinitialisation time at %d^3" % n, "unit": "ms", "nu": nu, "rho_cut": args.rho_cut,
           "dt": 0.01, "steps": 10, "reinit_iterations": 20, "runs": {}}
    for m2l in ("bf16x3", "fp32"):
        X = torch.tensor(f["x"], dtype=torch.float32, device="cuda")
        G = torch.tensor(f["alpha"], dtype=torch.float32, device="cuda")
        # rho_cut = 5 keeps 4h leaves within two rings up to sigma = 1.6 h (1 - q(5) = 1.5e-5)
        h = vf.VortexFMM(p=args.p, periodic_levels=args.periodic_levels, m2l=m2l, rho_cut=args.rho_cut)
        d0 = h.diagnostics(X, G)
        sigma = f["sigma"]
        sigma = h.rk_step(X, G, sigma, 0.01, nu)  # warm-up step
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            sigma = h.rk_step(X, G, sigma, 0.01, nu)
        e1.record()
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / 10
        # where one evaluation at the final core size goes: phases and the P2P's pair count
        Xs = X.clone()
        h.build_tree(Xs)
        h.eval(G, sigma)
        h.sync()
        phases = {k: round(v, 3) for k, v in h.timings().items()}
        info = h.tree_info()
        pairs, _ = p2p_work(X.double().cpu().numpy(), 2 * math.pi, info["depth"], info["near_rings"], sigma,
                            info["correction_rings"], args.rho_cut)
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record()
        xn, gn, res = h.reinit(X, G, sigma, n, iters=20)
        r1.record()
        torch.cuda.synchronize()
        d1 = h.diagnostics(xn, gn)
        h.close()
        out["runs"][m2l] = {"ms_per_heun_step": step_ms, "particles_per_s": N / (step_ms / 1e3),
                            "eval_at_final_sigma": {"phases_ms": phases, "depth": info["depth"],
                                                    "near_rings": info["near_rings"],
                                                    "correction_rings": info["correction_rings"],
                                                    "p2p_pairs_per_target": pairs / N,
                                                    "sigma_over_h": sigma / (2 * math.pi / n)},
                            "ms_reinit": r0.elapsed_time(r1), "reinit_residual": res, "sigma_final": sigma,
                            "total_vorticity_before": d0["total_vorticity"],
                            "total_vorticity_after_reinit": d1["total_vorticity"],
                            "sum_gamma2_before": d0["sum_gamma2"], "sum_gamma2_after_reinit": d1["sum_gamma2"]}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "timestep":
        run_timestep(args)
        return
    import numpy as np
    import torch
    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    import workload as wl
    import paper_1110_2921_gb300 as vf
    from paper_1110_2921_gb300 import build
    if rank == 0:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    n = args.n
    N = n ** 3
    f = wl.make_vortex_lattice(n, args.k0, 1 + rank)
    sigma = f["sigma"]
    X = torch.tensor(f["x"], dtype=torch.float32, device=dev)
    G = torch.tensor(f["alpha"], dtype=torch.float32, device=dev)
    U = torch.empty_like(G)
    S = torch.empty_like(G)
    cf = {} if args.concurrent_far < 0 else {"concurrent_far": args.concurrent_far}
    h = vf.VortexFMM(p=args.p, periodic_levels=args.periodic_levels, m2l=args.m2l, rho_cut=args.rho_cut,
                     depth=args.depth, **cf)
    stream = torch.cuda.current_stream()

    ev_pairs = []

    def step(mark=False):
        h.build_tree(X)
        if mark:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
        h.eval(G, sigma, out=(U, S))
        if mark:
            b.record(stream)
            ev_pairs.append((a, b))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    info = h.tree_info()
    launches = info["launches"]
    clocks = ClockSampler(dev.index) if rank == 0 else None
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    phase_ms = []
    t0.record(stream)
    for _ in range(args.steps):
        step(mark=True)
        h.sync()   # per-step phase timings are read from the library's own events
        phase_ms.append(h.timings())
    t1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ms = t0.elapsed_time(t1)
    eval_ms = statistics.median(a.elapsed_time(b) for a, b in ev_pairs)
    # outputs of the last timed step at the stored oracle targets (before other handles reuse U, S)
    gold = load_golden(n, args.k0) if (args.check and rank == 0) else None
    timed_out = None
    if gold is not None:
        idx = torch.tensor(gold["index"], dtype=torch.int64, device=dev)
        timed_out = (U[idx].double().cpu().numpy(), S[idx].double().cpu().numpy())
    clk = clocks.stop() if clocks else None
    ms_max, value = combine_ranks(ms, N, args.steps, device=dev)

    # end to end from pinned host memory through vfmm_eval_host (H2D x, gamma; D2H u, S)
    xh = torch.tensor(f["x"], dtype=torch.float32).pin_memory()
    gh = torch.tensor(f["alpha"], dtype=torch.float32).pin_memory()
    uh = torch.empty_like(gh).pin_memory()
    sh = torch.empty_like(gh).pin_memory()
    lib = vf._native
    lib.vfmm_eval_host(h.h, N, xh.data_ptr(), gh.data_ptr(), sigma, uh.data_ptr(), sh.data_ptr())
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.e2e_steps):
        lib.vfmm_eval_host(h.h, N, xh.data_ptr(), gh.data_ptr(), sigma, uh.data_ptr(), sh.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.e2e_steps
    _, e2e_value = combine_ranks(e2e_ms, N, 1, device=dev)
    # the copies of one e2e step alone (same pinned buffers, same stream): H2D of x and gamma,
    # D2H of u and S
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c2 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    X.copy_(xh, non_blocking=True)
    G.copy_(gh, non_blocking=True)
    c1.record(stream)
    uh.copy_(U, non_blocking=True)
    sh.copy_(S, non_blocking=True)
    c2.record(stream)
    torch.cuda.synchronize()
    copy_ms = (c0.elapsed_time(c1), c1.elapsed_time(c2))
    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
        return

    # roofline of the dominant kernel (P2P): FP32 ALU bound.  In the step the P2P shares the GPU
    # with the far field (side stream), so its own duration is timed on a second handle that
    # runs every phase in line (same tree, same inputs)
    ha = vf.VortexFMM(p=args.p, periodic_levels=args.periodic_levels, m2l=args.m2l, rho_cut=args.rho_cut,
                      depth=args.depth, concurrent_far=0)
    ha.build_tree(X)
    alone = []
    for it in range(4):
        ha.eval(G, sigma, out=(U, S))
        ha.sync()
        if it > 0:
            alone.append(ha.timings())
    ha.close()
    p2p_ms = statistics.mean(p["p2p"] for p in alone)
    phases_alone = {k: round(statistics.mean(p[k] for p in alone), 3) for k in alone[0]}
    R, Rc = info["near_rings"], info["correction_rings"]
    pairs, flops = p2p_work(f["x"], 2 * math.pi, info["depth"], R, sigma, Rc, args.rho_cut)
    achieved_kernel = flops / (p2p_ms / 1e3) / 1e12
    achieved = ALGO_FLOPS_PER_PAIR * pairs / (p2p_ms / 1e3) / 1e12
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    measured = measure_peaks(dev, stream) if args.peaks else None
    if measured:
        peak = measured["fp32_ffma"]
        peak_basis = "measured: FFMA probe (vfmm_probe_peak), burst"
    else:
        peak = 2 * 128 * sms * 2.070e9 / 1e12
        peak_basis = "derived: 2 x 128 FP32 lanes x %d SMs x 2070 MHz" % sms
    traffic = profiled_traffic("k_p2p_f32", ["p2p.cu"], N)
    phases = {k: round(statistics.mean(p[k] for p in phase_ms), 3) for k in phase_ms[0]}

    # the tensor-core M2L: algorithmic flops of the 121 x 121 translations (three split
    # products) on levels 3..D over the in-line M2L phase (which also holds levels 1-2 and the
    # hi/lo splits)
    nc = (args.p + 1) ** 2
    m2l_flops = 0.0
    for lvl in range(3, info["depth"] + 1):
        offs = 189 if (lvl < info["depth"] or R == 1) else 91
        m2l_flops += (8 ** lvl) * offs * 3 * nc * nc * 2 * 3
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    if args.m2l == "tf32x3" and measured:
        m2l_peak, m2l_basis = measured["tf32_tcgen05"], "measured TF32 tcgen05 probe, burst"
    elif args.m2l == "tf32x3":
        m2l_peak, m2l_basis = bf16_peak / 2, "measured BF16 burst x 1/2 (nominal TF32:BF16 ratio)"
    else:
        m2l_peak = bf16_peak
        m2l_basis = "measured BF16 burst (cuBLAS)" if "bf16_tflops" in peaks else "fallback 1.9 PFLOP/s"
    m2l_achieved = m2l_flops / (phases_alone["m2l"] / 1e3) / 1e12
    roof_m2l = {"bound": "tensor", "achieved": m2l_achieved, "peak": m2l_peak, "unit": "TFLOP/s",
                "frac": m2l_achieved / m2l_peak, "kernel": "k_m2l_lines / k_m2l_tc (levels 3..D)",
                "flops_per_eval": m2l_flops, "peak_basis": m2l_basis,
                "m2l_prec": args.m2l}

    out_err = {}
    if timed_out is not None:
        # the timed handle (27^3 images) against the oracle's full 27^3-box sum at the stored
        # targets: central 27 boxes + far-image increment (tests/golden/make_field256.py)
        full = ~np.isnan(gold["u_far"][:, 0])
        uo = gold["u_near"][full] + gold["u_far"][full]
        so = gold["S_near"][full] + gold["S_far"][full]
        ut, st = timed_out[0][full], timed_out[1][full]
        pu = np.linalg.norm(ut - uo, axis=1) / np.linalg.norm(uo, axis=1)
        ps = np.linalg.norm(st - so, axis=1) / np.linalg.norm(so, axis=1)
        face = gold["face"][full]
        out_err = {"rel_l2_u": float(np.linalg.norm(ut - uo) / np.linalg.norm(uo)),
                   "rel_l2_S": float(np.linalg.norm(st - so) / np.linalg.norm(so)),
                   "max_rel_target_u": float(pu.max()), "max_rel_target_S": float(ps.max()),
                   "targets": int(full.sum()), "face_targets": int(face.sum()),
                   "images": "27^3 boxes (the timed handle, S=2)",
                   "oracle": "FP64 direct sum, central 27 boxes + far-image increment, stored in "
                             "tests/golden/field256_k4_seed1.txt"}
    elif args.check:
        import oracle
        tid = wl.target_subset(N, args.check, seed=3)
        uo, so = oracle.direct(f["x"], f["alpha"], sigma, K=1, targets=tid)
        h0 = vf.VortexFMM(p=args.p, periodic_levels=0, m2l=args.m2l, rho_cut=args.rho_cut, depth=args.depth)
        h0.build_tree(X)
        u0, s0 = h0.eval(G, sigma)
        h0.sync()
        u0 = u0.double().cpu().numpy()[tid]
        s0 = s0.double().cpu().numpy()[tid]
        h0.close()
        pu = np.linalg.norm(u0 - uo, axis=1) / np.linalg.norm(uo, axis=1)
        ps = np.linalg.norm(s0 - so, axis=1) / np.linalg.norm(so, axis=1)
        out_err = {"rel_l2_u": float(np.linalg.norm(u0 - uo) / np.linalg.norm(uo)),
                   "rel_l2_S": float(np.linalg.norm(s0 - so) / np.linalg.norm(so)),
                   "max_rel_target_u": float(pu.max()), "max_rel_target_S": float(ps.max()),
                   "targets": args.check, "images": "27 central boxes (same tree, S=0)"}

    cb = cpu_baseline(f, args.cpu_targets or os.cpu_count()) if ws == 1 else None
    h2d = 2 * N * 3 * 4
    d2h = 2 * N * 3 * 4
    out = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": value / PAPER_PARTICLES_PER_S, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "vortex lattice %d^3 (%d particles), k0=%d, sigma=h, p=%d, 27^3 periodic images"
                   % (n, N, args.k0, args.p), "n_particles": N, "p": args.p, "m2l": args.m2l,
                   "periodic_levels": args.periodic_levels, "depth": info["depth"], "near_rings": R,
                   "correction_rings": Rc, "rho_cut": args.rho_cut,
                   "l2": "inputs (x, gamma %d MiB) larger than L2 (129 MB); no flush" % (2 * N * 3 * 4 // 2 ** 20),
                   "parallelism": "replicas" if ws > 1 else "single"},
        "e2e": {"value": e2e_value, "unit": "particles/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms, "h2d_ms_alone": copy_ms[0], "d2h_ms_alone": copy_ms[1],
                "h2d_gbs": h2d / (copy_ms[0] / 1e3) / 1e9, "d2h_gbs": d2h / (copy_ms[1] / 1e3) / 1e9},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "k_p2p_f32",
                     "pairs_per_launch": pairs, "algorithmic_flops_per_pair": ALGO_FLOPS_PER_PAIR,
                     "kernel_flops_per_launch": flops, "achieved_kernel_flops": achieved_kernel,
                     "frac_kernel_flops": achieved_kernel / peak,
                     "kernel_flops_per_pair": {"smoothed": FLOPS_PER_PAIR, "singular": FLOPS_PER_PAIR_SINGULAR},
                     "peak_basis": peak_basis},
        "roofline_m2l": roof_m2l,
        "peaks": measured,
        "excluding_tree_build": {"value": N / (eval_ms / 1e3), "unit": "particles/s", "ms_per_eval": eval_ms,
                                 "note": "median over the timed steps of vfmm_eval_velocity_stretching alone"},
        "phases_ms": phases,
        "phases_ms_in_line": phases_alone,
        "far_field": "side stream concurrent with the P2P (phases_ms overlap); phases_ms_in_line: every phase in line",
        "accuracy": out_err,
        "clocks": clk,
        "cpu_baseline": cb,
    }
    print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.barrier()


if __name__ == "__main__":
    main()
