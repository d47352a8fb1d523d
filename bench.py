#!/usr/bin/env python
"""Benchmark of the energy-minimisation prolongation loop on one GB300.

Workload: 3D 7-point finite-volume diffusion on a 128^3 grid (2,097,152 rows,
14,581,760 entries of A) with log-normal cell coefficients (sigma = 2,
seed 2), constant near kernel (k = 1), 3x3x3 aggregates (74,088 coarse
dofs), P pattern = pattern of A P0 (6,127,616 entries), 20 restricted PCG
iterations.  One step = one whole minimisation with the inputs resident in
HBM: set-up (Gram factorisation, constraint correction of P0, initial
residual), 20 iterations (masked product + projection + reductions +
Jacobi/vector updates), and the final prolongation P (in mixed precision
with its double-precision constraint restore).

Metric: restricted-PCG iterations/s (20 per step) of the whole job; the
dominant kernel (the masked product with fused projection) is reported
against the HBM roofline.  The headline line is the mixed (float bulk)
path; the plain FP64 path is reported beside it in the same line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Several GPUs run independent replicas (the method is not sharded here):
value = iterations of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KERNEL_SOURCES = ["paper_2208_02995_gb300/csrc/iter_kernels.cu",
                  "paper_2208_02995_gb300/csrc/device_util.cuh",
                  "paper_2208_02995_gb300/csrc/emin_internal.cuh"]
PROFILE = "profiles/kprod_k1_pk_fv3d128.md"

METRIC = ("restricted-PCG iterations/s and masked A·P effective HBM GB/s "
          "(% of peak), FP32 vs FP64")
WORKLOAD = 2
ITERS = 20
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (152 SMs x 2 FMA/clk x 2 flops x 2.07 GHz)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tau", action="store_true", help="skip the time-to-tau measurement")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the record of the other workloads (1, 3, 4, 5)")
    ap.add_argument("--no-sgs", action="store_true", help="skip the SGS preconditioner summary")
    ap.add_argument("--precond", choices=["jacobi", "sgs"], default="jacobi",
                    help="preconditioner of the timed runs (the headline is Jacobi)")
    ap.add_argument("--precision", choices=["both", "mixed", "fp64"], default="both",
                    help="profiling aid: run one arm only (the JSON line needs both)")
    ap.add_argument("--workload", type=int, default=WORKLOAD,
                    help="profiling aid: another workload (1-5) with --precision mixed|fp64")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only; a host-side max of the times)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group("gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# algorithmic work of one masked-product launch (Section 4; k = 1 here)
# ---------------------------------------------------------------------------
NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal (the measured copy rate is the roofline)


def kprod_bytes(prob, vbytes: int) -> int:
    """A (values + column indices + row pointers), P's pattern, Y read once,
    Y_ written once (vbytes each), and the fused projection's per-row
    factor of the Gram matrix and B_c in double (the method's factors are
    FP64 in both precisions)."""
    n, k = prob.n, prob.k
    a = prob.nnz_a * (vbytes + 4) + 4 * (n + 1)
    pat = 4 * prob.nnz_p + 4 * (n + 1)
    vec = 2 * vbytes * prob.nnz_p
    fac = n * (k * (k + 1) // 2) * 8 + prob.nc * k * 8
    return a + pat + vec + fac


def in_pattern_products(prob) -> tuple[int, int]:
    """(candidate products, products landing in P's pattern) of one
    mask_P(A Y), counted on the host from the two patterns."""
    import numpy as np
    n = prob.n
    m = np.diff(prob.P_rowptr)
    w = int(m.max())
    J = np.full((n, w), -1, dtype=np.int64)
    rows = np.repeat(np.arange(n), m)
    pos = np.arange(prob.nnz_p) - prob.P_rowptr[rows]
    J[rows, pos] = prob.P_col
    arow = np.repeat(np.arange(n), np.diff(prob.A_rowptr))
    cand = int(m[prob.A_col].sum())
    hits = 0
    for s0 in range(0, prob.nnz_a, 1 << 22):
        i = arow[s0:s0 + (1 << 22)]
        l = prob.A_col[s0:s0 + (1 << 22)]
        Ji, Jl = J[i], J[l]
        eq = (Ji[:, :, None] == Jl[:, None, :]) & (Ji[:, :, None] >= 0)
        hits += int(eq.sum())
    return cand, hits


def in_pattern_products_blocked(prob, nb=3, kb=6):
    """(candidate, in-pattern) products of one mask_P(A Y) for a node-blocked
    problem (nb dofs per node, columns of P in groups of kb per aggregate,
    the nb rows of a node sharing their patterns): every stored nb x nb block
    (v, b) of A contributes nb*nb*|J_b| candidates and nb*nb*|J_v & J_b|
    in-pattern products, counted at node level from the aggregate sets."""
    import numpy as np
    nn = prob.n // nb
    Ap, Aj, Pp, Pj = prob.A_rowptr, prob.A_col, prob.P_rowptr, prob.P_col
    na = np.diff(Pp[0:prob.n + 1:nb]) // (nb * kb)  # aggregates per node
    w = int(na.max())
    S = np.full((nn, w), -1, dtype=np.int64)
    first = Pp[0:prob.n:nb]
    for q in range(w):
        has = na > q
        S[has, q] = Pj[first[has] + kb * q] // kb
    # node neighbours: the nb rows of a node hold nb * deg entries each
    deg = np.diff(Ap[0:prob.n + 1:nb]) // (nb * nb)
    v = np.repeat(np.arange(nn), deg)
    row0 = Ap[0:prob.n:nb]
    j = np.arange(len(v)) - np.repeat(np.cumsum(deg) - deg, deg)
    b = Aj[row0[v] + nb * j] // nb
    cand = int(nb * nb * kb * na[b].sum())
    hits = 0
    for s0 in range(0, len(v), 1 << 20):
        Sv, Sb = S[v[s0:s0 + (1 << 20)]], S[b[s0:s0 + (1 << 20)]]
        eq = (Sv[:, :, None] == Sb[:, None, :]) & (Sv[:, :, None] >= 0)
        hits += int(eq.sum())
    return cand, nb * nb * kb * hits


def products(prob):
    """(candidate, in-pattern) products of one masked product, or (0, 0)
    when neither counting scheme applies."""
    import numpy as np
    if int(np.diff(prob.P_rowptr).max(initial=0)) <= 8:
        return in_pattern_products(prob)
    if prob.k == 6 and prob.n % 3 == 0 and prob.meta.get("kind") == "elasticity":
        return in_pattern_products_blocked(prob)
    return 0, 0


def captured_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None when the kernel sources changed since that capture."""
    import hashlib
    try:
        h = hashlib.sha256()
        for f in KERNEL_SOURCES:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        txt = open(os.path.join(ROOT, PROFILE)).read()
    except OSError:
        return None
    fields = dict(line.split(":", 1) for line in txt.splitlines()
                  if line.startswith(("traffic_bytes_per_launch:", "source_fingerprint:")))
    if fields.get("source_fingerprint", "").strip() != h.hexdigest():
        return None
    try:
        return int(fields["traffic_bytes_per_launch"].strip())
    except (KeyError, ValueError):
        return None


def kprod_flops(prob, hits: int) -> int:
    """FP64 flops of one masked product with projection and y^T y_:
    2 per in-pattern product, 4 k per entry of P (B_i^T x and x - B_i c),
    2 k^2 per row (G_i^{-1} t) and 2 per entry (the dot)."""
    k = prob.k
    return 2 * hits + 4 * k * prob.nnz_p + 2 * k * k * prob.n + 2 * prob.nnz_p


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self, period_ms: int = 10):
        """Start sampling every period_ms and wait (at most 5 s) until the
        first sample is written, so that the timed region that follows is
        covered from its start."""
        import tempfile
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", str(period_ms)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t_end = time.time() + 5.0
        while time.time() < t_end and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx = max(mx, float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def time_steps(ctx, out, K, W, stream, dist, iters=ITERS):
    """W untimed steps, then K timed steps; CUDA events on the library's
    stream, barrier + synchronize on both sides."""
    import torch

    def step():
        ctx.reset()
        ctx.iterate(iters, 0.0)
        ctx.get_p(out)

    for _ in range(W):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(K):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    return t0.elapsed_time(t1)


def headline_config(dist):
    """The workload of the headline line, shared by both arms."""
    return {
        "workload": ("3D 7-point FV diffusion 128^3 (n=2,097,152, nnz(A)=14,581,760), "
                     "log-normal kappa sigma=2 seed 2, k=1, 3x3x3 aggregates "
                     "(n_c=74,088), nnz(P)=6,127,616, 20 restricted PCG iterations"),
        "step": "set-up + 20 iterations + final P, inputs resident in HBM",
        "precision": "FP32 vs FP64: value = mixed (float A/P/products, double Gram "
                     "factorisation, reductions and final constraint restore), key fp64 = "
                     "plain FP64; the reference arm is the FP64 oracle",
        "l2": "inputs larger than L2 (A 175 MB + P vectors 123 MB > 129 MB)",
        "parallelism": f"replicas x{dist.world}",
    }


def run_ours(args, dist):
    import numpy as np
    import torch

    from paper_2208_02995_gb300 import inputs
    from paper_2208_02995_gb300.emin import (Context, emin_set_timing, emin_timing)

    torch.cuda.set_device(dist.local)
    prob = inputs.config(args.workload)
    iters = prob.iters
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"

    cand, hits = products(prob)
    stream = torch.cuda.Stream()
    results = {}
    precs = ("mixed", "fp64") if args.precision == "both" else (args.precision,)
    for prec in precs:
        with torch.cuda.stream(stream):
            ctx = Context(prob, precision=prec, stream=stream, precond=args.precond)
            out = torch.empty(prob.nnz_p, dtype=torch.float64, device="cuda")
        clocks = Clocks(dist.local) if prec == "mixed" else None
        l0 = emin_timing(ctx.h)["total_launches"]
        # the timed region also times the masked product of every 4th iteration
        emin_set_timing(ctx.h, 4)
        if clocks:
            clocks.start()
        ms = time_steps(ctx, out, args.steps, args.warmup, stream, dist, iters)
        clk = clocks.stop() if clocks else None
        tm = emin_timing(ctx.h)
        emin_set_timing(ctx.h, 0)
        launches = tm["total_launches"] - l0
        per_step_launches = launches / (args.steps + args.warmup)
        ms_max = dist.max(ms)
        kprod_avg_s = tm["ms"][0] / max(tm["launches"][0], 1) / 1e3
        results[prec] = {
            "ms": ms_max, "clocks": clk,
            "gpu_launches": int(round(per_step_launches * args.steps)),
            "kprod_avg_us": kprod_avg_s * 1e6,
            "kernel_share": {"kprod_ms": tm["ms"][0], "kprod_launches": int(tm["launches"][0])},
            "P": out.cpu().numpy(),
            "E": ctx.energy(),
        }
        ctx.close()
    if args.precision != "both" or args.workload != WORKLOAD:
        r = results[precs[0]]
        return {"workload": prob.name, "precision": precs[0], "precond": args.precond,
                "iters": iters,
                "ms_per_step": r["ms"] / args.steps,
                "kprod_avg_us": r["kprod_avg_us"], "kernel_ms": r["kernel_share"],
                "gpu_launches": r["gpu_launches"]}
    # end-to-end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(prob, args, dist)

    m = results["mixed"]
    K = args.steps
    value = dist.world * ITERS * K / (m["ms"] / 1e3)
    b32 = kprod_bytes(prob, 4)
    traffic = captured_traffic()
    ach = b32 / (m["kprod_avg_us"] * 1e-6) / 1e9
    f = results["fp64"]
    fl = kprod_flops(prob, hits)
    ach64 = fl / (f["kprod_avg_us"] * 1e-6) / 1e12
    f64peak = fp64_peak(stream)
    b64 = kprod_bytes(prob, 8)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "iterations/s",
        "n_gpus": dist.world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": m["ms"] / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": headline_config(dist),
        "roofline": {
            "kernel": "masked product + projection + y^T y_ (k_kprod_k1_pk<float>, packed SELL-32 plan)",
            "bound": "hbm",
            "achieved": ach,
            "peak": hbm_peak,
            "unit": "GB/s",
            "frac": ach / hbm_peak,
            "traffic": traffic,
            "algorithmic_bytes": b32,
            "avg_launch_us": m["kprod_avg_us"],
            "peak_source": hbm_src,
            # the same launch against the nominal HBM3e rate, the DRAM rate the
            # ncu traffic implies at the loop's launch time, and the products
            "frac_of_nominal_8tbs": ach / NOMINAL_HBM_GBS,
            "dram_gbs": (traffic / (m["kprod_avg_us"] * 1e-6) / 1e9) if traffic else None,
            "in_pattern_products_per_s": hits / (m["kprod_avg_us"] * 1e-6),
            "candidate_products": cand,
            "in_pattern_products": hits,
        },
        "fp64": {
            "value": dist.world * ITERS * K / (f["ms"] / 1e3),
            "unit": "iterations/s",
            "ms_per_step": f["ms"] / K,
            "dtype": "f64",
            "roofline": {
                "kernel": "masked product + projection + y^T y_ (k_kprod_k1_pk<double>, packed SELL-32 plan)",
                "bound": "alu",
                "achieved": ach64,
                "peak": f64peak["tflops"],
                "unit": "TFLOP/s",
                "frac": ach64 / f64peak["tflops"],
                "traffic": None,
                "flops": fl,
                "hbm_gbs": b64 / (f["kprod_avg_us"] * 1e-6) / 1e9,
                "avg_launch_us": f["kprod_avg_us"],
                "peak_source": f64peak["source"],
                "peak_nominal": FP64_PEAK_TFLOPS,
                "frac_of_nominal": ach64 / FP64_PEAK_TFLOPS,
                "peak_nominal_source": "152 SMs x 2 FP64 FMA/clk x 2 flops x 2070 MHz",
            },
            "gpu_launches": f["gpu_launches"],
        },
        "kernel_ms": {p: results[p]["kernel_share"] for p in results},
        "gpu_launches": m["gpu_launches"],
        "clocks": m["clocks"],
        "e2e": e2e,
        "mixed_vs_fp64": {
            "P_rel_diff": float(np.linalg.norm(results["mixed"]["P"] - results["fp64"]["P"]) /
                                np.linalg.norm(results["fp64"]["P"])),
            "time_to_P_ratio": f["ms"] / m["ms"],
        },
    }
    if not args.no_workloads:
        clk = Clocks(dist.local)
        clk.start()
        wl = {"2": {"workload": line["config"]["workload"], "note": "the headline above",
                    "mixed": {"iterations_per_s": value, "kprod_avg_us": m["kprod_avg_us"],
                              "kprod_frac_hbm": ach / hbm_peak},
                    "fp64": {"iterations_per_s": line["fp64"]["value"],
                             "kprod_avg_us": f["kprod_avg_us"],
                             "kprod_frac_fp64": ach64 / f64peak["tflops"]}}}
        for w in sorted(WORKLOAD_STEPS):
            wl[str(w)] = run_workload(w, args, dist, stream, hbm_peak, f64peak)
        wl["clocks"] = clk.stop()
        wl["peaks"] = {"hbm_gbs": hbm_peak, "hbm_source": hbm_src, "fp64": f64peak}
        line["workloads"] = wl
    if not args.no_tau:
        line["time_to_tau"] = time_to_tau(prob, stream)
    if not args.no_sgs:
        line["sgs"] = sgs_summary(prob, stream, dist)
    if dist.world == 1 and not args.no_cpu_baseline and dist.rank == 0:
        line["cpu_baseline"], oracle_P, oracle_E = cpu_baseline(prob)
        line["vs_oracle"] = versus_oracle(prob, results, oracle_P, oracle_E)
    return line


# the other workloads of the metric (the headline is workload 2): (warm-up,
# timed steps) per workload, sized so that each arm takes a few seconds; the
# oracle's P after the same iterations is compared where it finishes in
# seconds on the host
WORKLOAD_STEPS = {1: (5, 20), 3: (3, 10), 4: (3, 10), 5: (3, 4)}
ORACLE_PARITY = (1, 4)
BACKWARD = (4, 5)  # workloads whose configuration includes the implicit adjoint


def fp64_peak(stream):
    """Measured FP64 FMA rate of this GPU (TFLOP/s) from the library's probe,
    best of three launches, with the nominal rate for reference."""
    from paper_2208_02995_gb300.emin import emin_fma_rate
    best = max(emin_fma_rate("fp64", stream)[0] for _ in range(3))
    return {"tflops": 2.0 * best / 1e12, "source": "measured: emin_fma_rate (independent "
            "DFMA chains on every SM, CUDA events, best of 3)", "nominal_tflops": FP64_PEAK_TFLOPS}


def run_workload(w, args, dist, stream, hbm_peak, f64peak):
    """One record of the per-workload table: both precisions, the masked
    product's average CUDA-event time per launch against its roofline, the
    adjoint where the configuration names it, the oracle's P where it is fast."""
    import numpy as np
    import torch

    from paper_2208_02995_gb300 import inputs
    from paper_2208_02995_gb300.emin import Context, emin_set_timing, emin_timing
    prob = inputs.config(w)
    cand, hits = products(prob)
    W, K = WORKLOAD_STEPS[w]
    rec = {"workload": inputs.CONFIG_NAMES[w], "n": prob.n, "nnz_a": prob.nnz_a,
           "nnz_p": prob.nnz_p, "nc": prob.nc, "k": prob.k, "iterations": prob.iters,
           "candidate_products": cand, "in_pattern_products": hits, "warmup": W, "steps": K,
           "step": f"set-up + {prob.iters} iterations + final P, inputs resident in HBM"}
    Ps = {}
    for prec in ("mixed", "fp64"):
        with torch.cuda.stream(stream):
            ctx = Context(prob, precision=prec, stream=stream)
            out = torch.empty(prob.nnz_p, dtype=torch.float64, device="cuda")
        emin_set_timing(ctx.h, 1)
        ms = time_steps(ctx, out, K, W, stream, dist, prob.iters)
        tm = emin_timing(ctx.h)
        emin_set_timing(ctx.h, 0)
        ms = dist.max(ms)
        kus = tm["ms"][0] / max(tm["launches"][0], 1) * 1e3
        v = 4 if prec == "mixed" else 8
        b = kprod_bytes(prob, v)
        r = {"ms_per_step": ms / K, "iterations_per_s": dist.world * prob.iters * K / (ms / 1e3),
             "kprod_avg_us": kus, "kprod_launches": int(tm["launches"][0]),
             "kprod_algorithmic_bytes": b, "kprod_gbs": b / (kus * 1e-6) / 1e9}
        r["kprod_frac_hbm"] = r["kprod_gbs"] / hbm_peak
        if prec == "fp64" and hits:
            fl = kprod_flops(prob, hits)
            r["kprod_flops"] = fl
            r["kprod_tflops"] = fl / (kus * 1e-6) / 1e12
            r["kprod_frac_fp64"] = r["kprod_tflops"] / f64peak["tflops"]
        if w in BACKWARD:
            # L = tr(P^T A P) + ||P||_F^2 of the P just formed; the adjoint runs
            # as many restricted PCG steps as the forward
            _, dE, _ = ctx.energy_grad(out, 1.0, want_energy=False, want_dX=True)
            dLdP = dE + 2.0 * out
            ctx.backward(dLdP, prob.iters, 0.0)
            torch.cuda.synchronize()
            t = time.perf_counter()
            reps = 3
            for _ in range(reps):
                ctx.backward(dLdP, prob.iters, 0.0)
            torch.cuda.synchronize()
            r["backward_ms"] = (time.perf_counter() - t) / reps * 1e3
            r["backward"] = (f"implicit adjoint (FP64), {prob.iters} restricted PCG steps, "
                             "mask_P(A U), mask_A(U P^T), G^-1 B^T; host-timed per call")
        Ps[prec] = (out.cpu().numpy(), ctx.energy())
        rec[prec] = r
        ctx.close()
        del ctx, out
        torch.cuda.empty_cache()
    rec["mixed_vs_fp64_P_rel"] = float(np.linalg.norm(Ps["mixed"][0] - Ps["fp64"][0]) /
                                       np.linalg.norm(Ps["fp64"][0]))
    rec["time_to_P_ratio"] = rec["fp64"]["ms_per_step"] / rec["mixed"]["ms_per_step"]
    if w in ORACLE_PARITY and dist.rank == 0:
        from oracle.oracle import Oracle
        o = Oracle(prob)
        ref = o.minimize(prob.iters, 0.0)
        Eref = o.energy(ref["P"])
        rec["vs_oracle"] = {p: {"P_rel_fro": float(np.linalg.norm(Ps[p][0] - ref["P"]) /
                                                    np.linalg.norm(ref["P"])),
                                "E_rel": abs(Ps[p][1] - Eref) / abs(Eref),
                                "constraint_max_abs": constraint_error(prob, Ps[p][0])}
                            for p in Ps}
    else:
        rec["constraint_max_abs"] = {p: constraint_error(prob, Ps[p][0]) for p in Ps}
    return rec


def constraint_error(prob, P):
    """max |P B_c - B| over all entries (the constraint of Eq. (10))."""
    import numpy as np
    rows = np.repeat(np.arange(prob.n), np.diff(prob.P_rowptr))
    Bc = np.asarray(prob.Bc).reshape(prob.nc, prob.k)
    B = np.asarray(prob.B).reshape(prob.n, prob.k)
    worst = 0.0
    for c in range(prob.k):
        PB = np.bincount(rows, weights=P * Bc[prob.P_col, c], minlength=prob.n)
        worst = max(worst, float(np.abs(PB - B[:, c]).max(initial=0.0)))
    return worst


def versus_oracle(prob, results, oracle_P, oracle_E):
    """The timed runs' P (after the last timed step: set-up + 20 iterations)
    against the oracle's P of the same workload and iteration count."""
    import numpy as np
    out = {"iterations": ITERS, "oracle_energy": oracle_E}
    for prec, r in results.items():
        out[prec] = {
            "P_rel_fro": float(np.linalg.norm(r["P"] - oracle_P) / np.linalg.norm(oracle_P)),
            "E_rel": abs(r["E"] - oracle_E) / abs(oracle_E),
            "constraint_max_abs": constraint_error(prob, r["P"]),
        }
    return out


TAUS = (0.1, 1e-3, 1e-6)
TAU_MAXIT = 200


def sgs_summary(prob, stream, dist, steps=20, warm=3):
    """The projected block SGS preconditioner (M_2) beside Jacobi (M_1): the
    same timed step (set-up + 20 iterations + P) in both precisions, the
    energy reached after 5, 10 and 20 iterations with each preconditioner
    (FP64), and the time to the energy criterion with M_2."""
    import torch

    from paper_2208_02995_gb300.emin import Context
    out = {"step": "set-up + 20 iterations + final P, as the headline"}
    for prec in ("mixed", "fp64"):
        with torch.cuda.stream(stream):
            ctx = Context(prob, precision=prec, stream=stream, precond="sgs")
            P = torch.empty(prob.nnz_p, dtype=torch.float64, device="cuda")
        ms = time_steps(ctx, P, steps, warm, stream, dist, ITERS) / steps
        out[prec] = {"iterations_per_s": ITERS / (ms / 1e3), "ms_per_step": ms}
        ctx.close()
    energy = {}
    for pc in ("jacobi", "sgs"):
        with torch.cuda.stream(stream):
            ctx = Context(prob, precision="fp64", stream=stream, precond=pc)
        rows = {"0": ctx.energy()}
        for its in (5, 10, 20):
            ctx.reset()
            ctx.iterate(its)
            rows[str(its)] = ctx.energy()
        energy[pc] = rows
        ctx.close()
    out["energy_fp64"] = energy
    out["time_to_tau"] = time_to_tau(prob, stream, precond="sgs")
    return out


def time_to_tau(prob, stream, reps=5, warm=2, precond="jacobi"):
    """Time to the energy stop test of Eq. (relRed): one whole minimisation
    (set-up, iterations until dE_k < tau dE_1 with at most TAU_MAXIT, P) per
    sample, CUDA events on the library's stream, for the paper's default
    tau = 0.1 and two tighter ones, in both precisions."""
    import torch

    from paper_2208_02995_gb300.emin import Context
    out = {"maxit": TAU_MAXIT, "unit": "ms per minimisation (set-up + iterations to the "
           "stop test + P), mean of 5 after 2 warm-up", "samples": reps}
    for prec in ("mixed", "fp64"):
        with torch.cuda.stream(stream):
            ctx = Context(prob, precision=prec, stream=stream, precond=precond)
            P = torch.empty(prob.nnz_p, dtype=torch.float64, device="cuda")
        rows = []
        for tau in TAUS:
            done = [0]

            def step():
                ctx.reset()
                done[0] = ctx.iterate(TAU_MAXIT, tau)[0]
                ctx.get_p(P)

            for _ in range(warm):
                step()
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(reps):
                step()
            t1.record(stream)
            torch.cuda.synchronize()
            rows.append({"tau": tau, "iterations": int(done[0]),
                         "ms": t0.elapsed_time(t1) / reps})
        out[prec] = rows
        ctx.close()
    return out


def run_e2e(prob, args, dist):
    """Same metric through the C ABI with host buffers: every step creates a
    context from pinned host arrays (H2D copies), iterates, reads P back to
    pinned host memory (D2H) and destroys the context."""
    import numpy as np
    import torch

    from paper_2208_02995_gb300.emin import Context

    pinned = []
    for a in prob.arrays():
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        pinned.append(t.numpy())
    out = torch.empty(prob.nnz_p, dtype=torch.float64).pin_memory().numpy()
    h2d = sum(a.nbytes for a in pinned)
    d2h = out.nbytes
    K = max(1, min(args.steps, 5))

    def step():
        c = Context(n=prob.n, nc=prob.nc, k=prob.k, arrays=pinned, precision="mixed",
                    on_device=False)
        c.iterate(ITERS, 0.0)
        c.get_p(out)
        c.close()

    step()
    torch.cuda.synchronize()
    dist.barrier()
    t = time.perf_counter()
    for _ in range(K):
        step()
    torch.cuda.synchronize()
    el = dist.max(time.perf_counter() - t)
    return {"value": dist.world * ITERS * K / el, "unit": "iterations/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": K, "precision": "mixed"}


def cpu_baseline(prob):
    """The FP64 oracle as it stands (single thread) on the host: one whole
    minimisation (set-up + 20 iterations) of the same workload.  Returns the
    timing line and the oracle's P and energy (untimed) for the parity fields."""
    from oracle.oracle import Oracle
    t = time.perf_counter()
    o = Oracle(prob)
    res = o.minimize(ITERS, 0.0)
    el = time.perf_counter() - t
    line = {"value": ITERS / el, "unit": "iterations/s", "cores": 1, "kind": "oracle",
            "sample": "one whole minimisation (set-up + 20 iterations) of the 128^3 workload",
            "seconds": el}
    return line, res["P"], o.energy(res["P"])


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, dist):
    from oracle.oracle import Oracle
    from paper_2208_02995_gb300 import inputs

    prob = inputs.config(WORKLOAD)
    its = ITERS

    def step():
        o = Oracle(prob)
        o.minimize(its, 0.0)

    # the first warm-up step (one whole minimisation) is timed on the host:
    # every step stays a whole minimisation when the remaining steps fit in
    # about 4 minutes, else each is a bounded sample of fewer iterations
    budget_s = 240.0
    t = time.perf_counter()
    step()
    first_s = time.perf_counter() - t
    rest = args.steps + max(args.warmup - 1, 0)
    if rest * first_s > budget_s:
        its = max(1, int(ITERS * budget_s / (rest * first_s)))
    for _ in range(args.warmup - 1):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t
    value = its * args.steps / el
    sample = (f"{'whole minimisation' if its == ITERS else 'sample'}: set-up + {its} iterations "
              f"of the 128^3 workload per step, single-threaded FP64 oracle")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iterations/s",
        "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(dist),
        "arm": "the FP64 CPU oracle (plain C, single thread) on the host cores",
        "cpu_baseline": {"value": value, "unit": "iterations/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "iterations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def main():
    args = parse()
    dist = Dist()
    try:
        if args.impl == "reference":
            if dist.rank == 0:
                print(json.dumps(run_reference(args, dist)), flush=True)
            return
        line = run_ours(args, dist)
        if dist.rank == 0:
            print(json.dumps(line), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
