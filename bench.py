#!/usr/bin/env python
"""Benchmark of the factored Schur complement solve (arXiv 1312.5653, Sec. 3.1 + Sec. 4 + Sec. 5).

Workload: 2D unit square, 1024 x 1024 Q1 elements (1,046,529 interior dofs), homogeneous
Dirichlet boundary, 64 x 64 subdomains of 16 x 16 elements, beta cycling over
{1e-2, 1e-4, 1e-6, 1e-8}, one right-hand side b = M y_bar per step with y_bar = seeded i.i.d.
N(0,1) nodal values smoothed by 3 damped Jacobi sweeps (synthetic; the paper's targets are
analytic, no dataset).

One step = the whole path for one (beta, b): schur_setup (assembly, batched subdomain LDL^T,
local operators, coarse factorisation) + schur_solve (FETI-DP GMRES with FP64 refinement and the
-Im(z)/gamma shortcut) + schur_destroy.  Headline = mixed precision (complex FP32 FETI-DP, FP64
refinement); the plain FP64 form and the cached-factor solve rate are reported beside it.
L2 is flushed (256 MB write) between timed steps.

The roofline reported is that of the single kernel with the largest share of the step, timed by
CUDA events inside the timed region, against arithmetic peaks measured on the same GPU at the start
(schur_peak_probe) and the measured HBM copy bandwidth; its DRAM traffic per launch comes from the
committed ncu summary while the kernel's sources are unchanged.

Further rows in the same JSON line (rank 0, skipped with --no-extra): the 3D precision form
(128^3, 16^3 subdomains, mixed vs FP64), the full-space KKT form (512^2, MINRES, 8 right-hand
sides, two betas) and the serving stream (2000 requests of mixed 2D/3D sizes, 6 betas, 1-16
right-hand sides, Poisson arrivals at 0.8 x measured capacity; p50/p99 latency and batching
counters, mixed vs FP64 on the first 60 requests of the same stream).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-extra]
                  [--serve-requests R] [--peaks] [--ncu-case 2d|3d]
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_EL, N_SUB, BETAS = 1024, 64, (1e-2, 1e-4, 1e-6, 1e-8)
WORKLOAD = "2d-q1-1024x1024-dirichlet-64x64sub-16x16el-smoothed-noise-beta-sweep"
METRIC = "MDoF/s (S-solves at relerr<=1e-8, setup+solve per solve)"
OUTER_TOL = 1e-10  # ||b - A z|| / ||b|| at which the FP64 refinement stops (relerr ~1e-12 here)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=8)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-extra", action="store_true", help="skip the 3D, full-space and serving rows")
    p.add_argument("--serve-requests", type=int, default=2000, help="requests in the serving stream")
    p.add_argument("--peaks", action="store_true", help="only measure the arithmetic peaks and print them")
    p.add_argument("--ncu-case", nargs="?", const="2d", choices=["2d", "3d"],
                   help="one setup + one solve for profiler captures: 2d = the headline workload (beta = 1e-4); "
                        "3d = 64^3 Q1 elements in 8^3 subdomains of 8^3 (beta = 1e-6), the layer size of the "
                        "128^3 workload on 512 subdomains")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def rank_seed(rank):
    """Seed of the right-hand side a rank solves: independent problems per rank (weak scaling)."""
    return 1 + rank


def max_over_ranks(torch, value, device, world):
    """The job's time: the largest of the ranks' values (barrier-bracketed timed regions)."""
    if world == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, n, steps, total_ms):
    """Whole-job MDoF/s: every rank solves n dofs per step; time = max over ranks."""
    return world * n * steps / (total_ms / 1e3) / 1e6


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [t.strip() for t in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_solve(b, beta):
    import oracle
    t0 = time.perf_counter()
    x = oracle.fd_schur_solve(2, N_EL, beta, b)
    return x, time.perf_counter() - t0


def cpu_model():
    """The host CPU model name (lscpu), or the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def run_reference(args, rank, world):
    """The oracle (FP64 fast diagonalisation in C, sine-transform lines on every host core)."""
    if rank != 0:
        return
    import oracle
    from paper_1312_5653_gb300 import inputs
    oracle.build()
    ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    yb = inputs.smoothed_noise(2, N_EL, seed=1)
    b = oracle.apply_M(2, N_EL, yb)
    n = b.size
    for i in range(args.warmup):
        cpu_oracle_solve(b, BETAS[i % 4])
    ts = []
    for i in range(args.steps):
        ts.append(cpu_oracle_solve(b, BETAS[i % 4])[1])
    t = float(np.sum(ts))
    val = n * args.steps / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MDoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_dofs": n, "beta": list(BETAS), "nrhs_per_step": 1},
            "cpu_baseline": {"value": val, "unit": "MDoF/s", "cores": ncores, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": "one full-size right-hand side per step, fast-diagonalisation oracle "
                                       "(dense sine transforms, lines shared over %d OpenMP threads)" % ncores},
            "e2e": {"value": val, "unit": "MDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def flush_l2(buf):
    buf.add_(1.0)


# iterations of each arithmetic peak probe (a few milliseconds each on a GB300)
PEAK_ITERS = {0: 100, 1: 2000, 2: 100, 3: 50000}


def measure_peaks(S, peaks_file):
    """Arithmetic peaks measured on this GPU (schur_peak_probe: FP64 FMA, FP32 FMA, FP64 tensor
    MMA, TF32 tcgen05 MMA; best of three) and the HBM copy bandwidth of MEASURED_PEAKS.json."""
    out = {}
    for kind, name in S.PEAK_KINDS.items():
        out[name] = max(S.schur_peak_probe(kind, PEAK_ITERS[kind]) for _ in range(3))
    out["unit"] = "TFLOP/s"
    out["hbm_gbs"] = peaks_file.get("hbm_gbs")
    out["source"] = "schur_peak_probe on this GPU (best of 3); hbm_gbs from MEASURED_PEAKS.json"
    return out


def bcr_tasks(L):
    """Odd-even reduction schedule over L layers: per level the eliminated layers j and whether
    each has a remaining left (p) and right (q) neighbour."""
    rem = list(range(L))
    levels = []
    while rem:
        lev = []
        for t in range(0, len(rem), 2):
            lev.append((t > 0, t + 1 < len(rem)))
        levels.append(lev)
        rem = rem[1::2]
    return levels


# algorithmic traffic per launch (HBM-bound categories) or work per step (ALU-bound setup
# categories, which bracket several launches) of each kernel category, 2D square workload
def algorithmic(cat, info, prec_bytes):
    nsd, nD, nc, nlam, nco = info["n_sub"], info["n_delta"], 4, info["n_lambda"], info["n_coarse"]
    b = int(round(info["n_local"] ** 0.5))  # local layer size = layers (s + 1)
    cb_, cL = int(round(nco ** 0.5)), int(round(nco ** 0.5))  # coarse layer size, layers
    cb = 2 * prec_bytes  # complex entry
    cmac = 8  # real flops of one complex multiply-add
    packed = ((nD * (nD + 1) // 2) + 1) // 2 * 2  # stored upper triangle of one symmetric block
    if cat == "apply_F":
        # packed F and F_rc of every subdomain, the multipliers, the outputs Y and T_c
        byts = nsd * (packed + nD * nc) * cb + nlam * cb + nsd * (nD + nc) * cb
        return "hbm", byts
    if cat == "apply_S":
        byts = nsd * packed * cb + nlam * cb + nsd * nD * cb
        return "hbm", byts
    if cat == "coarse_apply":
        # level 0 of the reduction applied around the stored inverse of the reduced matrix: the
        # level-0 blocks (forward: A_pj D_j^-1 and (D_j^-1 A_jq)^T per neighbour; backward: D_j^-1
        # and both couplings), the upper 32 x 32 tiles of the reduced inverse, the corner couplings
        # of every subdomain (read by both steps), the reduced vectors and the output
        lev0 = bcr_tasks(cL)[0]
        nblk = sum(p + q for p, q in lev0) * 2 + len(lev0)
        nr = cb_ * (cL - len(lev0))
        nct = (nr + 31) // 32
        return "hbm", (nblk * cb_ * cb_ + nct * (nct + 1) // 2 * 1024 + 2 * nsd * nc + 2 * nr + nco) * cb
    if cat == "scatter":
        return "hbm", nlam * cb + 2 * nlam * cb
    if cat == "form":
        # forward and backward layer sweeps of nD + nc right-hand sides on every subdomain
        return "alu", nsd * 2 * b * b * b * (nD + nc) * cmac
    if cat == "form_corner":
        # K_cc ahead of the formation: the forward sweep of the nc corner columns
        return "alu", nsd * b * b * b * nc * cmac
    if cat == "factor":
        # per layer: explicit inverse of the b x b pivot block and the Schur update
        return "alu", nsd * b * (b ** 3 + 2 * 3 * b * b) * cmac
    if cat == "coarse_inverse":
        # cyclic-reduction solve of the reduced matrix (layers surviving level 0) with its n_r
        # identity columns: b x b by b x n_r products
        Lr = cL - len(bcr_tasks(cL)[0])
        ntask = sum(1 + p + q for lev in bcr_tasks(Lr) for p, q in lev) * 2
        return "alu", ntask * cb_ * cb_ * (cb_ * Lr) * cmac
    if cat == "coarse_setup":
        # FP64 reduction: level 0 banded (2D: tridiagonal inverses and 3-term products), the
        # other levels dense (Gauss-Jordan b^3 plus the products Lp, Lq, D_p, A_pq, D_q)
        tot = 0
        for lv, lev in enumerate(bcr_tasks(cL)):
            for p, q in lev:
                nprod = p + q + p + (p and q) + q
                tot += (1 + nprod) * (3 * cb_ * cb_ if lv == 0 else cb_ ** 3)
        return "alu", tot * cmac
    return None, None


CATEGORIES = ["factor", "form", "coarse_setup", "local_rhs", "apply_F", "apply_S", "scatter", "coarse_apply",
              "corner", "gmres_dots", "gmres_update", "gmres_other", "recover", "assemble_z", "residual",
              "coarse_inverse", "interior", "form_corner"]
# profiling categories that hold exactly one kernel on the 2D mixed workload (16^2-element
# subdomains: layer size 17, 60 interface slots, one right-hand side)
KERNEL_OF = {"form": "k_form_rr_cols<float, 17>", "apply_F": "k_local_apply_1<float, 0>",
             "apply_S": "k_local_apply_1<float, 1>", "assemble_z": "k_assemble_z<float>"}
# source files whose contents determine each kernel (a recorded DRAM traffic figure is used only
# while their hash is the one recorded with it)
KERNEL_SOURCES = {"k_form_rr_cols<float, 17>": ["warp.cuh", "layered.cuh", "common.cuh"],
                  "k_local_apply_1<float, 0>": ["kernels.cuh", "common.cuh"],
                  "k_local_apply_1<float, 1>": ["kernels.cuh", "common.cuh"],
                  "k_assemble_z<float>": ["kernels.cuh", "common.cuh"]}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic_2d_1024_mixed.md")


def kernel_source_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, "paper_1312_5653_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, path=TRAFFIC_FILE):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu summary, or None when
    there is none or the kernel's sources changed since it was captured.  Rows of the summary:
    | `kernel` | launches | dram bytes per launch | source hash |"""
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        f = [t.strip() for t in ln.strip().strip("|").split("|")]
        if len(f) >= 4 and f[0] == "`%s`" % kernel:
            try:
                byts = float(f[2].replace(",", ""))
            except ValueError:
                return None
            return byts if f[3].strip("`") == kernel_source_hash(kernel) else None
    return None


def category_roofline(cat, info, launches, total_ms, steps, peaks):
    """Roofline of one profiling category: algorithmic bytes (HBM-bound) or flops (ALU-bound) per
    launch over the event-timed average launch, against the measured peak of its bound."""
    prec_bytes = 4
    bound, algo = algorithmic(cat, info, prec_bytes)
    if bound is None or launches == 0:
        return None
    per_step = launches / steps
    if bound == "hbm":
        avg_s = total_ms / launches / 1e3
        ach = algo / avg_s / 1e9
        peak = peaks.get("hbm_gbs") or 6800.0
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                "launches": launches, "avg_us": avg_s * 1e6, "algorithmic_bytes_per_launch": algo,
                "peak_source": "measured copy (MEASURED_PEAKS.json)" if peaks.get("hbm_gbs") else "fallback"}
    # ALU categories: the model counts one step's work, spread over its launches
    avg_s = total_ms / launches / 1e3
    per_launch = algo / per_step
    is64 = cat in ("coarse_setup",)
    pk = peaks.get("fp64_fma" if is64 else "fp32_fma")
    ach = per_launch / avg_s / 1e12
    out = {"bound": "alu", "precision": "fp64" if is64 else "fp32", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
           "frac": ach / pk if pk else None, "traffic": None, "launches": launches, "avg_us": avg_s * 1e6,
           "algorithmic_flops_per_launch": per_launch,
           "peak_source": "measured %s FMA (schur_peak_probe)" % ("FP64" if is64 else "FP32")}
    if cat == "form":
        # the bytes it must move: read D^-1 of every subdomain, write packed F and F_rc
        nsd, nD, b = info["n_sub"], info["n_delta"], int(round(info["n_local"] ** 0.5))
        packed = ((nD * (nD + 1) // 2) + 1) // 2 * 2
        out["algorithmic_bytes_per_launch"] = nsd * (b * b * b + packed + nD * 4) * 2 * prec_bytes / per_step
    return out


# ------------------------------------------------------------------ further measured rows
def _events(torch, stream):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def row_3d(args, torch, S, inputs, oracle, dev, stream, peaks):
    """Precision form: 3D, 128^3 Q1 elements, 16^3 subdomains of 8^3, beta = 1e-6, 8 sine modes;
    setup + one solve, mixed (refined to 1e-10) and plain FP64, error against the oracle."""
    N, P, beta = 128, 16, 1e-6
    yb = inputs.random_modes_3d(N, count=8, seed=2)
    bh = oracle.apply_M(3, N, yb)
    b = torch.from_numpy(bh).to(dev)
    n = bh.size
    t0 = time.perf_counter()
    xref = oracle.fd_schur_solve(3, N, beta, bh)
    t_or = time.perf_counter() - t0
    out = {"workload": "3d-q1-128^3-dirichlet-16^3sub-8^3el-8-sine-modes-beta1e-6", "n_dofs": n,
           "oracle_s": t_or}
    # first use of the 3D kernels and of this much device memory (module loading, memory-pool
    # growth) outside the timed setups
    S.Solver(3, N, beta, nsub=P, precision=S.SCHUR_MIXED, tol=OUTER_TOL).close()
    torch.cuda.synchronize()
    # mixed: local operators from three TF32 products (FP32 accuracy); mixed_tf32: one product
    precs = [(S.SCHUR_MIXED, "mixed", 0), (S.SCHUR_MIXED, "mixed_tf32", 1)] + \
            ([] if args.no_fp64 else [(S.SCHUR_FP64, "fp64", 0)])
    for prec, key, split in precs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sol = S.Solver(3, N, beta, nsub=P, precision=prec, tol=OUTER_TOL, tc_split=split)
        t_setup = time.perf_counter() - t0
        e0, e1 = _events(torch, stream)
        e0.record(stream)
        x = sol.schur_solve(b)
        e1.record(stream)
        e1.synchronize()
        ms_solve = e0.elapsed_time(e1)
        st = sol.last_stats
        err = float(np.linalg.norm(x.cpu().numpy() - xref) / np.linalg.norm(xref))
        sol.close()
        out[key] = {"ms_setup": 1e3 * t_setup, "ms_solve": ms_solve,
                    "mdof_s": n / (t_setup + ms_solve / 1e3) / 1e6, "mdof_s_cached": n / (ms_solve / 1e3) / 1e6,
                    "relerr_vs_oracle": err, "gmres_iters": st["iters_total"], "outer_steps": st["outer_steps"],
                    "rel_residual": st["rel_residual"]}
    out["form_roofline"] = tc_form_roofline(S, N, P, beta, peaks)
    return out


def tc_form_counts(N, P):
    """Work of the 3D tensor-core formation on an N^3 cube in P^3 cubic subdomains: right-hand-side
    columns per subdomain (interface slots + 8 corners), column tiles run on the tensor pipe (a last
    tile of at most 16 columns runs on the CUDA cores), accumulator width, K steps of 8 per layer
    product, executed TF32 MMA flops (three products per step, M = 128) and useful complex
    FP32-equivalent flops (8 per complex multiply-add) of the 2L - 2 layer products."""
    s = N // P
    nsd, b, L = P ** 3, (s + 1) ** 2, s + 1
    ncol = 6 * (s - 1) ** 2 + 12 * (s - 1) + 8
    rem = ncol % 128
    ncol_tc = ncol - rem if 0 < rem <= 16 and ncol > 128 else ncol
    ntile, nb, ksteps = (ncol_tc + 127) // 128, (2 * b + 15) // 16 * 16, (2 * b + 7) // 8
    executed = nsd * ntile * (2 * L - 2) * ksteps * 3 * (2 * 128 * nb * 8)
    useful = nsd * ncol * (2 * L - 2) * b * b * 8
    return {"ncol": ncol, "ncol_tc": ncol_tc, "ntile": ntile, "nb": nb, "ksteps": ksteps, "executed": executed,
            "useful": useful}


def tc_form_roofline(S, N, P, beta, peaks):
    """Tensor-pipe roofline of the 3D tensor-core formation (mixed setup, three-product split):
    executed TF32 MMA flops and useful complex FP32-equivalent flops over the event-timed 'form'
    category, against the TF32 tcgen05 peak measured by schur_peak_probe."""
    cnt = tc_form_counts(N, P)
    executed, useful = cnt["executed"], cnt["useful"]
    S.schur_profile_begin(0x3FFFF)
    sol = S.Solver(3, N, beta, nsub=P, precision=S.SCHUR_MIXED, tol=OUTER_TOL)
    prof = S.schur_profile_end()
    sol.close()
    ms = prof.get("form", (0, float("nan")))[1]
    peak = peaks["tf32_tcgen05"]
    ach = executed / (ms * 1e-3) / 1e12
    return {"kernel": "k_form_rr_tc", "bound": "tensor", "precision": "tf32 (3-product split)", "ms": ms,
            "executed_tflop": executed / 1e12, "useful_fp32_tflop": useful / 1e12, "achieved": ach,
            "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "useful_tflops": useful / (ms * 1e-3) / 1e12,
            "peak_source": "measured tcgen05 kind::tf32 128x256x8 (schur_peak_probe)",
            "useful_frac_of_fp32_fma": useful / (ms * 1e-3) / 1e12 / peaks["fp32_fma"],
            "factor_ms": prof.get("factor", (0, float("nan")))[1]}


def row_kkt(args, torch, S, inputs, oracle, dev, stream):
    """Full-space form: 2D 512^2, 32 x 32 subdomains, MINRES with P_mgw on 8 right-hand sides
    (M y_bar_k, 0, 0), y_bar_k = smoothed noise seeds 10..17, to 1e-10; per beta, with the exact
    Schur block (S by the complex factorisation of Sec. 4) and with the Pearson-Wathen S_p of
    Sec. 3.2 (two real FETI-DP solves per application): MINRES iterations, S-block applications
    (one per iteration plus the initial one) and time, the analogue of the paper's Table 7."""
    N, P = 512, 32
    n = (N - 1) ** 2
    yb = inputs.smoothed_noise(2, N, seed=10, nrhs=8)
    ry = oracle.apply_M(2, N, yb)
    rhs = np.zeros((8, 3 * n))
    rhs[:, :n] = ry
    rd = torch.from_numpy(rhs).to(dev)
    out = {"workload": "2d-q1-512x512-32x32sub-kkt-minres-8rhs", "n_dofs_per_block": n, "nrhs": 8}
    # first use of the multi-right-hand-side kernels and workspaces outside the timed runs
    for factor in (S.SCHUR_FACTOR_EXACT, S.SCHUR_FACTOR_PW):
        sol = S.Solver(2, N, 1e-4, nsub=P, precision=S.SCHUR_MIXED, tol=OUTER_TOL, factor=factor)
        sol.schur_kkt_minres(rd, tol=1e-10, max_it=80)
        sol.close()
    torch.cuda.synchronize()
    for beta in (1e-4, 1e-8):
        y, u, l = oracle.fd_kkt_solve(2, N, beta, ry=ry)
        ref = np.concatenate([y, u, l], axis=1)
        row = {}
        for factor, key in ((S.SCHUR_FACTOR_EXACT, "S_c"), (S.SCHUR_FACTOR_PW, "S_p")):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sol = S.Solver(2, N, beta, nsub=P, precision=S.SCHUR_MIXED, tol=OUTER_TOL, factor=factor)
            t_setup = time.perf_counter() - t0
            e0, e1 = _events(torch, stream)
            e0.record(stream)
            x, it = sol.schur_kkt_minres(rd, tol=1e-10, max_it=80)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            xh = x.cpu().numpy()
            err = max(float(np.linalg.norm(xh[c] - ref[c]) / np.linalg.norm(ref[c])) for c in range(8))
            sol.close()
            row[key] = {"ms_setup": 1e3 * t_setup, "ms_minres": ms, "minres_iters": it, "s_block_applies": it + 1,
                        "ms_per_s_block_apply": ms / (it + 1), "max_relerr_vs_oracle": err,
                        "mdof_s": 8 * 3 * n / (t_setup + ms / 1e3) / 1e6}
        out["beta_%g" % beta] = row
    return out


# phi values of the paper's Table 1 (the thermal problem's regularisation sweep) run here
THERMAL_PHIS = (2e-2, 2e-4, 2e-6, 2e-8, 2e-10, 2e-12)
# the paper's Table 1, FETI-DPH iterations without augmentation on K + M/(i sqrt(phi)) ("+"), for context
TABLE1_PLUS = {2e-2: 32, 2e-4: 38, 2e-6: 34, 2e-8: 38, 2e-10: 44, 2e-12: 62}


def row_thermal(args, torch, S, inputs, oracle, dev, stream):
    """The paper's thermal problem (Sec. 6.1): target (2x-1)^2 (2y-1)^2 on [0,1/2]^2, Dirichlet data
    y_c = ybar, h = 2^-11 (2048^2 Q1 elements, 4,190,209 interior dofs), 128 x 128 subdomains of 16^2,
    phi swept over Table 1's range.  Per phi: the FP64 form with one FETI-DP solve to 1e-10 (the
    paper's threshold; iterations comparable with Table 1), the mixed form (setup + range-space
    solve, timed), the relative constraint violation (Eq. relativeconstraintviolation), the relative
    L2 (M-norm) distance of y to ybar and the L2 norm of u (the quantities of the paper's Fig. 2),
    and at phi = 2e-8 the error of (y, u) against the oracle (sine basis)."""
    N, P = 2048, 128
    n = (N - 1) ** 2
    yf = inputs.thermal_target(N)
    yfd = torch.from_numpy(yf).to(dev)
    ybi = oracle.interior_of(2, N, yf)
    out = {"workload": "2d-q1-2048^2-dirichlet-thermal-target-128x128sub-16x16el", "n_dofs": n, "per_phi": {}}
    S.Solver(2, N, THERMAL_PHIS[0], nsub=P, precision=S.SCHUR_MIXED, tol=OUTER_TOL).close()  # warm-up
    for phi in THERMAL_PHIS:
        r = {"table1_iters_plus_no_aug": TABLE1_PLUS.get(phi)}
        # one FETI-DP solve (the outer stop at 1e-3 ends the refinement after its first step)
        sol = S.Solver(2, N, phi, nsub=P, precision=S.SCHUR_FP64, tol=1e-3, inner_tol=1e-10, max_refine=1)
        sol.schur_control_solve(yfd, want_violation=False)
        r["fp64_gmres_iters"] = sol.last_stats["iters_first"]
        sol.close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sol = S.Solver(2, N, phi, nsub=P, precision=S.SCHUR_MIXED, tol=OUTER_TOL)
        y, u, lam, viol = sol.schur_control_solve(yfd)
        torch.cuda.synchronize()
        r["mixed_ms_setup_plus_solve"] = 1e3 * (time.perf_counter() - t0)
        r["mixed_gmres_iters"] = sol.last_stats["iters_total"]
        r["mixed_outer_steps"] = sol.last_stats["outer_steps"]
        r["constraint_violation"] = float(viol[0])
        sol.close()
        yh, uh = y.cpu().numpy(), u.cpu().numpy()
        d = yh - ybi
        r["rel_l2_y_minus_ybar"] = float(np.sqrt(d @ oracle.apply_M(2, N, d) / (ybi @ oracle.apply_M(2, N, ybi))))
        r["l2_norm_u"] = float(np.sqrt(uh @ oracle.apply_M(2, N, uh)))
        if phi == 2e-8:
            oracle.set_threads(os.cpu_count() or 1)
            yr, ur, _ = oracle.control_solve(2, N, phi, yf, fd=True)
            r["relerr_y_vs_oracle"] = float(np.linalg.norm(yh - yr) / np.linalg.norm(yr))
            r["relerr_u_vs_oracle"] = float(np.linalg.norm(uh - ur) / np.linalg.norm(ur))
        out["per_phi"]["%g" % phi] = r
    return out


# the paper's Table 1, FETI-DPH iterations with the rigid-body-mode augmentation on
# K + M/(i sqrt(phi)) ("RAUG+"), for context
TABLE1_RAUG_PLUS = {2e-2: 13, 2e-4: 13, 2e-6: 13, 2e-8: 13, 2e-10: 17, 2e-12: 26}


def row_augmented(args, torch, S, inputs, oracle, dev, stream):
    """The augmented coarse problem (Sec. 5, RAUG: one face-average constraint per pair of
    face-adjacent subdomains beside the corners) at the paper's subdomain size ratio H/h = 64:
    2D 1024^2 Q1 elements in 16 x 16 subdomains of 64^2 (the h = 1/1024 row of the paper's Table 2),
    phi over Table 1's range.  Per phi: GMRES iterations of one FP64 FETI-DP solve to 1e-10 without
    and with the augmentation, the mixed form's setup + solve time both ways, and at phi = 2e-8 the
    augmented mixed result against the oracle."""
    N, P = 1024, 16
    n = (N - 1) ** 2
    b = oracle.apply_M(2, N, inputs.smoothed_noise(2, N, seed=1))
    bd = torch.from_numpy(b).to(dev)
    out = {"workload": "2d-q1-1024^2-dirichlet-16x16sub-64x64el-smoothed-noise", "n_dofs": n,
           "coarse_unknowns": {"corners": (P - 1) ** 2, "augmented": (P - 1) ** 2 + 2 * (P - 1) * P}, "per_phi": {}}
    for aug in (0, 1):  # warm-up of both setups
        S.Solver(2, N, THERMAL_PHIS[0], nsub=P, precision=S.SCHUR_MIXED, tol=OUTER_TOL, augment=aug).close()
    for phi in THERMAL_PHIS:
        r = {"table1_iters_plus_no_aug": TABLE1_PLUS.get(phi), "table1_iters_plus_raug": TABLE1_RAUG_PLUS.get(phi)}
        for aug, key in ((0, "corners"), (1, "augmented")):
            sol = S.Solver(2, N, phi, nsub=P, precision=S.SCHUR_FP64, tol=1e-3, inner_tol=1e-10, max_refine=1,
                           augment=aug)
            sol.schur_solve(bd)
            r["fp64_gmres_iters_" + key] = sol.last_stats["iters_first"]
            sol.close()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sol = S.Solver(2, N, phi, nsub=P, precision=S.SCHUR_MIXED, tol=OUTER_TOL, augment=aug)
            t1 = time.perf_counter()
            x = sol.schur_solve(bd)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            r["mixed_ms_setup_" + key] = 1e3 * (t1 - t0)
            r["mixed_ms_solve_" + key] = 1e3 * (t2 - t1)
            r["mixed_gmres_iters_" + key] = sol.last_stats["iters_total"]
            sol.close()
            if phi == 2e-8 and aug:
                oracle.set_threads(os.cpu_count() or 1)
                xr = oracle.fd_schur_solve(2, N, phi, b)
                r["relerr_augmented_mixed_vs_oracle"] = float(np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr))
        out["per_phi"]["%g" % phi] = r
    return out


def serve_stream(args, S, inputs, oracle):
    """Serving form: Poisson arrivals of mixed 2D/3D sizes, beta from 6 cached values, 1-16 seeded
    right-hand sides per request.  Capacity is measured closed-loop (the first 400 requests all
    submitted at t = 0); the open-loop stream of all requests then arrives at 0.8 x that rate,
    served by the mixed form.  The plain FP64 form serves the first 60 requests of the same stream
    (same arrival times) and, closed-loop, gives its own capacity.  Latency = arrival -> result on
    the host.  Batching is reported from the server's counters: right-hand sides per multi-RHS solve,
    requests that shared a solve, most batches on the device at once, factor-cache misses."""
    nreq = args.serve_requests
    sizes = [(2, 64), (2, 128), (2, 256), (2, 512), (2, 1024), (3, 32), (3, 64), (3, 96)]
    betas = [10.0 ** (-8 + 1.2 * k) for k in range(6)]
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(nreq):
        r = np.random.default_rng(i)
        dim, N = sizes[r.integers(len(sizes))]
        reqs.append((dim, N, betas[r.integers(6)], int(r.integers(1, 17)), i))
    pool = {}
    for dim, N in sizes:  # 16 seeded targets per size, b = M y_bar
        yb = inputs.smoothed_noise(dim, N, seed=100 + N, nrhs=16) if dim == 2 else \
            inputs.random_modes_3d(N, count=8, seed=100 + N, nrhs=16)
        pool[(dim, N)] = np.ascontiguousarray(oracle.apply_M(dim, N, yb))

    def rhs_of(q):
        dim, N, beta, R, i = q
        return np.ascontiguousarray(np.roll(pool[(dim, N)], i, axis=0)[:R])

    def run(prec, arrivals, count):
        # Krylov space of at most 100 vectors per right-hand side for the FP64 form (it needs < 80
        # here), 60 for the mixed form (its inner solves stop at a loose tolerance, < 20 iterations);
        # a budget that holds the contexts of all 48 (mesh, beta) keys of the stream
        srv = S.Server(budget_bytes=160 << 30, workers=4, precision=prec, tol=1e-10,
                       max_iter=60 if prec == S.SCHUR_MIXED else 100)
        try:
            lat, pend, nsolve, rejected = [], {}, 0, 0
            t0 = time.perf_counter()
            k = 0
            while k < count or pend:
                now = time.perf_counter() - t0
                while k < count and arrivals[k] <= now:
                    q = reqs[k]
                    try:
                        pend[srv.submit(q[0], q[1], q[2], rhs_of(q))] = (arrivals[k], q)
                    except S.SchurError as e:  # larger than the whole memory budget
                        if e.code != S.SCHUR_EBUSY:
                            raise
                        rejected += 1
                    k += 1
                moved = False
                for t in list(pend):
                    ok, x, st = srv.poll(t)
                    if ok:
                        arr, q = pend.pop(t)
                        lat.append(time.perf_counter() - t0 - arr)
                        nsolve += q[3]
                        moved = True
                if not moved:
                    time.sleep(0.0002)
            span = time.perf_counter() - t0
            si = srv.info()
        finally:
            srv.close()
        lat = np.array(lat) * 1e3
        nb = max(1, si["batches"])
        return {"requests": count, "rejected": rejected, "rhs_solved": nsolve, "makespan_s": span,
                "solves_s": nsolve / span, "requests_s": count / span,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "batching": {"solve_calls": si["batches"], "rhs_per_solve_call": si["batch_columns"] / nb,
                             "requests_per_solve_call": count / nb,
                             "shared_request_fraction": si["shared_requests"] / max(1, count),
                             "max_concurrent_batches": si["max_concurrent"], "factor_setups": si["setups"]}}

    ncap = min(nreq, 400)
    closed = run(S.SCHUR_MIXED, np.zeros(ncap), ncap)
    rate = 0.8 * ncap / closed["makespan_s"]
    arrivals = np.cumsum(rng.exponential(1.0 / rate, nreq))
    out = {"workload": "serve-mixed-2d-64..1024^2-3d-32..96^3-6-betas-1..16-rhs-poisson", "requests": nreq,
           "capacity_requests_s": ncap / closed["makespan_s"], "capacity_from_requests": ncap,
           "capacity_closed_loop": closed, "arrival_rate_requests_s": rate,
           "mixed": run(S.SCHUR_MIXED, arrivals, nreq)}
    if not args.no_fp64:
        nf = min(nreq, 60)
        out["fp64"] = {"sample": "first %d requests of the same stream" % nf,
                       "closed_loop": run(S.SCHUR_FP64, np.zeros(nf), nf),
                       "same_arrivals": run(S.SCHUR_FP64, arrivals, nf)}
    # spot check of served results against the oracle: the first requests of each kind (2D up to
    # 256^2, 2D 1024^2, 3D up to 64^3; first two columns of each)
    oracle.set_threads(os.cpu_count() or 1)
    srv = S.Server(budget_bytes=64 << 30, workers=2, precision=S.SCHUR_MIXED, tol=1e-10, max_iter=60)
    try:
        errs = []
        picks = [q for q in reqs if q[0] == 2 and q[1] <= 256][:3] + [q for q in reqs if q[1] == 1024][:1] + \
                [q for q in reqs if q[0] == 3 and q[1] <= 64][:2]
        for q in picks:
            b = rhs_of(q)[:2]
            x, _ = srv.wait(srv.submit(q[0], q[1], q[2], b))
            xr = oracle.fd_schur_solve(q[0], q[1], q[2], b)
            errs.append(float(np.linalg.norm(x - xr) / np.linalg.norm(xr)))
        out["spot_check"] = {"requests": ["%dD %d, beta %.1e" % (q[0], q[1], q[2]) for q in picks],
                             "max_relerr_vs_oracle": max(errs) if errs else None}
    finally:
        srv.close()
    return out


def ncu_case(which):
    """One mixed-precision setup + solve: the profiled unit of work (2d: the headline workload;
    3d: a 64^3 cube with the 8^3 subdomains of the 128^3 workload)."""
    import torch
    from paper_1312_5653_gb300 import inputs
    from paper_1312_5653_gb300 import schur as S
    if which == "3d":
        yb = torch.from_numpy(inputs.random_modes_3d(64, count=8, seed=2)).cuda()
        sol = S.Solver(3, 64, 1e-6, nsub=8, precision=S.SCHUR_MIXED, tol=OUTER_TOL)
    else:
        yb = torch.from_numpy(inputs.smoothed_noise(2, N_EL, seed=1)).cuda()
        sol = S.Solver(2, N_EL, 1e-4, nsub=N_SUB, precision=S.SCHUR_MIXED, tol=OUTER_TOL)
    b = sol.schur_apply_mass(yb)
    sol.schur_solve(b)
    torch.cuda.synchronize()
    print(json.dumps(sol.last_stats))
    sol.close()


def main():
    args = parse()
    rank, local_rank, world = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.ncu_case:
        return ncu_case(args.ncu_case)
    if args.peaks:
        from paper_1312_5653_gb300 import schur as S
        pf = {}
        try:
            pf = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        print(json.dumps(measure_peaks(S, pf)), flush=True)
        return
    import torch
    from paper_1312_5653_gb300 import inputs
    from paper_1312_5653_gb300 import schur as S

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)
    lib = S.load()
    n = S.schur_ndof(2, N_EL)
    # each rank solves its own seeded right-hand side (independent problems: weak scaling)
    yb = inputs.smoothed_noise(2, N_EL, seed=rank_seed(rank))
    ybd = torch.from_numpy(yb).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def make(beta, prec):
        return S.Solver(2, N_EL, beta, nsub=N_SUB, precision=prec, tol=OUTER_TOL)

    # b = M y_bar on the device (library mass apply)
    s0 = make(BETAS[0], S.SCHUR_MIXED)
    b = s0.schur_apply_mass(ybd)
    s0.close()
    x = torch.empty_like(b)
    torch.cuda.synchronize()

    def step(i, prec):
        sol = make(BETAS[i % 4], prec)
        sol.schur_solve(b, x)
        st = sol.last_stats
        nl = lib.schur_launch_count(sol.ctx)
        sol.close()
        return st, nl

    def timed(prec, steps, warmup, profile_mask=0):
        for i in range(warmup):
            step(i, prec)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if profile_mask:
            lib.schur_profile_begin(profile_mask)
        times, stats, launches = [], [], 0
        for i in range(steps):
            flush_l2(flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, nl = step(i, prec)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            stats.append(st)
            launches += nl
        torch.cuda.synchronize()
        prof = S.schur_profile_end() if profile_mask else None
        if world > 1:
            torch.distributed.barrier()
        total = max_over_ranks(torch, float(np.sum(times)), dev, world)
        return total, times, stats, launches, prof

    import ctypes

    # untimed profiling pass, one step per beta, every category: the per-category breakdown and the
    # single kernel with the largest share (only that kernel's events are recorded while timing)
    _, _, _, _, prof_all = timed(S.SCHUR_MIXED, 4, 0, profile_mask=0x3FFFF)
    single = [c for c in (prof_all or {}) if c in KERNEL_OF]
    dom = max(single, key=lambda c: prof_all[c][1]) if single else None
    dom_mask = (1 << CATEGORIES.index(dom)) if dom else 0

    # headline: mixed precision, timed region
    with Clocks(local_rank) as clk:
        total, times, stats, launches, prof = timed(S.SCHUR_MIXED, args.steps, args.warmup, profile_mask=dom_mask)
    ms_step = total / args.steps
    value = job_rate(world, n, args.steps, total)

    # accuracy of the timed path vs the oracle on one step, and the oracle timed on the host cores
    # (rank 0): all cores on one right-hand side per beta, one core on one right-hand side
    relerr = relerrs = None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        bh = b.cpu().numpy()
        ncores = os.cpu_count() or 1
        oracle.set_threads(ncores)
        t_all, relerrs = [], []
        for beta in BETAS:
            xref, t = cpu_oracle_solve(bh, beta)
            t_all.append(t)
            sol = make(beta, S.SCHUR_MIXED)
            xg = sol.schur_solve(b).cpu().numpy()
            sol.close()
            relerrs.append(float(np.linalg.norm(xg - xref) / np.linalg.norm(xref)))
        relerr = max(relerrs)
        oracle.set_threads(1)
        _, t_one = cpu_oracle_solve(bh, BETAS[0])
        cpu = {"value": n * len(t_all) / float(np.sum(t_all)) / 1e6, "unit": "MDoF/s", "cores": ncores,
               "kind": "oracle", "cpu_model": cpu_model(),
               "sample": "one full-size right-hand side (1,046,529 dofs) per beta (4 solves), fast-diagonalisation "
                         "oracle with its sine-transform lines on %d OpenMP threads, %.1f s in all" %
                         (ncores, float(np.sum(t_all))),
               "single_thread": {"value": n / t_one / 1e6, "unit": "MDoF/s", "cores": 1,
                                 "sample": "one full-size right-hand side, one thread, %.1f s" % t_one}}

    # cached-factor solve rate (factorisation reused across right-hand sides, as the server does)
    cached = {}
    for prec, key in ((S.SCHUR_MIXED, "mixed"), (S.SCHUR_FP64, "fp64")):
        if prec == S.SCHUR_FP64 and args.no_fp64:
            continue
        ts, its = [], []
        for beta in BETAS:
            sol = make(beta, prec)
            sol.schur_solve(b, x)
            flush_l2(flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sol.schur_solve(b, x)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            its.append(sol.last_stats)
            sol.close()
        cached[key] = {"ms_per_solve": float(np.mean(ts)), "mdof_s": n / (np.mean(ts) / 1e3) / 1e6,
                       "solves_s": 1e3 / float(np.mean(ts)),
                       "per_beta": [{"beta": bb, "ms": t, "outer_steps": s["outer_steps"],
                                     "gmres_iters": s["iters_total"], "ms_setup": s["ms_setup"]}
                                    for bb, t, s in zip(BETAS, ts, its)]}

    # plain FP64 form, same steps (setup + solve), one per beta
    fp64 = None
    if not args.no_fp64:
        t64, tt64, st64, _, _ = timed(S.SCHUR_FP64, 4, 1)
        fp64 = {"value": n * 4 / (t64 / 1e3) / 1e6, "unit": "MDoF/s", "ms_per_step": t64 / 4,
                "gmres_iters": [s["iters_total"] for s in st64], "outer_steps": [s["outer_steps"] for s in st64]}

    # end to end through the host-buffer entry point (pinned host b, host x), setup included
    bh_pin = torch.empty(n, dtype=torch.float64, pin_memory=True)
    bh_pin.copy_(b.cpu())
    xh_pin = torch.empty(n, dtype=torch.float64, pin_memory=True)
    e2e_t = []
    for i in range(max(2, args.steps // 2)):
        flush_l2(flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sol = make(BETAS[i % 4], S.SCHUR_MIXED)
        st = S.schur_stats()
        rc = lib.schur_solve_host(sol.ctx, ctypes.c_void_p(bh_pin.data_ptr()), ctypes.c_void_p(xh_pin.data_ptr()), 1,
                                  n, S._stream_ptr(stream), ctypes.byref(st))
        assert rc == 0, S.last_error()
        sol.close()
        e2e_t.append(time.perf_counter() - t0)
    e2e = {"value": world * n * len(e2e_t) / float(np.sum(e2e_t)) / 1e6, "unit": "MDoF/s",
           "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n}

    # rooflines from the event-timed categories of the timed region, against measured peaks; the
    # reported one is the single kernel with the largest share of the step
    peaks_file = {}
    try:
        peaks_file = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peaks = measure_peaks(S, peaks_file)
    sol = make(BETAS[0], S.SCHUR_MIXED)
    info = sol.info()
    sol.close()
    by_cat = {}
    for cat, (nl_, tot_ms) in (prof_all or {}).items():
        r = category_roofline(cat, info, nl_, tot_ms, 4, peaks)
        if r:
            by_cat[cat] = r
    roof = None
    if dom and prof and dom in prof:
        nl_, tot_ms = prof[dom]
        roof = category_roofline(dom, info, nl_, tot_ms, args.steps, peaks)
        roof["kernel"] = KERNEL_OF[dom]
        roof["category"] = dom
        roof["share_of_step"] = tot_ms / total
        roof["timed"] = "CUDA events on the solve stream around each launch of this kernel, inside the timed region"
        roof["traffic"] = recorded_traffic(KERNEL_OF[dom])
        if roof["traffic"] is not None:
            roof["traffic_over_algorithmic"] = roof["traffic"] / roof["algorithmic_bytes_per_launch"]

    extra = {}
    if rank == 0 and not args.no_extra:
        import oracle
        oracle.build()
        extra["precision_form_3d"] = row_3d(args, torch, S, inputs, oracle, dev, stream, peaks)
        extra["full_space_kkt"] = row_kkt(args, torch, S, inputs, oracle, dev, stream)
        extra["thermal_range_space"] = row_thermal(args, torch, S, inputs, oracle, dev, stream)
        extra["augmented_coarse"] = row_augmented(args, torch, S, inputs, oracle, dev, stream)
        extra["serving"] = serve_stream(args, S, inputs, oracle)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_dofs": n, "subdomains": N_SUB * N_SUB, "beta": list(BETAS),
                       "nrhs_per_step": 1, "step": "schur_setup + schur_solve + schur_destroy",
                       "precision": "complex FP32 FETI-DP, FP64 refinement to ||b-Az||/||b||<=1e-10",
                       "l2": "flushed (256 MB write) between timed steps"},
            "solves_per_s": world * args.steps / (total / 1e3),
            "relerr_vs_oracle": relerr,
            "relerr_vs_oracle_per_beta": relerrs,
            "gmres_iters": [s["iters_total"] for s in stats], "outer_steps": [s["outer_steps"] for s in stats],
            "ms_setup": [s["ms_setup"] for s in stats],
            "cached_factor_solve": cached, "fp64": fp64,
            "roofline": roof, "roofline_by_category": by_cat, "peaks": peaks,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "profile_ms_per_step_by_category": {k: v[1] / 4 for k, v in (prof_all or {}).items()},
            "clocks": clk.summary(),
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
