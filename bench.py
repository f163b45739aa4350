#!/usr/bin/env python
"""Benchmark of the restricted additive Vanka (RAV) multigrid V-cycle on GB300.

Workload (default): 2-D Stokes, Q2-Q1 on a uniform 512x512 grid of the unit
square (2,101,250 velocity + 263,169 pressure DoFs), 7 levels (512 -> 8),
manufactured solution u = curl(sin^2(pi x) sin^2(pi y)), p = cos(pi x) cos(pi y),
viscosity 1, plain FP64 RAV smoother with damping 0.5, V(2,2).

A step is one V(2,2) cycle on the finest level (smoothing, residuals,
transfers, coarse solve on every level).  value = DoFs x steps / seconds.

Reported with it:
  roofline      the dominant kernel (the fine-level RAV subdomain apply),
                timed live with CUDA events on its launching stream over the
                timed region, against the FP64 arithmetic peak (it is bound by
                fp64 FMA throughput on GB300; patch_work() holds the counts);
  e2e           the same metric with host buffers, host<->device copies inside;
  cpu_baseline  the FP64 oracle on a bounded sample, on one host core and on
                every host core (its subdomain loops in parallel);
  time_to_tol   wall time of a full solve to a 1e-8 residual reduction;
  forms_to_tol  (default workload) time to 1e-8 of the reduced-precision and
                batched forms against the plain FP64 GPU form on the same
                problems: 512^2 stationary and 32^3 FGMRES(30) with FP64 /
                FP32 / BF16 factored inverses, and the 256-cavity x 8-RHS batch
                with FP32 and FP64 rows on the batched path, each group with
                its own clock record (forms_vs_fp64()).

--impl reference times the oracle itself as the reference arm.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP64 peak derived from unit counts and clocks: 152 SMs x 2 FP64 FMA/clk/SM x
# 2 flop x 2.07 GHz (the nominal 1.25 TFLOP/s of GB300).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
L2_BYTES = 129 * 2 ** 20

WORKLOADS = {
    "2d512": dict(dim=2, N=512, nlev=7, bc=1, forcing=1, kind=0, prec=0, omega=0.5, nu=2,
                  desc="2D Stokes Q2-Q1 512x512 unit square, 7 levels, manufactured psi solution, "
                       "viscosity 1, RAV V(2,2) omega 0.5, FP64"),
    "2d512-rows": dict(dim=2, N=512, nlev=7, bc=1, forcing=1, kind=0, prec=4, omega=0.5, nu=2,
                       desc="as 2d512 with the owned rows of the patch inverses stored densely in FP64"),
    "2d512-f32": dict(dim=2, N=512, nlev=7, bc=1, forcing=1, kind=0, prec=1, omega=0.5, nu=2,
                      desc="as 2d512 with FP32-stored patch inverses (FP32 accumulation)"),
    "2d512-f32fact": dict(dim=2, N=512, nlev=7, bc=1, forcing=1, kind=0, prec=5, omega=0.5, nu=2,
                          desc="as 2d512 with the factored inverses stored in FP32 (FP32 accumulation)"),
    "2d512-bf16fact": dict(dim=2, N=512, nlev=7, bc=1, forcing=1, kind=0, prec=6, omega=0.5, nu=2,
                           desc="as 2d512 with the factored inverses stored in BF16 (FP32 accumulation)"),
    "3d32": dict(dim=3, N=32, nlev=4, bc=1, forcing=2, kind=0, prec=0, omega=0.5, nu=2, blobs=(20, 3.0),
                 desc="3D Stokes Q2-Q1 32^3 unit cube, 4 levels, 20 seeded viscosity blobs (contrast <= 1e3), "
                      "sinker forcing, no-slip, RAV V(2,2) omega 0.5, FP64 factored inverses"),
    "3d32-bf16": dict(dim=3, N=32, nlev=4, bc=1, forcing=2, kind=0, prec=6, omega=0.5, nu=2, blobs=(20, 3.0),
                      desc="as 3d32 with the factored inverses stored in BF16 (FP32 accumulation)"),
    "2d1024-q1": dict(dim=2, N=1024, nlev=8, bc=0, forcing=0, kind=0, prec=0, omega=0.66, nu=2, elem=1,
                      beta=0.02, desc="2D Stokes stabilised Q1-Q1 (beta 0.02) 1024x1024 lid-driven cavity, "
                                      "8 levels, viscosity 1, RAV V(2,2) omega 0.66, FP64 factored inverses"),
    "2d1024-q1-f32": dict(dim=2, N=1024, nlev=8, bc=0, forcing=0, kind=0, prec=5, omega=0.66, nu=2, elem=1,
                          beta=0.02, desc="as 2d1024-q1 with the factored inverses stored in FP32 "
                                          "(FP32 accumulation)"),
    "3d64-q1": dict(dim=3, N=64, nlev=5, bc=1, forcing=2, kind=0, prec=0, omega=0.66, nu=2, blobs=(20, 2.0),
                    elem=1, beta=0.02,
                    desc="3D Stokes stabilised Q1-Q1 (beta 0.02) 64^3 unit cube, 5 levels, 20 seeded viscosity "
                         "blobs (contrast <= 1e2), sinker forcing, no-slip, RAV V(2,2) omega 0.66, FP64 "
                         "factored inverses"),
}
STORAGE = {0: "f64 factored", 1: "f32 rows", 2: "bf16 rows", 3: "fp8 rows", 4: "f64 rows", 5: "f32 factored",
           6: "bf16 factored"}


def make_blobs(W):
    if "blobs" not in W:
        return None
    from paper_2103_10127_gb300 import inputs
    k, s_max = W["blobs"]
    return inputs.viscosity_blobs(inputs.BASE_SEED, k=k, s_max=s_max)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-single", action="store_true",
                    help="2d-batch: skip timing the single-problem FP64 form on the same problems")
    ap.add_argument("--workload", default="2d512",
                    choices=sorted(WORKLOADS) + ["2d-batch", "2d-batch-q1", "3d-precision", "3d-precision-q1",
                                                 "3d-learned", "3d-learned-q1", "2d-steps", "2d-steps-q1"])
    ap.add_argument("--nprob", type=int, default=256, help="problems of the 2d-batch workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tol", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="default workload: skip the reduced-precision / batched vs FP64 time-to-tolerance runs")
    ap.add_argument("--fused", action="store_true",
                    help="RAV workloads with factored storage (Q1-Q1: fp64): one fused residual + "
                         "subdomain-apply kernel per smoothing step")
    ap.add_argument("--apply-staged", type=int, default=None,
                    help="reduced factored storage: force the staged apply with this many threads per subdomain "
                         "on the finest level (0: the grouped kernel; default: the set-up tuner's choice)")
    ap.add_argument("--residual-blocked", type=int, default=None, choices=[0, 1],
                    help="Q2-Q1: force the node-blocked (1) or the row-wise (0) residual on every level "
                         "(default: the set-up tuner's choice per level)")
    ap.add_argument("--N", type=int, default=None, help="override the grid size (profiling runs)")
    ap.add_argument("--levels", type=int, default=None)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, dist, device):
    """The slowest rank's timed region (ms): every rank ran its own replica."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(ws, dofs, steps, ms):
    """Whole-job DoFs/s: ws replicas of `dofs` DoFs, `steps` cycles each, in ms."""
    return ws * dofs * steps / (ms / 1e3)


# ---------------------------------------------------------------------------
def patch_work(dim, N, prec, n, q=2):
    """Algorithmic (flops, bytes) of one fine-level subdomain apply, counting
    only the DoFs inside each subdomain (compact sizes, Sec. 4.3): n_i DoFs,
    ñ_i owned rows, nodes_i velocity nodes, own_i owned velocity nodes
    (q = 2: Q2-Q1 boxes of 5^d nodes owning up to 2^d; q = 1: Q1-Q1 boxes of
    3^d vertices owning the centre).
      dense rows:  ñ_i n_i FMAs and stored entries per subdomain;
      factored:    d own_i nodes_i + d nodes_i + d own_i + 1 FMAs and
                   own_i nodes_i + d nodes_i + 1 stored values (fp64, fp32 or bf16).
    Vectors: r read once (8 n bytes), owned x read and written (16 ñ_i)."""
    import numpy as np
    per_n, per_o = [], []
    for v in range(N + 1):
        if q == 1:
            per_n.append(sum(1 for a in range(3) if 1 <= v - 1 + a <= N - 1))
            per_o.append(1 if 1 <= v <= N - 1 else 0)
        else:
            per_n.append(sum(1 for a in range(5) if 1 <= 2 * v - 2 + a <= 2 * N - 1))
            per_o.append(sum(1 for a in (2, 3) if 1 <= 2 * v + a - 2 <= 2 * N - 1))
    pn, po = np.array(per_n, float), np.array(per_o, float)
    if dim == 2:
        nodes, own = np.outer(pn, pn), np.outer(po, po)
    else:
        nodes, own = np.einsum("i,j,k->ijk", pn, pn, pn), np.einsum("i,j,k->ijk", po, po, po)
    ni, nown = dim * nodes + 1, dim * own + 1
    vec = 8.0 * n + 16.0 * nown.sum()
    if prec in (0, 5, 6):
        fma = (dim * own * nodes + dim * nodes + dim * own + 1).sum()
        stored = {0: 8.0, 5: 4.0, 6: 2.0}[prec] * (own * nodes + dim * nodes + 1).sum()
    else:
        fma = (ni * nown).sum()
        stored = {4: 8, 1: 4, 2: 2, 3: 1}[prec] * fma
    return 2.0 * float(fma), float(stored + vec), float(stored)


def clocks_start():
    f = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    try:
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100"],
                             stdout=f, stderr=subprocess.DEVNULL)
    except OSError:
        p = None
    return p, f.name


def clocks_stop(handle, gpu_index):
    p, path = handle
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9 or not f[0].isdigit() or int(f[0]) != gpu_index:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    os.unlink(path)
    sm.sort()
    return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "samples": len(sm), "reasons": sorted(reasons)}


def measured_traffic(kernel_key, source="smoother.cu"):
    """dram bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source file (else None)."""
    src = os.path.join(ROOT, "paper_2103_10127_gb300", "csrc", source)
    digest = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
    path = os.path.join(ROOT, "profiles", f"{kernel_key}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha1") != digest:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def workload_config(W, n, nnz, stored, ws, fused=False):
    """The `config` object of a default-style line, the same for both arms."""
    return {"workload": W["desc"], "dofs": n, "levels": W["nlev"], "nu": [W["nu"], W["nu"]],
            "smoother": "RAV" + (", fused residual + apply per step" if fused else ""),
            "inverse_storage": STORAGE[W["prec"]],
            "l2": "inputs larger than L2: each fine-level pass streams the operator "
                  f"({nnz * 12 / 1e9:.2f} GB) and the stored patch inverses "
                  f"({stored / 1e9:.2f} GB) > 129 MB L2",
            "parallelism": "replicas" if ws > 1 else "single GPU"}


# ---------------------------------------------------------------------------
def oracle_for(W):
    """The oracle on the workload, set up (untimed) with every host core."""
    import oracle as O
    O.set_threads(os.cpu_count() or 1)
    orc = O.Oracle(W["dim"], W["N"], W["nlev"], bc=W["bc"], blobs=make_blobs(W), element=W.get("elem", 0),
                   beta=W.get("beta", 0.0))
    orc.setup_smoother(O.RAV, W["omega"], W["prec"] if W["prec"] in (1, 2, 3, 5, 6) else 0)
    return O, orc


def cpu_baseline(W, cycles=1):
    """The oracle, as it stands, on the same workload: untimed set-up, then
    `cycles` timed V-cycles on one host core (the paper's setting) and the
    same on every host core (its independent subdomain loops in parallel,
    everything else serial).  Returns (DoF/s one core, s, DoF/s all cores, s,
    cores, n)."""
    O, orc = oracle_for(W)
    b = orc.rhs(W["forcing"])
    x0 = orc.initial_guess()
    n = orc.sizes(W["nlev"] - 1)["n"]
    res = []
    for threads in (1, os.cpu_count() or 1):
        used = O.set_threads(threads)
        x = x0
        t0 = time.perf_counter()
        for _ in range(cycles):
            x = orc.vcycle(x, b, W["nu"], W["nu"])
        dt = time.perf_counter() - t0
        res.append((n * cycles / dt, dt, used))
    O.set_threads(1)
    del orc
    return res[0][0], res[0][1], res[1][0], res[1][1], res[1][2], n


def run_reference(args, W):
    """The reference arm: the oracle itself on the same workload, one host core
    for the timed cycles (the paper's setting), set-up untimed."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    O, orc = oracle_for(W)
    O.set_threads(1)
    b = orc.rhs(W["forcing"])
    x = orc.initial_guess()
    sz = orc.sizes(W["nlev"] - 1)
    n = sz["n"]
    for _ in range(args.warmup):
        x = orc.vcycle(x, b, W["nu"], W["nu"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x = orc.vcycle(x, b, W["nu"], W["nu"])
    dt = time.perf_counter() - t0
    v = n * args.steps / dt
    _, _, stored = patch_work(W["dim"], W["N"], W["prec"], n, q=1 if W.get("elem", 0) == 1 else 2)
    out = {"impl": "reference", "metric": "V-cycle DoFs/s", "value": v, "unit": "DoF/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(W, n, sz["nnz"], stored, args.gpus),
           "cpu_baseline": {"value": v, "unit": "DoF/s", "cores": 1, "kind": "oracle",
                            "sample": f"{args.steps} V(2,2) cycles of the full workload after untimed set-up"},
           "e2e": {"value": v, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, W):
    import numpy as np
    import torch
    import paper_2103_10127_gb300 as R
    from paper_2103_10127_gb300 import _capi

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib = _capi.load()
    stream = torch.cuda.current_stream()

    mg = R.Multigrid(W["dim"], W["N"], W["nlev"], bc=W["bc"], blobs=make_blobs(W), element=W.get("elem", 0),
                     beta=W.get("beta", 0.0))
    sm = R.Smoother(mg, W["kind"], W["prec"], W["omega"])
    if args.fused:
        sm.fused(True)
    fine = W["nlev"] - 1
    if args.apply_staged is not None:
        sm.apply_staged(fine, args.apply_staged)
    if args.residual_blocked is not None:
        for lev in range(W["nlev"]):
            mg.residual_blocked(lev, args.residual_blocked)
    n = mg.n()
    b = mg.rhs(W["forcing"])
    x0 = mg.initial_guess()
    x = x0.clone()
    nu = W["nu"]

    def step():
        mg.vcycle(sm, x, b, nu, nu)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region (device): V-cycles replayed as captured CUDA graphs ----
    cnt = ctypes_i64()
    tot = ctypes_f64()
    launches0 = lib.rav_kernel_launches()
    clk = clocks_start()
    time.sleep(0.3)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps (ncu --nvtx-include timed/)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    ms = e0.elapsed_time(e1)
    clocks = clocks_stop(clk, local)
    launches = lib.rav_kernel_launches() - launches0

    # ---- the same steps again, kernel by kernel, with CUDA events on the launching
    # stream around every fine-level subdomain apply (the roofline's kernel) ----
    lib.rav_profile_enable(mg.h, 1, fine)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    ms_nograph = p0.elapsed_time(p1)
    lib.rav_profile_read(mg.h, fine, 0, cnt, tot)
    apply_ms = tot.value / max(cnt.value, 1)
    apply_launches = cnt.value

    # ---- per-level, per-kernel-class breakdown (separate untimed pass, events on every kernel) ----
    kb = max(5, args.steps // 10)
    lib.rav_profile_enable(mg.h, 31, -1)
    for _ in range(kb):
        step()
    torch.cuda.synchronize()
    breakdown = {}
    names = ["apply", "residual", "restrict", "prolong", "coarse"]
    for lev in range(W["nlev"]):
        row = {}
        for k, nm in enumerate(names):
            lib.rav_profile_read(mg.h, lev, k, cnt, tot)
            if cnt.value:
                row[nm] = round(1e3 * tot.value / kb, 2)
        breakdown[f"N={mg.counts(lev)['N']}"] = row
    lib.rav_profile_enable(mg.h, 0, -1)
    ms = max_over_ranks(ms, dist, "cuda")
    value = replicas_value(ws, n, args.steps, ms)

    # ---- roofline of the dominant kernel: fine-level subdomain apply ----
    q1 = W.get("elem", 0) == 1
    flops, bytes_alg, stored = patch_work(W["dim"], W["N"], W["prec"], n, q=1 if q1 else 2)
    if args.fused:  # the fused kernel also forms the residual: one FMA per assembled entry
        flops += 2.0 * mg.counts(fine)["nnz"]
    if W["prec"] in (0, 4):  # fp64 arithmetic: bound by the FP64 pipes, not HBM
        roof = {"bound": "alu", "achieved": flops / (apply_ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s",
                "peak_note": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"}
        meas = ctypes_f64()
        if lib.rav_fp64_fma_rate(ctypes.byref(meas), stream.cuda_stream) == 0:
            roof["peak_measured"] = meas.value
            roof["frac_of_measured"] = roof["achieved"] / meas.value
            roof["peak_measured_note"] = ("rav_fp64_fma_rate: 8 independent FP64 FMA chains per thread, "
                                          "8 x 256 threads per SM, CUDA events")
    else:
        mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
        peak = json.load(open(mp))["hbm_gbs"] if os.path.exists(mp) else 6800.0
        roof = {"bound": "hbm", "achieved": bytes_alg / (apply_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                "peak_note": "of measured (MEASURED_PEAKS.json hbm_gbs)" if os.path.exists(mp) else
                "of fallback (6.8 TB/s, one earlier GB300 copy measurement)"}
        # what a plain read of the same byte count reaches (short kernels stay
        # below the large-copy bandwidth): context for the fraction above
        rr = ctypes_f64()
        if lib.rav_hbm_read_rate(ctypes.c_int64(int(bytes_alg)), ctypes.byref(rr), stream.cuda_stream) == 0:
            roof["size_matched_read_gbs"] = rr.value
            roof["frac_of_size_matched_read"] = roof["achieved"] / rr.value
            roof["size_matched_read_note"] = ("rav_hbm_read_rate: coalesced 16-byte evict-first read of the "
                                              "kernel's algorithmic bytes after an L2 flush, CUDA events")
    roof["frac"] = roof["achieved"] / roof["peak"]
    staged = sm.apply_staged(fine) if W["prec"] in (5, 6) and not q1 else 0
    stream_k = staged == 1  # one thread per subdomain: the streamed kernel
    traffic = (measured_traffic(f"rav_apply_stream_{args.workload}", "stream.cu") if stream_k else
               measured_traffic(f"rav_apply_staged_{args.workload}", "staged.cu") if staged else
               measured_traffic(f"rav_apply_{args.workload}"))
    roof["traffic"] = traffic
    roof["kernel"] = (("k_fused_q1" if q1 else "k_fused_q2") if args.fused else "k_rav_apply_q1" if q1 else
                      ("k_rav_apply_stream" if stream_k else "k_rav_apply_staged" if staged else "k_rav_apply_fact")
                      if W["prec"] in (0, 5, 6) else "k_rav_apply") + " (fine level)"
    if args.fused:
        roof["traffic"] = None
    roof["launch_ms"] = apply_ms
    roof["launches_timed"] = apply_launches
    roof["algorithmic_bytes"] = bytes_alg
    roof["algorithmic_flops"] = flops
    roof["hbm_gbs_equiv"] = bytes_alg / (apply_ms / 1e3) / 1e9

    out = {"metric": "V-cycle DoFs/s", "value": value, "unit": "DoF/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(W, n, mg.counts(fine)["nnz"], stored, ws, args.fused),
           "roofline": roof, "gpu_launches": int(launches), "clocks": clocks,
           "ms_per_step_kernel_by_kernel": ms_nograph / args.steps,
           "breakdown_us_per_cycle": breakdown,
           "launch_shapes": {f"N={mg.counts(lev)['N']}": {
               "residual": "node-blocked" if mg.residual_blocked(lev) else f"rows, {mg.residual_split(lev)} thr/row",
               **({"apply": (f"staged, {sm.apply_staged(lev)} thr/subdomain" if sm.apply_staged(lev)
                             else f"grouped, split {sm.apply_split(lev)}")} if lev > 0 and W["prec"] in (0, 5, 6)
                  and not q1 else {})} for lev in range(W["nlev"])}}

    # ---- end to end through the public API with host buffers ----
    # Every step uploads its x and b from pinned host memory, runs one V-cycle
    # and reads its x back.  Steps are pipelined over two device buffer pairs:
    # the upload of step k+1 (one stream) and the read-back of step k-1
    # (another) overlap the V-cycle of step k (a third), ordered by events.
    if not args.no_e2e:
        xh = x0.cpu().pin_memory()
        bh = b.cpu().pin_memory()
        xo = [torch.empty_like(xh).pin_memory() for _ in range(2)]
        xd = [torch.empty_like(x) for _ in range(2)]
        bd = [torch.empty_like(b) for _ in range(2)]
        s_up, s_comp, s_down = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        up_done = [torch.cuda.Event() for _ in range(2)]
        comp_done = [torch.cuda.Event() for _ in range(2)]
        down_done = [torch.cuda.Event() for _ in range(2)]
        for j in range(2):  # capture each buffer pair's cycle before timing
            xd[j].copy_(xh)
            bd[j].copy_(bh)
            with torch.cuda.stream(s_comp):
                mg.vcycle(sm, xd[j], bd[j], nu, nu)
        torch.cuda.synchronize()
        K = max(10, args.steps // 10)
        barrier()
        t0 = time.perf_counter()
        for k in range(K):
            j = k % 2
            if k >= 2:
                s_up.wait_event(down_done[j])  # step k-2 has left buffer j
            with torch.cuda.stream(s_up):
                xd[j].copy_(xh, non_blocking=True)
                bd[j].copy_(bh, non_blocking=True)
                up_done[j].record(s_up)
            s_comp.wait_event(up_done[j])
            with torch.cuda.stream(s_comp):
                mg.vcycle(sm, xd[j], bd[j], nu, nu)
                comp_done[j].record(s_comp)
            s_down.wait_event(comp_done[j])
            with torch.cuda.stream(s_down):
                xo[j].copy_(xd[j], non_blocking=True)
                down_done[j].record(s_down)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out["e2e"] = {"value": ws * n * K / dt, "unit": "DoF/s", "h2d_bytes_per_step": 2 * n * 8,
                      "d2h_bytes_per_step": n * 8, "steps": K,
                      "pipelined": "uploads and read-backs of neighbouring steps overlap each V-cycle "
                                   "(three streams, two device buffer pairs)"}

    # ---- time to a 1e-8 residual reduction (host-driven stationary solve) ----
    if not args.no_tol:
        xs = x0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, hist, rc = mg.solve(sm, xs, b, tol=1e-8, maxit=200, nu_pre=nu, nu_post=nu, raise_on_error=False)
        dt = time.perf_counter() - t0
        out["time_to_tol"] = {"seconds": dt, "cycles": it, "tol": 1e-8, "status": rc,
                              "rho": float(hist[-1] ** (1.0 / max(it, 1)))}

    # ---- reduced-precision and batched forms against plain FP64, to 1e-8 ----
    if rank == 0 and ws == 1 and not args.no_forms and args.workload == "2d512" and not args.N:
        try:
            out["forms_to_tol"] = forms_vs_fp64()
        except Exception as exc:  # the measured line above still prints; the failure is reported in it
            out["forms_to_tol"] = {"error": f"{type(exc).__name__}: {exc}"}

    if rank == 0 and ws == 1 and not args.no_cpu_baseline and W["dim"] == 2:
        v, dt, va, dta, cores, nn = cpu_baseline(W)
        out["cpu_baseline"] = {"value": v, "unit": "DoF/s", "cores": 1, "kind": "oracle",
                               "sample": "1 V(2,2) cycle of the full workload on one host core after untimed "
                                         f"set-up ({dt:.2f} s)",
                               "all_cores": {"value": va, "unit": "DoF/s", "cores": cores, "kind": "oracle",
                                             "sample": f"the same cycle with the subdomain loops on {cores} "
                                                       f"threads, the rest serial ({dta:.2f} s)"}}
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def ctypes_i64():
    import ctypes
    return ctypes.c_int64(0)


def ctypes_f64():
    import ctypes
    return ctypes.c_double(0.0)


def batch_problems(nprob, nrhs, q1=False):
    """The batched workload's hierarchies and vectors: nprob 2-D lid-driven
    cavities, N = 16 m with m uniform on {2..16} (seed 2103), nrhs right-hand
    sides each (lid values + iid N(0,1) forcing on free velocity DoFs),
    RHS-interleaved.  q1: the stabilised Q1-Q1 element (beta 0.02)."""
    import numpy as np
    import torch
    import paper_2103_10127_gb300 as R
    from paper_2103_10127_gb300 import inputs

    sizes = inputs.batched_sizes(inputs.BASE_SEED, nprob)
    mgs, xs, bs = [], [], []
    for i, N in enumerate(sizes):
        N = int(N)
        if q1:
            mg = R.Multigrid(2, N, inputs.levels_for(N), bc=R.BC_CAVITY, element=R.ELEM_Q1Q1, beta=0.02)
        else:
            mg = R.Multigrid(2, N, inputs.levels_for(N), bc=R.BC_CAVITY)
        M = (1 if q1 else 2) * N + 1
        idx = np.indices((M, M)).reshape(2, -1)[::-1]
        inner = np.repeat(np.all((idx > 0) & (idx < M - 1), axis=0), 2)
        free = np.concatenate([inner, np.zeros((N + 1) ** 2, bool)])
        lid = mg.rhs(R.F_NONE).cpu().numpy()
        b = np.repeat(lid[:, None], nrhs, axis=1)
        b[free, :] += inputs.normal(inputs.BASE_SEED + 7919 * (i + 1), int(free.sum()) * nrhs).reshape(-1, nrhs)
        x0 = mg.initial_guess().cpu().numpy()
        mgs.append(mg)
        bs.append(torch.from_numpy(np.ascontiguousarray(b)).cuda())
        xs.append(torch.from_numpy(np.ascontiguousarray(np.repeat(x0[:, None], nrhs, axis=1))).cuda())
    return sizes, mgs, xs, bs


def single_problem_fp64_ms(mgs, nrhs, omega):
    """The plain FP64 form on the batch's problems: one single-problem V(2,2)
    cycle (FP64 factored inverses, captured graph) per problem and right-hand
    side, CUDA-event timed and summed (ms)."""
    import torch
    import paper_2103_10127_gb300 as R

    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    for mg in mgs:
        sm64 = R.Smoother(mg, R.RAV, R.F64, omega)
        x1, b1 = mg.vector(), mg.rhs(R.F_NONE)
        mg.vcycle(sm64, x1, b1, 2, 2)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(nrhs):
            mg.vcycle(sm64, x1, b1, 2, 2)
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
        del sm64
    return total


def run_batch(args, q1=False):
    """256 independent 2-D lid-driven cavities, N = 16 m with m uniform on
    {2..16} (seeded), 8 right-hand sides each (lid values + iid N(0,1) forcing
    on free velocity DoFs), FP32 patch inverses, FP64 residuals; a step is one
    batched V(2,2) cycle of every problem and right-hand side.  q1: the same
    problems on the stabilised Q1-Q1 element (beta 0.02, RAV omega 0.66)."""
    import torch
    import paper_2103_10127_gb300 as R
    from paper_2103_10127_gb300 import _capi, inputs

    torch.cuda.set_device(0)
    lib = _capi.load()
    nprob, nrhs = args.nprob, 8
    t0 = time.perf_counter()
    omega = 0.66 if q1 else 0.5
    sizes, mgs, xs, bs = batch_problems(nprob, nrhs, q1)
    sms = [R.Smoother(mg, R.RAV, R.F32, omega) for mg in mgs]
    bt = R.Batch(mgs, sms, nrhs)
    setup_s = time.perf_counter() - t0
    dofs = sum(m.n() for m in mgs)
    x_init = [x.clone() for x in xs]
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        bt.vcycle(xs, bs, 2, 2)
    torch.cuda.synchronize()
    launches0 = lib.rav_kernel_launches()
    clk = clocks_start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        bt.vcycle(xs, bs, 2, 2)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clocks = clocks_stop(clk, 0)
    launches = lib.rav_kernel_launches() - launches0
    # per-depth, per-kernel-class breakdown (separate untimed pass, events around every phase)
    kb = max(2, args.steps // 2)
    bt.profile(True)
    for _ in range(kb):
        bt.vcycle(xs, bs, 2, 2)
    torch.cuda.synchronize()
    breakdown = {}
    names = ["apply", "residual", "restrict", "prolong", "coarse"]
    for d in range(int(max(inputs.levels_for(int(N)) for N in sizes))):
        row = {}
        for k, nm in enumerate(names):
            c, t = bt.profile_read(d, k)
            if c:
                row[nm] = round(t / kb, 3)
        if row:
            breakdown[f"depth {d}"] = row
    bt.profile(False)
    for x, xi in zip(xs, x_init):
        x.copy_(xi)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it, ratios, rc = bt.solve(xs, bs, tol=1e-8, maxit=100, raise_on_error=False)
    tsolve = time.perf_counter() - t0
    # the same batch with the interior subdomains of uniform levels on the tensor cores
    tensor = None
    if not q1:
        nlev_tc = bt.tensor_apply(True)
        for x, xi in zip(xs, x_init):
            x.copy_(xi)
        for _ in range(2):
            bt.vcycle(xs, bs, 2, 2)
        torch.cuda.synchronize()
        clk_tc = clocks_start()
        e0.record(stream)
        for _ in range(args.steps):
            bt.vcycle(xs, bs, 2, 2)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_tc = e0.elapsed_time(e1)
        bt.profile(True)
        for _ in range(kb):
            bt.vcycle(xs, bs, 2, 2)
        torch.cuda.synchronize()
        bd_tc = {}
        for d in range(int(max(inputs.levels_for(int(N)) for N in sizes))):
            c, tm = bt.profile_read(d, 0)
            if c:
                bd_tc[f"depth {d}"] = round(tm / kb, 3)
        bt.profile(False)
        for x, xi in zip(xs, x_init):
            x.copy_(xi)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        it_tc, _, rc_tc = bt.solve(xs, bs, tol=1e-8, maxit=100, raise_on_error=False)
        tsolve_tc = time.perf_counter() - t1
        tensor = {"levels_using_it": nlev_tc, "ms_per_cycle": ms_tc / args.steps,
                  "apply_ms_per_cycle_by_depth": bd_tc, "clocks": clocks_stop(clk_tc, 0),
                  "time_to_tol": {"seconds": tsolve_tc, "max_cycles": int(it_tc.max()), "status": rc_tc}}
        bt.tensor_apply(False)
    single_ms = 0.0 if args.no_single else single_problem_fp64_ms(mgs, nrhs, omega)
    out = {"metric": "V-cycle DoFs/s", "value": dofs * nrhs * args.steps / (ms / 1e3), "unit": "DoF/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{nprob} 2D {'stabilised Q1-Q1 (beta 0.02)' if q1 else 'Q2-Q1'} lid-driven "
                                  f"cavities, N = 16 m, m ~ U{{2..16}} (seed 2103), {nrhs} RHS each, RAV V(2,2) "
                                  f"omega {omega}, FP32 patch inverses, FP64 residuals",
                      "problems": nprob, "rhs": nrhs, "dofs_total": dofs, "sizes_min_max": [int(sizes.min()),
                                                                                            int(sizes.max())],
                      "tuning": dict(bt.tuning(), apply_tile_by_depth=bt.apply_tile()), "setup_s": setup_s},
           "gpu_launches": int(launches), "clocks": clocks, "breakdown_ms_per_cycle": breakdown,
           "single_problem_fp64": None if args.no_single else {
               "ms_per_cycle_all": single_ms, "value": dofs * nrhs / (single_ms / 1e3), "unit": "DoF/s",
               "note": "one-problem, one-RHS V(2,2) cycles with FP64 factored inverses, graphs, summed over "
                       "every problem and RHS"},
           "time_to_tol": {"seconds": tsolve, "max_cycles": int(it.max()), "min_cycles": int(it.min()),
                           "status": rc, "tol": 1e-8},
           "tensor_core_shared_inverse_apply": tensor}
    print(json.dumps(out), flush=True)


def timed_solve(mg, sm, b, outer, reps=3, maxit=200):
    """Best wall time of `reps` solves to a 1e-8 residual reduction from the
    initial guess (stationary V(2,2) multigrid, or FGMRES(30) preconditioned by
    one V(2,2) cycle), after one warm call that captures the cycle graphs."""
    import torch
    x = mg.initial_guess()
    mg.solve(sm, x, b, tol=1e-8, maxit=1, outer=outer, raise_on_error=False)
    best = None
    for _ in range(reps):
        x = mg.initial_guess()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, hist, rc = mg.solve(sm, x, b, tol=1e-8, maxit=maxit, outer=outer, raise_on_error=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        best = dt if best is None or dt < best else best
    return {"seconds": best, "iterations": int(it), "status": int(rc), "final_ratio": float(hist[-1])}


def forms_vs_fp64(nprob=256, nrhs=8):
    """Time to a 1e-8 residual reduction of the reduced-precision and batched
    forms against the plain FP64 GPU form, on the same problems, each group
    with its own clock record:
      2d512:  the 512^2 manufactured problem, stationary RAV(0.5) V(2,2), FP64
              vs FP32 vs BF16 factored inverses (fp32 accumulation);
      3d32:   the 32^3 blob problem (contrast <= 1e3, sinker), FGMRES(30) with
              one V(2,2) cycle, FP64 vs FP32 vs BF16 factored inverses;
      batch:  the 256 cavities x 8 right-hand sides on the batched path with
              FP32 rows against the same batched path with FP64 rows (the
              batching gain and the precision gain apart), and the sum of the
              single-problem FP64 cycles over every problem and RHS."""
    import torch
    import paper_2103_10127_gb300 as R
    from paper_2103_10127_gb300 import inputs

    # the last form adds fp32 coarse-grid work: residuals on the levels between
    # the coarsest and the finest (rav_set_coarse_residual_f32) and the grid
    # transfers (rav_set_transfers_f32); the finest residual stays fp64
    formats = (("f64-factored", R.F64, False), ("f32-factored", R.F32_FACT, False),
               ("bf16-factored", R.BF16_FACT, False), ("bf16-factored+f32-coarse-grid", R.BF16_FACT, True))
    out = {}
    for key, dim, N, nlev, outer in (("2d512_stationary", 2, 512, 7, 0), ("3d32_fgmres30", 3, 32, 4, 1)):
        if dim == 2:
            mg = R.Multigrid(2, N, nlev, bc=R.BC_NOSLIP)
            b = mg.rhs(R.F_PSI)
        else:
            mg = R.Multigrid(3, N, nlev, blobs=inputs.viscosity_blobs(inputs.BASE_SEED, k=20, s_max=3.0),
                             bc=R.BC_NOSLIP)
            b = mg.rhs(R.F_SINKER)
        row = {"dofs": mg.n()}
        clk = clocks_start()
        for name, prec, coarse32 in formats:
            sm = R.Smoother(mg, R.RAV, prec, 0.5)
            mg.coarse_residual_f32(coarse32)
            mg.transfers_f32(coarse32)
            row[name] = timed_solve(mg, sm, b, outer)
            mg.coarse_residual_f32(False)
            mg.transfers_f32(False)
            del sm
        row["clocks"] = clocks_stop(clk, torch.cuda.current_device())
        base = row["f64-factored"]["seconds"]
        row["speedup_vs_f64"] = {nm: base / row[nm]["seconds"] for nm, _, _ in formats}
        out[key] = row
        del mg
    # the batch: the same problems and right-hand sides on the batched path, FP32 and FP64 rows
    t0 = time.perf_counter()
    sizes, mgs, xs, bs = batch_problems(nprob, nrhs)
    x_init = [x.clone() for x in xs]
    row = {"problems": nprob, "rhs": nrhs, "dofs_total": int(sum(m.n() for m in mgs))}
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = clocks_start()
    # "f32-coarse-residuals": fp32 residuals below the finest depth
    # (batch_set_coarse_residual_f32); "f32-coarse-grid": those and fp32
    # transfers (batch_set_transfers_f32); the other rows keep fp64 ones
    for name, prec in (("batched-f32-rows", R.F32), ("batched-f32-rows-tensor-core", R.F32),
                       ("batched-f32-rows-f32-coarse-residuals", R.F32),
                       ("batched-f32-rows-f32-coarse-grid", R.F32), ("batched-f64-rows", R.F64_ROWS)):
        sms = [R.Smoother(mg, R.RAV, prec, 0.5) for mg in mgs]
        bt = R.Batch(mgs, sms, nrhs)
        if name.endswith("tensor-core"):
            bt.tensor_apply(True)
        if name.endswith("f32-coarse-residuals") or name.endswith("f32-coarse-grid"):
            bt.coarse_residual_f32(True)
        if name.endswith("f32-coarse-grid"):
            bt.transfers_f32(True)
        for _ in range(2):
            bt.vcycle(xs, bs, 2, 2)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            bt.vcycle(xs, bs, 2, 2)
        e1.record(stream)
        torch.cuda.synchronize()
        cyc = e0.elapsed_time(e1) / 3
        for x, xi in zip(xs, x_init):
            x.copy_(xi)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        it, _, rc = bt.solve(xs, bs, tol=1e-8, maxit=100, raise_on_error=False)
        torch.cuda.synchronize()
        row[name] = {"ms_per_cycle": cyc, "seconds_to_tol": time.perf_counter() - t1, "status": int(rc),
                     "cycles_min_max": [int(it.min()), int(it.max())]}
        for x, xi in zip(xs, x_init):
            x.copy_(xi)
        del bt, sms
    row["single-problem-f64-factored"] = {"ms_per_cycle_all": single_problem_fp64_ms(mgs, nrhs, 0.5),
                                          "note": "one V(2,2) cycle per problem and RHS, summed"}
    row["clocks"] = clocks_stop(clk, torch.cuda.current_device())
    row["setup_and_run_s"] = time.perf_counter() - t0
    f32, f64 = row["batched-f32-rows"], row["batched-f64-rows"]
    row["tensor_core_vs_cuda_core"] = f32["ms_per_cycle"] / row["batched-f32-rows-tensor-core"]["ms_per_cycle"]
    row["speedup"] = {"precision (batched f64 / batched f32, time to tol)": f64["seconds_to_tol"] /
                      f32["seconds_to_tol"],
                      "batching (single-problem f64 / batched f64, per cycle)":
                      row["single-problem-f64-factored"]["ms_per_cycle_all"] / f64["ms_per_cycle"],
                      "both (single-problem f64 / batched f32, per cycle)":
                      row["single-problem-f64-factored"]["ms_per_cycle_all"] / f32["ms_per_cycle"],
                      "both, fp32 residuals below the finest depth (single-problem f64 / batched f32, per cycle)":
                      row["single-problem-f64-factored"]["ms_per_cycle_all"] /
                      row["batched-f32-rows-f32-coarse-residuals"]["ms_per_cycle"],
                      "both, fp32 residuals below the finest depth and fp32 transfers "
                      "(single-problem f64 / batched f32, per cycle)":
                      row["single-problem-f64-factored"]["ms_per_cycle_all"] /
                      row["batched-f32-rows-f32-coarse-grid"]["ms_per_cycle"]}
    out["batch_256x8"] = row
    return out


def run_precision(args, q1=False):
    """3-D Stokes Q2-Q1 on 32^3 (or --N), 4 levels, 20 viscosity blobs
    (contrast up to 1e3, seed 2103), no-slip, sinker force; FGMRES(30) with one
    RAV V(2,2) cycle as preconditioner, fp64 residual / coarse solve / LU, the
    patch inverses stored as fp64 (factored), fp64 rows, fp32, bf16 or fp8:
    wall time and iterations to a 1e-8 residual reduction for each.  q1: the
    stabilised Q1-Q1 element (beta 0.02) on 64^3, 5 levels, contrast up to 1e2,
    RAV omega 0.66, with the same storage formats."""
    import torch
    import paper_2103_10127_gb300 as R
    from paper_2103_10127_gb300 import inputs

    torch.cuda.set_device(0)
    N = args.N or (64 if q1 else 32)
    nlev = args.levels or (5 if q1 else 4)
    blobs = inputs.viscosity_blobs(inputs.BASE_SEED, k=20, s_max=2.0 if q1 else 3.0)
    if q1:
        mg = R.Multigrid(3, N, nlev, blobs=blobs, bc=R.BC_NOSLIP, element=R.ELEM_Q1Q1, beta=0.02)
        formats = (("f64-factored", R.F64), ("f64-rows", R.F64_ROWS), ("f32", R.F32), ("bf16", R.BF16),
                   ("fp8", R.FP8), ("f32-factored", R.F32_FACT), ("bf16-factored", R.BF16_FACT))
    else:
        mg = R.Multigrid(3, N, nlev, blobs=blobs, bc=R.BC_NOSLIP)
        formats = (("f64-factored", R.F64), ("f64-rows", R.F64_ROWS), ("f32", R.F32), ("bf16", R.BF16),
                   ("fp8", R.FP8), ("f32-factored", R.F32_FACT), ("bf16-factored", R.BF16_FACT))
    b = mg.rhs(R.F_SINKER)
    n = mg.n()
    res = {}
    for name, prec in formats:
        t0 = time.perf_counter()
        sm = R.Smoother(mg, R.RAV, prec, 0.66 if q1 else 0.5)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        x = mg.initial_guess()
        mg.solve(sm, x, b, tol=1e-8, maxit=1, outer=1, raise_on_error=False)  # capture graphs, warm
        best = None
        for _ in range(3):
            x = mg.initial_guess()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, hist, rc = mg.solve(sm, x, b, tol=1e-8, maxit=200, outer=1, raise_on_error=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None or dt < best else best
        _, r_true = mg.residual(nlev - 1, x, b, norm=True)
        _, r0 = mg.residual(nlev - 1, mg.initial_guess(), b, norm=True)
        res[name] = {"seconds": best, "iterations": it, "status": rc, "true_ratio": r_true / r0,
                     "setup_s": setup}
        del sm
    base = res["f64-factored"]["seconds"]
    out = {"metric": "time to 1e-8 residual reduction (FGMRES(30), RAV V(2,2) preconditioner)",
           "value": min(r["seconds"] for r in res.values()), "unit": "s", "higher_is_better": False,
           "n_gpus": 1, "dtype": "f64", "data": "synthetic",
           "config": {"workload": (f"3D Stokes stabilised Q1-Q1 (beta 0.02) {N}^3, {nlev} levels, 20 blobs "
                                   "contrast <= 1e2, sinker") if q1 else
                      f"3D Stokes Q2-Q1 {N}^3, {nlev} levels, 20 blobs contrast <= 1e3, sinker", "dofs": n},
           "formats": res, "speedup_vs_f64_factored": {k: base / v["seconds"] for k, v in res.items()}}
    print(json.dumps(out), flush=True)


def run_steps(args, q1=False):
    """Smoothing-steps study (the paper's comparison of AV, MV and RAV over the
    number of smoothing steps, Sec. 4.2, Fig. 7) on the 2-D 512^2 manufactured
    Stokes problem (or --N): for nu = 1..6, a stationary V(nu, nu) solve to a
    1e-8 residual reduction with RAV (omega 0.5, FP64 factored inverses), AV
    (0.1) and coloured MV (0.66), all FP64; cycles, seconds and seconds per
    cycle for each.  q1: the same on the paper's stabilised Q1-Q1 element
    (beta 0.02) with its damping, RAV and MV 0.66, AV 0.1."""
    import torch
    import paper_2103_10127_gb300 as R

    torch.cuda.set_device(0)
    N = args.N or 512
    nlev = args.levels or 7
    if q1:
        mg = R.Multigrid(2, N, nlev, bc=R.BC_NOSLIP, element=R.ELEM_Q1Q1, beta=0.02)
    else:
        mg = R.Multigrid(2, N, nlev, bc=R.BC_NOSLIP)
    b = mg.rhs(R.F_PSI)
    res = {}
    for name, kind, omega in (("RAV", R.RAV, 0.66 if q1 else 0.5), ("AV", R.AV, 0.1),
                              ("MV", R.MV_COLOURED, 0.66)):
        sm = R.Smoother(mg, kind, R.F64, omega)
        row = {}
        for nu in range(1, 7):
            x = mg.initial_guess()
            mg.solve(sm, x, b, tol=1e-8, maxit=1, nu_pre=nu, nu_post=nu, raise_on_error=False)  # graphs, warm
            x = mg.initial_guess()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, hist, rc = mg.solve(sm, x, b, tol=1e-8, maxit=300, nu_pre=nu, nu_post=nu, raise_on_error=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            row[nu] = {"cycles": it, "status": rc, "seconds": dt, "ms_per_cycle": 1e3 * dt / max(it, 1),
                       "rho": float(hist[-1] ** (1.0 / max(it, 1)))}
        res[name] = row
        del sm
    best = {k: min((v for v in row.values() if v["status"] == 0), key=lambda v: v["seconds"], default=None)
            for k, row in res.items()}
    out = {"metric": "time to 1e-8 residual reduction per smoother and smoothing steps", "unit": "s",
           "higher_is_better": False, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"2D Stokes {'stabilised Q1-Q1 (beta 0.02)' if q1 else 'Q2-Q1'} {N}x{N}, "
                                  f"{nlev} levels, manufactured psi solution, stationary V(nu,nu), nu = 1..6",
                      "dofs": mg.n()},
           "results": res,
           "best_seconds": {k: (v["seconds"] if v else None) for k, v in best.items()}}
    print(json.dumps(out), flush=True)


def run_learned(args, q1=False):
    """Learned damping on 3-D 40^3 (or --N), 4 levels, 20 blobs with contrast
    up to 1e4 and z-graded cells of aspect 8 (seed 2103): the MLP is trained on
    line-search labels from eight 2-D/3-D runs with other seeds, then FGMRES(30)
    and stationary solves to 1e-8 with fixed damping 0.5 and with the learned
    per-level damping.  q1: the same on the stabilised Q1-Q1 element (beta
    0.02, fixed damping 0.66) with contrasts capped at 1e2 (beta does not
    scale with the viscosity) and cell aspects at 2 (at aspect 4 the fixed
    smoother already needs tens of FGMRES iterations on small grids)."""
    import torch
    import paper_2103_10127_gb300 as R
    from paper_2103_10127_gb300 import inputs, learned

    torch.cuda.set_device(0)
    omega = 0.66 if q1 else 0.5

    def spec(dim, N, nlev, seed, s_max, asp):
        if q1:
            asp = min(asp, 2.0)
        d = dict(dim=dim, N=N, n_levels=nlev, bc=R.BC_NOSLIP,
                 coords=inputs.graded_coordinates(N, asp, dim) if asp > 1 else None,
                 blobs=inputs.viscosity_blobs(seed, k=12 if seed != inputs.BASE_SEED else 20,
                                              s_max=min(s_max, 2.0) if q1 else s_max))
        if q1:
            d.update(element=R.ELEM_Q1Q1, beta=0.02)
        return d

    train_set = [(101, 2, 32, 3, 4.0, 8.0), (102, 2, 48, 3, 2.0, 1.0), (103, 3, 8, 2, 4.0, 8.0),
                 (104, 3, 12, 2, 2.0, 1.0), (105, 3, 16, 2, 3.0, 4.0), (106, 2, 64, 4, 3.0, 4.0),
                 (107, 3, 16, 2, 1.0, 1.0), (108, 2, 64, 4, 1.0, 2.0)]
    t0 = time.perf_counter()
    Xs, ys = [], []
    for seed, dim, N, nlev, s_max, asp in train_set:
        mg = R.Multigrid(**spec(dim, N, nlev, seed, s_max, asp))
        sm = R.Smoother(mg, R.RAV, R.F64, omega)
        X, y = learned.collect(mg, sm, mg.initial_guess(), mg.rhs(R.F_SINKER), cycles=3)
        Xs.append(X)
        ys.append(y)
    collect_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    P, losses = learned.train(torch.cat(Xs), torch.cat(ys), steps=1500, lr=3e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    N = args.N or 40
    nlev = args.levels or 4
    results = {}
    cases = ((("contrast1e2-aspect2", (2.0, 2.0)), ("contrast1e2-aspect1", (2.0, 1.0))) if q1 else
             (("contrast1e4-aspect8", (4.0, 8.0)), ("contrast1e3-aspect1", (3.0, 1.0))))
    for label, (s_max, asp) in cases:
        mg = R.Multigrid(**spec(3, N, nlev, inputs.BASE_SEED, s_max, asp))
        sm = R.Smoother(mg, R.RAV, R.F64, omega)
        b = mg.rhs(R.F_SINKER)
        row = {}
        # baseline: the best fixed damping of a sweep (FGMRES(30) iterations and seconds)
        sweep = {}
        for om in (0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9):
            sw = R.Smoother(mg, R.RAV, R.F64, om)
            x = mg.initial_guess()
            mg.solve(sw, x, b, tol=1e-8, maxit=1, outer=1, raise_on_error=False)
            x = mg.initial_guess()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            it, hist, rc = mg.solve(sw, x, b, tol=1e-8, maxit=200, outer=1, raise_on_error=False)
            torch.cuda.synchronize()
            sweep[str(om)] = {"iterations": it, "status": rc, "seconds": time.perf_counter() - t1}
            del sw
        row["fixed-sweep-fgmres"] = sweep
        for mode in ("fixed", "learned", "learned-per-subdomain"):
            if mode == "learned":
                learned.install(sm, P, shrink=0.0)
            elif mode == "learned-per-subdomain":
                learned.install(sm, P, shrink=1.0)
            for outer, oname in ((1, "fgmres"), (0, "stationary")):
                x = mg.initial_guess()
                mg.solve(sm, x, b, tol=1e-8, maxit=1, outer=outer, raise_on_error=False)
                x = mg.initial_guess()
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                it, hist, rc = mg.solve(sm, x, b, tol=1e-8, maxit=200, outer=outer, raise_on_error=False)
                torch.cuda.synchronize()
                row[f"{mode}-{oname}"] = {"iterations": it, "status": rc, "seconds": time.perf_counter() - t1}
        results[label] = row
    out = {"metric": "iterations / time to 1e-8, learned vs fixed damping", "n_gpus": 1, "data": "synthetic",
           "config": {"workload": f"3D Stokes {'stabilised Q1-Q1 (beta 0.02)' if q1 else 'Q2-Q1'} {N}^3, {nlev} "
                                  "levels, 20 blobs, sinker", "train_problems": 8,
                      "train_samples": int(sum(len(y) for y in ys)), "collect_s": collect_s, "train_s": train_s,
                      "loss_first_last": [losses[0][1], losses[-1][1]]},
           "results": results}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.workload in ("2d-batch", "2d-batch-q1"):
        run_batch(args, q1=args.workload == "2d-batch-q1")
        return
    if args.workload in ("3d-precision", "3d-precision-q1"):
        run_precision(args, q1=args.workload == "3d-precision-q1")
        return
    if args.workload in ("3d-learned", "3d-learned-q1"):
        run_learned(args, q1=args.workload == "3d-learned-q1")
        return
    if args.workload in ("2d-steps", "2d-steps-q1"):
        run_steps(args, q1=args.workload == "2d-steps-q1")
        return
    W = dict(WORKLOADS[args.workload])
    if args.N:
        W["N"] = args.N
        W["nlev"] = args.levels or W["nlev"]
        W["desc"] += f" [size override: {args.N}^{W['dim']}, {W['nlev']} levels]"
    if args.impl == "reference":
        run_reference(args, W)
    else:
        run_ours(args, W)


if __name__ == "__main__":
    main()
