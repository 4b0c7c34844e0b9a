"""ET-AIM march benchmark: seconds per time step and per-kernel HBM roofline.

A step is one time step of the march of Eq. 5 for every plane wave of the workload:
excitation, delayed-interaction sum over the N_g history slabs (right-hand side), and
the solve of the immediate system -- GMRES with the complex64 ET-AIM operator in
every iteration, then FP64 refinement of the residual (FP64 grid stages) until it
meets the tolerance.

Default workload (the largest configuration that fits one GPU): 4 x 4 array of PEC
spheres, icosphere subdivision 5 each (491 520 RWG), 1 GHz +-5 %, 384^3 grid (768 x 768
x 192 transforms: the z transform follows the 72-plane depth of the active box), 16
seeded plane waves, tol 1e-5, near-zone SAI preconditioner.  Inputs are synthetic
(seeded meshes and pulses).  The waves march in chunks of as many as fit in device
memory next to their history rings (all 16 in one at this workload): every chunk marches
W untimed steps from rest, then K timed steps; the step time is the sum over chunks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl aim|reference]
                    [--workload NAME]

Under torchrun every rank marches its own share of the plane waves (independent
right-hand sides, no collective); the reported time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ET-AIM s/time-step (with AIM matvec HBM GB/s vs peak)"
UNIT = "s/step"
CSRC = os.path.join(ROOT, "paper_1408_7060_gb300", "csrc")

# solver settings per workload: preconditioner pattern radius (in near radii; the SAI
# rejects sets above 144 RWGs), FP64 refinement corrections allowed per step
PRESETS = {
    "array491k": dict(precond="sai", precond_scale=1.4, refine=4),
    "sphere7680": dict(precond="sai", precond_scale=2.5, refine=4),
    "sphere7680_wide": dict(precond="sai", precond_scale=2.5, refine=0),
    "sphere7680_b64": dict(precond="sai", precond_scale=2.5, refine=4),
    "ellipsoid20k": dict(precond="sai", precond_scale=1.0, refine=4),
}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_digest(kind):
    """Digest of a kernel's source text and the FFT core it uses: measured DRAM traffic
    is only reported while the kernel is unchanged since the capture."""
    src = open(os.path.join(CSRC, "operator_impl.cuh")).read()
    names = {"zconv": r"k_zconv(_p2)?", "interp_near": r"k_interp_near", "anterp_xfft": r"k_anterp_rows",
             "zrhs": r"k_zrhs(_spec)?(_tma)?"}
    if kind not in names:
        return None
    blocks = [m.group(0) for m in re.finditer(r"__global__ void __launch_bounds__\([^)]*\) " + names[kind]
                                              + r"\(.*?\n}\n", src, re.S)]
    if not blocks:
        return None
    h = hashlib.sha1("".join(blocks).encode())
    for f in ("fft.cuh", "fft_kernels.cuh"):
        h.update(open(os.path.join(CSRC, f)).read().encode())
    return h.hexdigest()[:16]


# DRAM bytes (read + write) of one launch, keyed by (kernel, workload, kernel_digest):
# the profiles/ summaries give the command and the capture.
TRAFFIC = {}


def kernel_bytes(kind, N, ns, nnz, ng, nb, box=None, esz=8, lz=None):
    """Algorithmic HBM bytes of one launch of each kernel (each byte counted once), for the
    grid lines each pass touches: with the active box (nx, ny, nz nodes per axis) the
    anterpolation writes the box rows of A, the forward y pass reads them and writes the
    box-z rows of the slab, the z pass reads and writes those rows, the inverse y pass
    writes the box rows of A and the inverse x pass the box of P.  lz: the length of the
    z transform (2N without a shorter one)."""
    L = 2 * N
    lz = lz or L
    bx, by, bz = box if box else (N, N, N)
    slab = 4 * bz * L * L * esz * nb          # [nb][4][z in box][L][L]
    spec = 4 * lz * L * L * esz * nb          # [nb][4][lz][L][L]: z-spectrum of a slab (power-of-two lz)
    pow2 = (lz & (lz - 1)) == 0
    A = 4 * bz * by * L * esz * nb            # [nb][4][z, y in box][L]
    P = 4 * bz * by * bx * esz * nb           # [nb][4][box]
    oct_ = (N + 1) ** 2 * (lz // 2 + 1) * esz  # one kernel spectrum octant
    lam = ns * 256 * (esz // 2)               # interpolation rows
    csrT = 64 * ns * (4 + 2 * esz) + (bz * by * N + 1) * 4
    near = nnz * (4 + 16) + (ns + 1) * 4
    vec = ns * 16 * nb
    return {
        "prep": vec + ns * 16 + ns * (esz + 16) * nb,
        "anterp_xfft": csrT + ns * esz * nb + A,
        "yfft_fwd": A + slab,
        "zconv": 2 * slab + 2 * oct_,
        "zrhs": ng * (spec if pow2 else slab) + slab + 2 * ng * oct_,
        "zfwd": slab + spec if pow2 else None,
        "yfft_inv": slab + A,
        "xfft_inv": A + P,
        "interp_near": P + lam + ns * 12 + near + 2 * vec,
    }.get(kind)


# FP32 arithmetic peak of the z pass's roofline (it is bound by FP32 instruction issue,
# not by DRAM): 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
ALU_KERNELS = ("zconv", "zrhs")


def kernel_flops(kind, N, nb, ng, lz=None):
    """Algorithmic FP32 flops of one launch of the z-pass kernels: per z column the
    conventional 5 n log2 n of a length-n complex FFT (n = lz, the z transform length)
    forward and inverse, and 6 n for the product with the kernel spectrum (the delay sum:
    N_g forward transforms and products, one inverse); 4 nb L^2 columns per launch."""
    L = 2 * N
    n = lz or L
    fft = 5 * n * math.log2(n)
    cols = 4 * nb * L * L
    if kind == "zconv":
        return cols * (2 * fft + 6 * n)
    if kind == "zrhs":
        return cols * ((ng + 1) * fft + 8 * ng * n)
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nme, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nme)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def reduce_max(x, ws, device="cuda"):
    """The largest of the ranks' values (the slowest rank's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def wave_share(n_waves, ws, rank):
    """Indices of the plane waves rank marches: contiguous, disjoint, covering all waves
    (independent right-hand sides; no data-path exchange between ranks)."""
    return np.array_split(np.arange(n_waves), ws)[rank]


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# --------------------------------------------------------------------------- memory plan

Z_LENGTHS = (16, 32, 64, 128, 192, 256, 768)   # z transform lengths the library is built for


def box_depth(w):
    """Estimated z-planes of the active box (the stencils of edges between the mesh's
    lowest and highest vertices, 4 nodes each) and the z transform length the context
    picks for it (the shortest built length >= 2 nz)."""
    V = w.mesh[0]
    N, L = w.grid_n, 2 * w.grid_n
    nz = min(N, int((V[:, 2].max() - V[:, 2].min()) / w.h) + 5)
    lz = next((n for n in Z_LENGTHS if 2 * nz <= n <= L), L)
    return nz, lz


def chunk_size(w, ng_est, refine, total_bytes, restart=50):
    """Right-hand sides per context that fit in device memory: per-RHS work buffers and
    history ring over the box's z-planes (x/y-transformed slabs for z lengths with a
    factor 3, z-spectra for powers of two) against the tables (kernel octants in both
    precisions, anterpolation, near zone and preconditioner estimated at 80 entries per
    row, FP64 refinement buffers of up to 8 GiB) and a 6 GB margin."""
    N, L = w.grid_n, 2 * w.grid_n
    nz, lz = box_depth(w)
    V, F = w.mesh
    ns = len(F) * 3 // 2
    es = 8
    Z = lz if (lz & (lz - 1)) == 0 else nz
    grid = 4 * nz * (N * L + L * L + N * N)
    per = es * grid + ng_est * es * 4 * Z * L * L + ns * 16 * (restart + 2 * ng_est + 10)
    base = (ng_est + 1) * 2 * (N + 1) ** 2 * (lz // 2 + 1) * 24 + ns * 256 * 12 + 64 * ns * 52 + 4 * N ** 3
    base += ns * 80 * (16 * (ng_est + 1) + 8 + 24)
    if refine:
        base += min(16 * grid * 16, 8 << 30)
    return max(1, int((total_bytes - base - 6e9) // per))


# --------------------------------------------------------------------------- GPU arm

def run_aim(args):
    import torch

    from paper_1408_7060_gb300 import AimContext, abi
    from paper_1408_7060_gb300.inputs import make_workload

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.init()
    pre = dict(PRESETS.get(args.workload, dict(precond="sai", precond_scale=1.0, refine=4)))
    if args.precond:
        pre["precond"] = args.precond
    if args.refine is not None:
        pre["refine"] = args.refine
    if args.precond_scale:
        pre["precond_scale"] = args.precond_scale
    w = make_workload(args.workload, precond=pre["precond"], refine=pre["refine"], autotune=args.autotune)
    w.refine_every = max(1, args.refine_every)
    w.rhs_blocked = args.rhs_blocked
    if args.basis:
        w.basis = args.basis
    if args.order:
        w.order = args.order
    w.precond_radius = pre["precond_scale"] * w.near_radius if w.precond == "sai" else 0.0
    waves_k, waves_p = w.khat, w.phat
    if args.max_waves:
        waves_k, waves_p = waves_k[:args.max_waves], waves_p[:args.max_waves]
    if ws > 1:  # every rank its own share of the plane waves (independent right-hand sides)
        share = wave_share(len(waves_k), ws, rank)
        waves_k, waves_p = waves_k[share], waves_p[share]
    nw = len(waves_k)
    total = torch.cuda.get_device_properties(local).total_memory
    # N_g estimate for the memory plan (the context reports the exact value)
    V = w.mesh[0]
    diam = float(np.linalg.norm(V.max(0) - V.min(0))) + 3 * math.sqrt(3) * w.h
    ng_est = int(diam / (299792458.0 * w.dt) + w.order) + 1
    chunk = min(nw, args.chunk or chunk_size(w, ng_est, w.refine, total))
    stream = torch.cuda.Stream()
    ctx = None
    while ctx is None:
        try:
            t0 = time.time()
            with torch.cuda.stream(stream):
                ctx = AimContext.from_workload(w, batch_max=chunk, stream=stream.cuda_stream)
            log(f"setup {w.name}: {time.time() - t0:.1f} s, {chunk} waves per context, "
                f"{ctx.info['device_bytes'] / 1e9:.1f} GB")
        except abi.AimError as e:
            if e.code != abi.AIM_ERR_OOM or chunk == 1:
                raise
            chunk -= 1
            log(f"out of memory, {chunk} waves per context")
    info = ctx.info
    ns = ctx.ns
    chunks = [(waves_k[i:i + chunk], waves_p[i:i + chunk]) for i in range(0, nw, chunk)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    K, W = args.steps, args.warmup
    Ke = max(1, min(K, args.e2e_steps))
    keep = min(K, args.compare_steps)          # steps of wave 0 kept for the comparisons
    wave0 = []
    step_ms = np.zeros((len(chunks), K))
    iters, split, resid, corr = [], [], [], 0
    e2e_s = 0.0
    prof = None
    barrier(ws)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    launches = 0
    for ci, (k, p) in enumerate(chunks):
        nb = len(k)
        warm = torch.empty((W, nb, ns), dtype=torch.complex128, device="cuda")
        ctx.march(k, p, w.sigma, w.t_d, W, w.tol, out=warm)
        if ci == 0:
            wave0.append(warm[:, 0].cpu().numpy())
        outs = torch.empty((K, 1, nb, ns), dtype=torch.complex128, device="cuda")
        _, l_before = ctx.get_profile()   # the library's launch counter (synchronises)
        torch.cuda.synchronize()
        evs = []
        for s in range(K):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)            # L2 flush between timed steps (inputs are also > L2)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, st, rc = ctx.march_continue(k, p, w.sigma, w.t_d, 1, w.tol, out=outs[s])
            b.record(stream)
            evs.append((a, b))
            iters.append(st["total_iters"] / nb)
            split.append((st["rhs_ms"], st["solve_ms"]))
            resid.append(st["max_rel_res"])
            corr += st["refine_corrections"]
        torch.cuda.synchronize()
        launches += ctx.get_profile()[1] - l_before  # kernels launched in the timed steps
        step_ms[ci] = [a.elapsed_time(b) for a, b in evs]
        if ci == 0:
            wave0.append(outs[:keep, 0, 0].cpu().numpy())
        # end to end through the C ABI with host buffers: Ke more steps of the same march,
        # currents written to pinned host memory every step
        host_out = torch.empty((1, nb, ns), dtype=torch.complex128).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(Ke):
            ctx.march_continue(k, p, w.sigma, w.t_d, 1, w.tol, out=host_out)
        torch.cuda.synchronize()
        e2e_s += (time.perf_counter() - t0) / Ke
        if ci == 0:  # per-kernel device time: a few more steps with per-launch events
            ctx.profile(True)
            pout = torch.empty((1, nb, ns), dtype=torch.complex128, device="cuda")
            for _ in range(args.profile_steps):
                ctx.march_continue(k, p, w.sigma, w.t_d, 1, w.tol, out=pout)
            prof, _ = ctx.get_profile()
            ctx.profile(False)
            prof_nb = nb
        log(f"chunk {ci + 1}/{len(chunks)} ({nb} waves): {np.mean(step_ms[ci]):.1f} ms/step")
    clk = clocks.stop()
    torch.cuda.synchronize()
    barrier(ws)
    t_step = reduce_max(float(step_ms.sum(axis=0).mean()) / 1e3, ws)
    e2e = reduce_max(e2e_s, ws)

    # roofline of the dominant operator kernel (algorithmic bytes / event time)
    hbm, src = load_peaks()
    box = tuple(hi - lo + 1 for lo, hi in zip(info["box_lo"], info["box_hi"]))
    lz = info["z_len"]
    kb = lambda kind: kernel_bytes(kind, w.grid_n, ns, info["near_nnz"], info["n_delays"], prof_nb, box, lz=lz)
    tot_ms = sum(v[1] for v in prof.values()) or 1e-12
    kernels = {}
    for kind, (n_l, ms_l) in prof.items():
        if not n_l:
            continue
        b = kb(kind)
        kernels[kind] = {"launches": n_l, "ms": round(ms_l, 4), "share": round(ms_l / tot_ms, 4),
                         "gbs": round(b / (ms_l / n_l * 1e-3) / 1e9, 1) if b and ms_l > 0 else None,
                         "frac": round(b / (ms_l / n_l * 1e-3) / 1e9 / hbm, 4) if b and ms_l > 0 else None}
    for kind in ALU_KERNELS:
        if kind in kernels and kernels[kind]["ms"] > 0:
            fl = kernel_flops(kind, w.grid_n, prof_nb, info["n_delays"], lz)
            tf = fl / (kernels[kind]["ms"] / kernels[kind]["launches"] * 1e-3) / 1e12
            kernels[kind]["tflops"] = round(tf, 2)
            kernels[kind]["alu_frac"] = round(tf / FP32_PEAK_TFLOPS, 4)
    dom = max((kd for kd in kernels if kb(kd)), key=lambda kd: kernels[kd]["ms"])
    n_l, ms_l = prof[dom]
    per_launch_ms = ms_l / n_l
    achieved = kb(dom) / (per_launch_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": t_step, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": t_step * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 grid / f64 solve + f64 refinement" if w.refine else "c64 grid / f64 solve",
        "data": "synthetic",
        "config": {"workload": w.name, "ns": ns, "grid": f"{w.grid_n}^3",
                   "fft": f"{2 * w.grid_n} x {2 * w.grid_n} x {lz} (z: {box[2]} box planes)",
                   "n_delays": info["n_delays"], "near_nnz": info["near_nnz"], "plane_waves": nw,
                   "waves_per_context": chunk, "chunks": len(chunks), "tol": w.tol, "chi": round(w.chi, 3),
                   "precond": w.precond, "precond_radius_m": round(w.precond_radius, 6),
                   "precond_nnz": info["precond_nnz"], "fp64_refinement": w.refine,
                   "fp64_check_every": w.refine_every, "rhs": "blocked" if w.rhs_blocked else "direct",
                   "temporal_basis": f"{w.basis} {'Q' if w.basis == 'cppif' else 'M'}={w.order}",
                   "active_box": {"lo": list(info["box_lo"]), "hi": list(info["box_hi"])},
                   "launch_plan": {k: info["plan_" + k] for k in ("zw", "cw", "rp", "ypb")} |
                   {"source": ["default", "measured", "cached"][info["plan_source"]]},
                   "gmres_start": "previous step",
                   "l2": "inputs larger than L2; also flushed between timed steps (256 MB write)",
                   "parallelism": "plane waves split over GPUs" if ws > 1 else "single GPU"},
        "gmres_iters_per_wave_step": round(float(np.mean(iters)), 2),
        "fp64_relres_max": float(np.max(resid)),
        "refine_corrections_per_step": round(corr / (K * len(chunks)), 2),
        "split_ms_per_step": {"rhs": round(float(np.mean([s[0] for s in split])) * len(chunks), 3),
                              "solve": round(float(np.mean([s[1] for s in split])) * len(chunks), 3)},
        "roofline": roofline_entry(dom, kb(dom), kernel_flops(dom, w.grid_n, prof_nb, info["n_delays"], lz),
                                   per_launch_ms, hbm, src, w.name, prof_nb),
        "kernels": kernels,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": nw * 6 * 8, "d2h_bytes_per_step": nw * ns * 16},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    line["rel_error_vs_oracle"] = oracle_rows_error(w, ctx)
    wave0 = np.concatenate(wave0)
    k0, p0 = chunks[0][0][:1], chunks[0][1][:1]
    ctx.close()
    torch.cuda.empty_cache()
    if not args.no_compare:
        line["plain_c128"] = compare_march(w, k0, p0, wave0, stream, dict(precision="c128", refine=0), W, keep)
        line["no_refine"] = compare_march(w, k0, p0, wave0, stream, dict(refine=0), W, keep)
        line["diag_precond"] = compare_march(w, k0, p0, wave0, stream, dict(precond="diag"), W, keep)
    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w, info["n_delays"], float(np.mean(iters)), nw)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def roofline_entry(kind, nbytes, nflops, per_launch_ms, hbm, src, workload, nb):
    """The dominant kernel against its bound: the z-pass kernels against the FP32 peak
    (instruction-bound, DRAM a few per cent busy in the ncu profile), the other passes
    against the measured HBM copy bandwidth."""
    t = per_launch_ms * 1e-3
    traffic = TRAFFIC.get((kind, workload, kernel_digest(kind)))
    if kind in ALU_KERNELS and nflops:
        achieved = nflops / t / 1e12
        return {"bound": "alu", "kernel": kind, "achieved": round(achieved, 2), "peak": round(FP32_PEAK_TFLOPS, 1),
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz", "unit": "TFLOP/s",
                "frac": round(achieved / FP32_PEAK_TFLOPS, 4), "traffic": traffic,
                "hbm_gbs": round(nbytes / t / 1e9, 1), "hbm_frac": round(nbytes / t / 1e9 / hbm, 4),
                "flops_per_launch": nflops, "bytes_per_launch": nbytes, "ms_per_launch": round(per_launch_ms, 5),
                "waves_per_launch": nb}
    achieved = nbytes / t / 1e9
    return {"bound": "hbm", "kernel": kind, "achieved": round(achieved, 1), "peak": hbm, "peak_source": src,
            "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": traffic, "bytes_per_launch": nbytes,
            "ms_per_launch": round(per_launch_ms, 5), "waves_per_launch": nb}


def oracle_rows_error(w, ctx):
    """Relative error of the library's operator products against the oracle's direct
    sums on the rows stored by tests/golden/make_<workload>_rows.py (if present)."""
    from paper_1408_7060_gb300.inputs import seeded_vector

    path = os.path.join(ROOT, "tests", "golden", f"{w.name}_matvec_rows.txt")
    if not os.path.exists(path):
        return None
    ref = {}
    for ln in open(path):
        if ln.startswith("#"):
            continue
        m, r, re_, im = ln.split()
        ref.setdefault(int(m), []).append((int(r), float(re_) + 1j * float(im)))
    x = seeded_vector(ctx.ns, 11)[None]
    out = {}
    for m, rv in ref.items():
        rows = np.array([r for r, _ in rv])
        want = np.array([v for _, v in rv])
        got = ctx.matvec(m, x)[0][rows]
        out[f"Z{m}"] = float(np.linalg.norm(got - want) / np.linalg.norm(want))
    out["rows"] = len(rows)
    out["what"] = "complex64 product rows vs the oracle's direct grid sums + near zone"
    return out


def compare_march(w, k0, p0, ref, stream, over, W, keep):
    """Wave 0 marched with other settings (plain complex128 path, or the paper's diagonal
    preconditioner): its time per wave-step over `keep` steps after the same warm-up,
    its GMRES iterations, and its relative difference from the benchmark march."""
    import torch

    from paper_1408_7060_gb300 import AimContext

    with torch.cuda.stream(stream):
        c = AimContext.from_workload(w, batch_max=1, stream=stream.cuda_stream, **over)
    ns = c.ns
    out = torch.empty((W + keep, 1, ns), dtype=torch.complex128, device="cuda")
    c.march(k0, p0, w.sigma, w.t_d, W, w.tol, out=out[:W])
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    _, st, _ = c.march_continue(k0, p0, w.sigma, w.t_d, keep, w.tol, out=out[W:])
    b.record(stream)
    torch.cuda.synchronize()
    n = min(W + keep, len(ref))
    got, ref = out[:n, 0].cpu().numpy(), ref[:n]
    c.close()
    torch.cuda.empty_cache()
    return {"s_per_wave_step": a.elapsed_time(b) / keep / 1e3, "gmres_iters_per_step": st["total_iters"] / keep,
            "rel_diff_vs_bench_march": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "steps_compared": n, "settings": {k: v for k, v in over.items()}}


# --------------------------------------------------------------------------- CPU oracle

def oracle_setup(w):
    """The oracle's operator for the workload (its setup is not timed)."""
    from oracle import aim as oaim
    from oracle import efie
    from oracle.rwg import build_rwg

    rwg = build_rwg(*w.mesh)
    p = efie.Params(dt=w.dt, f_c=w.f_c, Q=w.order)
    return rwg, p, oaim.AimOracle(rwg, w.grid_n, w.h, w.origin, w.near_radius, p)


NODES_PER_SAMPLE = 4


def oracle_node_seconds(A, rng):
    """The oracle's direct grid sum of G^A_0 (the convolution of Eq. 5's grid part, as it
    stands) at NODES_PER_SAMPLE target nodes, over a source grid with values on every
    active node of the workload (random values: the cost depends only on the node sets);
    seconds per target node."""
    src = np.zeros(A.n ** 3, dtype=complex)
    src[A.active] = rng.standard_normal(len(A.active)) + 1j * rng.standard_normal(len(A.active))
    tg = rng.choice(A.active, NODES_PER_SAMPLE, replace=False)
    t0 = time.perf_counter()
    A.conv_direct(0, src, 0, targets=tg)
    return (time.perf_counter() - t0) / NODES_PER_SAMPLE


def node_sample_text(A, t, n_delays, iters, n_waves):
    return (f"the oracle's direct grid sum at {NODES_PER_SAMPLE} target nodes over the workload's "
            f"{len(A.active)} active nodes ({t * 1e3:.1f} ms per node), extrapolated to its direct-sum "
            f"products: x 4 components x {len(A.active)} nodes x {n_delays + iters:.1f} products per wave-step "
            f"(N_g = {n_delays} delayed + {iters:.1f} GMRES iterations) x {n_waves} waves")


def cpu_baseline(w, n_delays, iters_per_step, n_waves, samples=3):
    rwg, p, A = oracle_setup(w)
    rng = np.random.default_rng(0)
    t = float(np.mean([oracle_node_seconds(A, rng) for _ in range(samples)]))
    value = t * 4 * len(A.active) * (n_delays + iters_per_step) * n_waves
    return {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{samples} x " + node_sample_text(A, t, n_delays, iters_per_step, n_waves)}


def run_reference(args):
    ws, rank, local = dist_setup()
    if rank != 0:
        return
    from paper_1408_7060_gb300.inputs import make_workload

    w = make_workload(args.workload)
    t0 = time.time()
    rwg, p, A = oracle_setup(w)
    ng = A.n_delays
    log(f"oracle setup {w.name}: {time.time() - t0:.0f} s")
    iters = ITERS_PER_STEP.get(args.workload, 10.0)
    nw = len(w.khat)
    rng = np.random.default_rng(1)
    for _ in range(args.warmup):
        oracle_node_seconds(A, rng)
    ts = [oracle_node_seconds(A, rng) for _ in range(args.steps)]
    value = float(np.mean(ts)) * 4 * len(A.active) * (ng + iters) * nw
    sample = "per step: " + node_sample_text(A, float(np.mean(ts)), ng, iters, nw)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "ns": rwg.ns, "grid": f"{w.grid_n}^3", "n_delays": ng,
                   "plane_waves": nw},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": os.cpu_count(), "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# GMRES iterations per wave-step of the immediate system at the workload's tolerance as
# measured by the CUDA path (a property of the preconditioned linear system): the
# reference arm scales its per-product cost by it.
ITERS_PER_STEP = {"sphere7680": 7.4, "array491k": 10.0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="aim", choices=["aim", "reference"])
    ap.add_argument("--workload", default="array491k")
    ap.add_argument("--chunk", type=int, default=0, help="plane waves per context (default: as many as fit)")
    ap.add_argument("--max-waves", type=int, default=0, help="march only the first waves of the workload")
    ap.add_argument("--precond", default=None, choices=["sai", "diag"])
    ap.add_argument("--refine", type=int, default=None, help="FP64 refinement corrections per step (0: off)")
    ap.add_argument("--refine-every", type=int, default=1, help="FP64 residual checked at every k-th step")
    ap.add_argument("--rhs-blocked", type=int, default=0,
                    help="1: delayed grid sums by the multilevel blocked schedule (power-of-two z lengths)")
    ap.add_argument("--precond-scale", type=float, default=0.0, help="SAI pattern radius in near radii")
    ap.add_argument("--basis", default=None, choices=["cppif", "blif"],
                    help="temporal basis (default: the workload's); blif uses the workload's beta as its band")
    ap.add_argument("--order", type=int, default=0, help="CPPIF order Q or BLIF half-width M (0: the workload's)")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1, 2],
                    help="launch plan: 0 defaults, 1 tuned at setup (cached plan reused), 2 re-tuned")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--profile-steps", type=int, default=2)
    ap.add_argument("--compare-steps", type=int, default=3)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-compare", action="store_true", help="skip the complex128 and diagonal comparisons")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_aim(args)


if __name__ == "__main__":
    main()
