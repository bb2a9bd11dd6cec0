#!/usr/bin/env python3
"""Benchmark of the ParO hot path on one GB300: one ParO-merged SCF iteration (Algorithm 1 with the
SCF loop of Section 2.3) of the 64-atom synthetic diamond cell (a = 20.52 Bohr, E_cut = 15 Ha,
23847 plane waves, 72^3 grid, 144 orbitals, local + Kleinman-Bylander pseudopotential, LDA,
Pulay depth 8), in mixed precision (FP32 FFT / V.psi / PCG / KB projectors, FP64 Gram, Cholesky,
Rayleigh-Ritz, residuals and energies), with the plain-FP64 GPU iteration timed beside it.

One step = one ParO-SCF iteration: source problems by batched PCG, Cholesky orthonormalisation,
density and Pulay mixing, new potential, Rayleigh-Ritz, energy. The cell's bands 128 and 129 cross, so
the SCF uses Fermi-Dirac occupations (kT = 0.002 Ha). The timed iterations are those of the converged
run: the SCF first iterates from the seeded start vectors until the free energy changes by less than
1e-6 Ha/atom on two consecutive iterations. The mixed result is then compared with an FP64 run at
the fixed point, whose converged iteration is timed too. Every step's working set (orbitals, stick
buffers, PCG vectors: several hundred MB) exceeds the 129 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own independent copy of the cell (weak scaling, no data
exchange); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "si64_scf"
WORKLOAD_DESC = ("64-atom diamond cell a=20.52 Bohr, Ecut 15 Ha (23847 PW, 72^3 grid), 144 orbitals "
                 "(128 occupied), local + KB s/p pseudopotential, LDA-PZ, Pulay 8; one ParO-SCF iteration "
                 "(Algorithm 1)")
METRIC = "ParO-SCF iterations/s (64-atom cell, mixed FP32/FP64)"
UNIT = "iter/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p.get("hbm_gbs", 6800.0), "measured"
    except OSError:
        return 6800.0, "fallback"


# FP64 FMA rate of GB300 (plain ALU; the recipe's 1.25 TFLOP/s, which a probe reproduced).
FP64_TFLOPS = 1.25
FP64_SOURCE = "FP64 1.25 TFLOP/s (nominal, the profiling recipe's table)"
# FP32 FMA rate: nominal 152 SMs x 128 lanes x 2 flops x 2.07 GHz (maximum SM clock) = 80.5 TFLOP/s.
FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP32_SOURCE = "FP32 nominal: 152 SMs x 128 FMA lanes x 2 x 2070 MHz"


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.tmp.read())) if len(r) >= 9]
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def shapes(ctx):
    mil = ctx.miller()
    ncol = len({(int(a), int(b)) for a, b, _ in mil})
    n1, n2, n3 = ctx.grid
    nxr = len({int(a) for a, _, _ in mil})  # grid rows (x) that hold sticks: the y-direction lines of a plane
    return dict(nb=ctx.n_bands, npw=ctx.npw(), ncol=ncol, n1=n1, n2=n2, n3=n3, ngrid=n1 * n2 * n3,
                nproj=4 * ctx.n_atoms, nocc=ctx.n_occ, nxr=nxr)


def launch_work(name: str, s):
    """Algorithmic work of one launch of a profiled kernel with a fixed shape: (kind, amount).
    kind: "hbm" (bytes), "alu32"/"alu64" (FP32 / FP64 CUDA-core flops), "tensor" (complex products on the
    tensor cores: 8 M N K real flops of the product; the 3xTF32 split issues three TF32 MMAs for each)."""
    b = 16 if "<f64>" in name else 8
    nb, npw, ncol, n3, ng, npj = s["nb"], s["npw"], s["ncol"], s["n3"], s["ngrid"], s["nproj"]
    tag, _, kern = name.partition(":")
    if tag == "rr":
        if kern.startswith("k_zpass_inv"):
            return "hbm", nb * npw * b + nb * n3 * ncol * b
        if kern.startswith("k_plane"):
            # compute-bound (13.7 flop per byte, above the 9.9 balance): FFT flops, 5 N log2 N per line of N,
            # inverse and forward along y (stick rows) and x (every column), and the V psi product
            import math
            n1, n2, nxr = s["n1"], s["n2"], s["nxr"]
            per_plane = (2 * nxr * 5 * n2 * math.log2(n2) + 2 * n2 * 5 * n1 * math.log2(n1) + 2 * n1 * n2)
            return "alu32", nb * n3 * per_plane
        if kern.startswith("k_zpass_fwd"):
            return "hbm", nb * n3 * ncol * b + 2 * nb * npw * b
        if kern in ("k_gemm_cn_tc", "k_gemm_wx_tc"):
            return "tensor", 8 * npj * nb * npw
    if kern.startswith("k_gemm_cn") and tag in ("gram", "hsub"):
        # Hermitian products: the nb (nb + 1) / 2 distinct entries are the algorithmic work
        return "alu32", 8 * nb * (nb + 1) // 2 * npw
    if kern in ("k_gemm_cn_tc", "k_gemm_wx_tc", "k_gemm_cn_tcb", "k_gemm_wx_tcb") and tag == "pcg":
        # projector products of the inner solves: every source column, whatever the active set
        return "tensor", 8 * npj * nb * npw
    if kern == "k_gemm_wx_tc" and tag in ("orth",):
        return "tensor", 8 * nb * nb * npw
    if kern == "k_tridiag_cta":  # FP32 one-CTA reduction of the mixed eigensolver
        return "alu32", 16.0 / 3.0 * nb ** 3
    if kern.startswith("k_tridiag"):
        return "alu64", 16.0 / 3.0 * nb ** 3
    if kern == "eigh_refine":  # two refinement steps + the cluster Rayleigh-Ritz: 10 FP64 n x n complex GEMMs
        return "alu64", 10 * 8.0 * nb ** 3
    if kern.startswith("k_plane_density") and tag in ("energy", "mix"):
        # inverse plane FFTs of the occupied orbitals: stick buffer read once, one partial plane per group
        # of 8 bands written (FP32 sums for FP32 orbitals, FP64 otherwise)
        nocc = s["nocc"]
        return "hbm", nocc * n3 * ncol * b + (nocc + 7) // 8 * ng * (4 if b == 8 else 8)
    if kern.startswith("k_chol"):
        return "alu64", 4.0 / 3.0 * nb ** 3 * 2
    return None, None


# DRAM bytes per launch from one ncu capture, valid only for the kernel source it was taken on
# (sha256 prefix of the file defining the kernel); otherwise the roofline's traffic is null.
TRAFFIC = {
    # k_plane_reg<float, 72, 72, 9>, one full 144-band launch: 84.24 MB read + 27.46 MB written
    "k_plane<f32>": (111695360, "paper_1702_04045_gb300/csrc/hpsi_passes_reg.cuh", "7cba8b0d0c9bce73"),
}


def traffic_of(kernel: str):
    import hashlib
    ent = TRAFFIC.get(kernel.partition(":")[2])
    if not ent:
        return None
    nbytes, path, digest = ent
    try:
        with open(os.path.join(ROOT, path), "rb") as f:
            cur = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    return nbytes if cur == digest else None


def tensor_peak():
    """Dense TF32 tensor peak: the measured bf16 GEMM rate times the nominal TF32/bf16 ratio (1.1/2.25)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)["bf16_tflops"] * 1.1 / 2.25, "measured bf16 x 1.1/2.25"
    except (OSError, KeyError):
        return 1900.0 * 1.1 / 2.25, "fallback bf16 x 1.1/2.25"


def hpsi_bytes(s, b):
    """Algorithmic bytes of one H psi batch over all bands (three stick-pruned passes, V once)."""
    return s["nb"] * (3 * s["npw"] * b + 4 * s["ncol"] * s["n3"] * b) + s["ngrid"] * b // 2


def _scf_until(ctx, opts, nat, tol, max_it, min_it=2, eig_tol=None):
    """SCF steps until |F^{n+1} - F^n| / atom < tol on two consecutive iterations (and, with eig_tol, the
    occupied eigenvalues moved by less than eig_tol in each), or max_it; returns (iterations, seconds on
    the device, last energy terms)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    prev, small, terms, eps_prev = None, 0, None, None
    for it in range(1, max_it + 1):
        terms, _ = ctx.scf_step(opts)
        e = terms["total"]
        ok = prev is not None and abs(e - prev) / nat < tol
        if eig_tol is not None:
            eps = ctx.eigenvalues()[0][: ctx.n_occ]
            ok = ok and eps_prev is not None and float(np.abs(eps - eps_prev).max()) < eig_tol
            eps_prev = eps
        small = small + 1 if ok else 0
        prev = e
        if small >= 2 and it >= min_it:
            break
    e1.record()
    torch.cuda.synchronize()
    return it, e0.elapsed_time(e1) / 1e3, terms


def _timed_steps(ctx, opts, k):
    """k SCF steps bracketed by CUDA events on torch's current stream (the library's stream): ms, energy."""
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    terms = None
    for _ in range(k):
        terms, _ = ctx.scf_step(opts)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), terms


def run_ours(args, rank, world, local, pg):
    import torch
    from paper_1702_04045_gb300 import inputs, paro
    torch.cuda.set_device(local)
    lat, pos, d, c = inputs.config_inputs(args.workload)
    nat = len(pos)
    ctx = paro.context_from_config(args.workload, args.precision)
    nb, npw = c["n_bands"], ctx.npw()
    c0 = inputs.start_vectors(nb, npw, c["seed_psi"] + 7919 * rank)
    ctx.set_orbitals(c0)
    opts = paro.ScfOptions(alg=args.alg, tol_per_atom=0.0, inner_rel_tol=0.25, inner_max_it=8)
    # 1. converge from the seeded start vectors (|dF|/atom < conv_tol twice); not timed as the metric
    n_conv, s_conv, _ = _scf_until(ctx, opts, nat, args.conv_tol, args.max_conv_iter)
    # 2. the metric: K converged iterations after W warm-up iterations, CUDA events, no instrumentation
    for _ in range(args.warmup):
        ctx.scf_step(opts)
    torch.cuda.synchronize()
    barrier(pg)
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    l0 = ctx.launch_count()
    ms, terms = _timed_steps(ctx, opts, args.steps)
    launches = ctx.launch_count() - l0
    clk = clocks.stop()
    barrier(pg)
    ms_max = max_over_ranks(pg, ms)
    # 3. the same iterations once more with the library's per-kernel CUDA events (roofline of each kernel)
    ctx.profile(True)
    ms_prof, _ = _timed_steps(ctx, opts, args.steps)
    prof = {n: ctx.profile_read(n) for n in ctx.profile_names()}
    ctx.profile(False)

    # 4. end to end through the C ABI with host buffers: restore the state from pinned host memory,
    # run the iteration, read the energy back
    psi_h = torch.from_numpy(ctx.get_orbitals()).pin_memory()
    eps_h = ctx.eigenvalues()[0].copy()
    torch.cuda.synchronize()
    barrier(pg)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.set_state(psi_h, eps_h)
        e_host, _ = ctx.scf_step(opts)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(pg, time.perf_counter() - t0)

    # 5. mixed against FP64 at the converged state (rank 0, N = 1): the mixed run goes on to its fixed
    # point with Algorithm 3 (MParO II, the same fixed point, far fewer iterations), an FP64 context starts
    # from that state and iterates to its own fixed point; per-eigenvalue and per-atom errors of the
    # mixed result, and the FP64 iteration time at the converged state (CUDA events, nine iterations:
    # one whole cycle of eight carried and one direct H application)
    cmp = None
    if not args.no_fp64 and args.precision != "fp64" and world == 1:
        cmp = compare_fp64(ctx, args, nat, opts)

    s = shapes(ctx)
    totals = {n: t for n, (k, t) in prof.items()}
    dom = max(totals, key=totals.get) if totals else None
    hbm, hbm_src = peaks()

    def roof_of(cand):
        kind, work = launch_work(cand, s)
        if kind is None:
            return None
        cnt, tot = prof[cand]
        avg_s = tot / cnt / 1e3
        common = {"kernel": cand, "avg_launch_ms": avg_s * 1e3, "share_of_step": tot / ms_prof,
                  "traffic": traffic_of(cand)}
        if kind == "hbm":
            ach = work / avg_s / 1e9
            return dict(common, bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                        peak_source=hbm_src, bytes_per_launch=work)
        if kind == "tensor":
            tp, tsrc = tensor_peak()
            ach = 3 * work / avg_s / 1e12
            return dict(common, bound="tensor", achieved=ach, peak=tp, unit="TFLOP/s", frac=ach / tp,
                        peak_source=tsrc, flops_per_launch=work,
                        note="3xTF32: three TF32 MMAs per real product; achieved counts all three")
        peak = FP64_TFLOPS if kind == "alu64" else FP32_TFLOPS
        ach = work / avg_s / 1e12
        return dict(common, bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                    peak_source=FP64_SOURCE if kind == "alu64" else FP32_SOURCE, flops_per_launch=work)

    # the dominant kernel: the largest total over all its call sites; its roofline from the call site with
    # a fixed per-launch shape (e.g. the H psi plane pass runs masked to the active orbitals inside the
    # inner solves, on every orbital in the Rayleigh-Ritz apply)
    by_kernel = {}
    for name, t in totals.items():
        by_kernel.setdefault(name.partition(":")[2] or name, []).append((t, name))
    roof = None
    for kern in sorted(by_kernel, key=lambda k: -sum(t for t, _ in by_kernel[k])):
        for _, cand in sorted(by_kernel[kern], reverse=True):
            roof = roof_of(cand)
            if roof:
                roof["kernel_share_all_sites"] = sum(t for t, _ in by_kernel[kern]) / ms_prof
                break
        if roof:
            break
    roof_tensor = {k: roof_of(k) for k in ("pcg:k_gemm_cn_tcb", "pcg:k_gemm_wx_tcb") if k in prof} or None
    if roof_tensor:  # the same launches against HBM: the projector image (hi + lo, 16 bytes per complex entry)
        # and the orbital rows read; the update also reads and writes H x
        for k, r in roof_tensor.items():
            if r:
                nbytes = 16 * s["nproj"] * s["npw"] + 8 * s["nb"] * s["npw"] * (1 if "cn" in k else 2)
                r["bytes_per_launch"] = nbytes
                r["hbm_gbs"] = nbytes / (r["avg_launch_ms"] / 1e3) / 1e9
                r["hbm_frac"] = r["hbm_gbs"] / hbm
    bsz = 16 if args.precision == "fp64" else 8
    tag = "f64" if bsz == 16 else "f32"
    hpsi = None
    for site in ("rr", "pcg"):
        pas = [f"{site}:k_zpass_inv<{tag}>", f"{site}:k_plane<{tag}>", f"{site}:k_zpass_fwd<{tag}>"]
        if site == "rr" and all(p in prof for p in pas):
            t_h = sum(prof[p][1] / prof[p][0] for p in pas) / 1e3
            hpsi = {"gbs": hpsi_bytes(s, bsz) / t_h / 1e9, "ms_per_batch": t_h * 1e3, "bands": s["nb"],
                    "frac_of_hbm": hpsi_bytes(s, bsz) / t_h / 1e9 / hbm, "bytes_per_batch": hpsi_bytes(s, bsz),
                    "site": "Rayleigh-Ritz apply (all bands)"}
    out = {
        "metric": METRIC, "value": world * args.steps / (ms_max / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "precision": args.precision, "algorithm": args.alg,
                   "inner_pcg": "rel_tol 0.25, max 8 steps", "parallelism": f"replicas x{world}",
                   "state": f"converged: timed after |dF|/atom < {args.conv_tol:g} twice (+{args.warmup} warm-up)",
                   "smearing_kT_ha": c.get("kT", 0.0),
                   "l2": "working set per iteration > L2 (no flush)"},
        "e2e": {"value": world * args.steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": nb * npw * 16 + nb * 8, "d2h_bytes_per_step": 8 * 8},
        "gpu_launches": launches,
        "launches_before_timed": l0,  # every kernel of this process so far (a profiler's launch-skip count)
        "convergence": {"precision": args.precision, "algorithm": args.alg, "tol_per_atom": args.conv_tol,
                        "iterations": n_conv, "seconds": s_conv, "ms_per_iteration": s_conv / n_conv * 1e3},
        "roofline": roof,
        "roofline_tensor_projector": roof_tensor,
        "hpsi": hpsi,
        "mixed_vs_fp64": cmp,
        "fp64_ms_per_step": cmp["fp64_ms_per_step"] if cmp else None,
        "speedup_vs_fp64": (cmp["fp64_ms_per_step"] / (ms_max / args.steps)) if cmp else None,
        "dominant_kernel": dom,
        "profiled_ms_per_step": ms_prof / args.steps,
        "kernel_ms": {k: round(v[1], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
        "kernel_calls": {k: v[0] for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
        "clocks": clk,
        "energy_last_step": terms["total"] if terms else None,
    }
    ctx.close()
    return out


def compare_fp64(ctx, args, nat, opts):
    """Mixed vs FP64 at the SCF fixed point of the same cell (see run_ours, step 5)."""
    import torch
    from paper_1702_04045_gb300 import paro
    o3 = paro.ScfOptions(alg=3, tol_per_atom=0.0, inner_rel_tol=0.25, inner_max_it=8)
    # the mixed run stops once its occupied eigenvalues move by less than 1e-6 Ha (the FP32 noise floor
    # of this cell is ~3e-7) on two consecutive iterations, after at least 60
    n_mix, s_mix, t_mix = _scf_until(ctx, o3, nat, 1e30, args.max_fix_iter, min_it=60, eig_tol=1e-6)
    eps_mix = ctx.eigenvalues()[0]
    f_mix, mu_mix, _ = ctx.occupations()
    psi = ctx.get_orbitals(device=True)
    rho = ctx.density()
    ctx64 = paro.context_from_config(args.workload, "fp64")
    ctx64.set_density(rho)
    ctx64.set_orbitals(psi)
    # eigenvalues follow the density error at first order (the energy at second): the FP64 run also waits
    # for its occupied eigenvalues to stand still to 1e-9 Ha
    n64, s64, t64 = _scf_until(ctx64, o3, nat, args.fix_tol, args.max_fix_iter, min_it=10, eig_tol=1e-9)
    eps64 = ctx64.eigenvalues()[0]
    f64, mu64, _ = ctx64.occupations()
    occ = f64[0] > 1e-3  # bands that carry charge
    # orthonormality of the mixed orbitals as stored (FP32 rows widened to FP64)
    g = psi.conj() @ psi.T
    orth = float((g - torch.eye(g.shape[0], dtype=g.dtype, device=g.device)).abs().max())
    # FP64 iteration time at its converged state: one whole 9-iteration cycle of carried / direct H
    ms64, _ = _timed_steps(ctx64, opts, 9)
    ctx64.close()
    return {"reference": "FP64 GPU run from the mixed fixed point to its own (Algorithm 3, MParO II)",
            "tol_per_atom": args.fix_tol, "fp64_eig_tol_ha": 1e-9, "mixed_eig_tol_ha": 1e-6,
            "mixed_iterations_alg3": n_mix, "fp64_iterations_alg3": n64,
            "mixed_s_alg3": s_mix, "fp64_s_alg3": s64,
            "max_eig_err_occupied_ha": float(np.abs(eps_mix[occ] - eps64[occ]).max()),
            "mean_eig_err_occupied_ha": float((eps_mix[occ] - eps64[occ]).mean()),
            "worst_bands": [[int(i), float(eps_mix[i] - eps64[i])]
                            for i in np.argsort(-np.abs(np.where(occ, eps_mix - eps64, 0.0)))[:4]],
            "e_per_atom_err_ha": abs(t_mix["total"] - t64["total"]) / nat,
            "fermi_level_err_ha": abs(mu_mix - mu64),
            "mixed_orthonormality_err": orth,
            "within_1e-6_ha": bool(np.abs(eps_mix[occ] - eps64[occ]).max() < 1e-6
                                   and abs(t_mix["total"] - t64["total"]) / nat < 1e-6),
            "fp64_ms_per_step": ms64 / 9, "fp64_alg": args.alg}


def run_adjoint(nb=1088, calls=2):
    """Adjoint of H psi on the 512-atom cell (137059 plane waves, 128^3 grid, 2048 KB projectors), FP32
    inputs: ms per call over all three outputs (dL/dpsi, dL/dV, dL/dR) with CUDA events."""
    import torch
    from paper_1702_04045_gb300 import paro
    ctx = paro.context_from_config("si512", "mixed")
    npw = ctx.npw()
    g = torch.Generator(device="cuda").manual_seed(5124)
    psi = torch.randn((nb, npw), dtype=torch.complex64, device="cuda", generator=g)
    w = torch.randn((nb, npw), dtype=torch.complex64, device="cuda", generator=g)
    ctx.apply_h_adjoint(psi, w)
    torch.cuda.synchronize()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(calls):
        ctx.apply_h_adjoint(psi, w)
    e1.record()
    torch.cuda.synchronize()
    prof = {n: ctx.profile_read(n) for n in ctx.profile_names()}
    ctx.profile(False)
    ms = e0.elapsed_time(e1) / calls
    top = sorted(prof.items(), key=lambda kv: -kv[1][1])[:6]
    out = {"workload": "512-atom diamond cell a=41.04 Bohr, Ecut 12 Ha (137059 PW, 128^3 grid), 2048 KB "
                       "projectors, FP32 inputs", "bands": nb, "ms_per_call": ms,
           "outputs": "dL/dpsi, dL/dV_eff(r), dL/dR (512 atoms)",
           "kernel_ms_per_call": {k: round(v[1] / calls, 3) for k, v in top}}
    ctx.close()
    return out


def run_gamma(args):
    """The same cell and converged-iteration timing with the Gamma-point real-wavefunction mode (two real
    orbitals per packed complex H application and density transform): its own convergence from the seeded
    start vectors, then K timed iterations (CUDA events)."""
    import torch
    from paper_1702_04045_gb300 import inputs, paro
    lat, pos, d, c = inputs.config_inputs(args.workload)
    ctx = paro.context_from_config(args.workload, args.precision)
    ctx.set_gamma_real(True)
    ctx.set_orbitals(inputs.start_vectors(c["n_bands"], ctx.npw(), c["seed_psi"]))
    opts = paro.ScfOptions(alg=args.alg, tol_per_atom=0.0, inner_rel_tol=0.25, inner_max_it=8)
    n_conv, s_conv, _ = _scf_until(ctx, opts, len(pos), args.conv_tol, args.max_conv_iter)
    for _ in range(args.warmup):
        ctx.scf_step(opts)
    ms, terms = _timed_steps(ctx, opts, args.steps)
    out = {"mode": "Gamma-point real wavefunctions (paro_set_gamma_real)", "ms_per_step": ms / args.steps,
           "iterations_to_converge": n_conv, "seconds_to_converge": s_conv, "energy_last_step": terms["total"]}
    ctx.close()
    return out


def run_hpsi512(nb=1088, calls=3):
    """Forward H psi batch of the 512-atom cell (137059 plane waves, 128^3 grid, 2048 KB projectors), all
    1088 bands in FP32 through paro_apply_h: ms per batch with CUDA events, the three FFT passes' share
    (the library's per-kernel events) and their algorithmic GB/s (3 N_pw b + 4 N_col N_3 b per band, plus V)."""
    import torch
    from paper_1702_04045_gb300 import paro
    ctx = paro.context_from_config("si512", "mixed")
    npw = ctx.npw()
    g = torch.Generator(device="cuda").manual_seed(5125)
    psi = torch.randn((nb, npw), dtype=torch.complex64, device="cuda", generator=g)
    out = torch.empty_like(psi)
    ctx.apply_h(psi, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(calls):
        ctx.apply_h(psi, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / calls
    ctx.profile(True)
    for _ in range(calls):
        ctx.apply_h(psi, out=out)
    prof = {n: ctx.profile_read(n) for n in ctx.profile_names()}
    ctx.profile(False)
    s = shapes(ctx)
    s["nb"] = nb
    fft = [k for k in prof if k.startswith(("k_zpass_inv", "k_plane", "k_zpass_fwd"))]
    t_fft = sum(prof[k][1] for k in fft) / calls / 1e3
    byt = hpsi_bytes(s, 8)
    hbm, src = peaks()
    res = {"workload": "512-atom diamond cell a=41.04 Bohr, Ecut 12 Ha (137059 PW, 128^3 grid), 1088 bands, "
                       "2048 KB projectors, FP32", "ms_per_batch": ms,
           "fft_passes_ms": t_fft * 1e3, "fft_passes_gbs": byt / t_fft / 1e9, "fft_passes_frac_of_hbm": byt / t_fft / 1e9 / hbm,
           "bytes_per_batch": byt, "peak_source": src,
           "kernel_ms_per_batch": {k: round(v[1] / calls, 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}}
    ctx.close()
    return res


def run_batched(name, steps=10, warmup=3, ref_steps=3):
    """Batched ParO (one persistent H psi launch over all orbitals, one CUDA graph per step) on a workload
    of uneven problems, mixed precision, against the per-context calls on the same problems. Each step
    synchronises, so host wall time brackets it."""
    import torch
    from paper_1702_04045_gb300 import inputs, paro
    cells = inputs.batch_inputs(name)
    ctxs = []
    for c in cells:
        ctx = paro.Context(c["lat"], c["pos"], c["ecut"], c["n_bands"], c["n_occ"], "mixed", kpts=c["kpts"],
                           kweights=c["kweights"])
        ctx.set_local_pp(**inputs.LOCAL_PP)
        for ik in range(len(c["kpts"])):
            ctx.set_orbitals(inputs.start_vectors(c["n_bands"], ctx.npw(ik), c["seeds"][ik]), ik)
        ctxs.append(ctx)
    b = paro.Batch(ctxs)
    for _ in range(warmup):
        b.step(0.25, 8)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        r = b.step(0.25, 8)
    t_b = (time.perf_counter() - t0) / steps
    # one fused H psi over every orbital of every problem
    psis = [ctxs[i].get_orbitals(k, device=True).to(torch.complex64) for i, k in b.problems]
    b.apply_h(psis)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        b.apply_h(psis)
    e1.record()
    torch.cuda.synchronize()
    t_h = e0.elapsed_time(e1) / 5
    info = b.info()
    tun = b.tuning()
    best = tun[int(np.argmin(tun[:, 4]))]
    coop = tun[tun[:, 0] == 1]
    for c in ctxs:
        c.step(1, 0.25, 8)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ref_steps):
        for c in ctxs:
            c.step(1, 0.25, 8)
    t_c = (time.perf_counter() - t0) / ref_steps
    npw = [ctxs[i].npw(k) for i, k in b.problems]
    out = {"workload": name, "problems": info["problems"], "orbitals": info["items"],
           "npw_range": [min(npw), max(npw)], "precision": "mixed",
           "ms_per_step_batched": t_b * 1e3, "ms_per_step_per_context": t_c * 1e3, "speedup": t_c / t_b,
           "hpsi_ms_all_orbitals": t_h,
           "hpsi_kernel": {"launches_per_apply": info["launches_per_apply"], "grid": info["grid"],
                           "sticks_per_unit": int(best[2]), "plane_points_per_unit": int(best[3]),
                           "autotuned_ms": float(best[4]), "candidates": int(len(tun)),
                           "best_cooperative_ms": float(coop[:, 4].min()) if len(coop) else None},
           "kernels_per_step": info["kernels_per_step"], "max_resid_after": r}
    b.close()
    for c in ctxs:
        c.close()
    return out


def cpu_sample(args, steps=1, warmup=0):
    """The FP64 CPU oracle on this host: seconds per ParO-SCF iteration of the same cell."""
    from oracle import scf
    from paper_1702_04045_gb300 import inputs
    lat, pos, d, c = inputs.config_inputs(args.workload)
    sys_ = scf.ScfSystem(lat, pos, c["ecut"], c["n_bands"], c["n_occ"], inputs.LOCAL_PP, d, inputs.KB_RC,
                         kT=c.get("kT", 0.0))
    c0 = inputs.start_vectors(c["n_bands"], sys_.bases[0].npw, c["seed_psi"])
    times = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        try:
            scf.paro_scf(sys_, [c0], tol=0.0, max_iter=1)
        except RuntimeError:
            pass
        if i >= warmup:
            times.append(time.perf_counter() - t0)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return times, cores


def run_reference(args, rank, world, pg):
    if rank != 0:
        return None
    times, cores = cpu_sample(args, steps=args.steps, warmup=args.warmup)
    v = len(times) / sum(times)
    sample = ("one FP64 oracle ParO-SCF iteration per step (NumPy; includes the start-up Rayleigh-Ritz of "
              "the seeded start vectors)")
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD_DESC, "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--alg", type=int, default=1, choices=[1, 2])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-hpsi512", action="store_true")
    ap.add_argument("--no-gamma", action="store_true")
    ap.add_argument("--conv-tol", type=float, default=1e-6, help="|dF|/atom before the timed region")
    ap.add_argument("--max-conv-iter", type=int, default=4000)
    ap.add_argument("--fix-tol", type=float, default=1e-9, help="|dF|/atom of the mixed-vs-FP64 fixed points")
    ap.add_argument("--max-fix-iter", type=int, default=120)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank, world, local, pg = dist_setup()
    if args.impl == "reference":
        out = run_reference(args, rank, world, pg)
        if rank == 0:
            print(json.dumps(out))
        return
    out = run_ours(args, rank, world, local, pg)
    if rank == 0 and world == 1 and not args.no_gamma:
        out["gamma_real"] = run_gamma(args)
        out["gamma_real"]["speedup_vs_complex"] = out["ms_per_step"] / out["gamma_real"]["ms_per_step"]
    if rank == 0 and world == 1 and not args.no_hpsi512:
        out["hpsi_512"] = run_hpsi512()
    if rank == 0 and world == 1 and not args.no_adjoint:
        out["adjoint_512"] = run_adjoint()
    if rank == 0 and world == 1 and not args.no_batched:
        out["batched"] = [run_batched("si8_mp27"), run_batched("cells64")]
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            times, cores = cpu_sample(args)
            out["cpu_baseline"] = {"value": 1.0 / times[0], "unit": UNIT, "cores": cores, "kind": "oracle",
                                   "sample": "one FP64 oracle ParO-SCF iteration of the same cell on the host "
                                             "cores (NumPy FFT single-threaded, BLAS threads = cores; includes "
                                             "the start-up Rayleigh-Ritz)"}
        print(json.dumps(out))


if __name__ == "__main__":
    main()
