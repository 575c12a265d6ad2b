#!/usr/bin/env python
"""Benchmark of the LR-TDDFT response path on one GB300 (or N, one process per GPU).

Workload: fcc Al, 1 atom, 12^3 k-mesh (time-reversal-symmetric, shifted by -q/2), 120 bands
(16 Ha cut-off), T = 10 eV, 8 q with |q| in [0.5, 2.5] 1/A along x, 59 response G-vectors,
1024 frequencies on [-40, 120] eV, eta = 0.5 eV, RPA + ALDA kernel.  A step is the whole
response path for all 8 q: pair densities, the chi0 contraction (split precision FP16x3 by
default), the FP64 Dyson solve, S(q,w), F(q,tau) on 64 tau in [0, beta/2] with its metrics,
and the attenuation of narrow-band fluctuations.  The ground state (eigensolves) is set up
once, outside the timed region.

Reported value: chi0 complex MACs per second over the step, counting the full Adler-Wiser
sum N_G^2 N_w N_p per q (N_p = N_k N_b^2), all ranks together.  Every operand is larger than
the 129 MB L2 (pair densities: 11.8 GB per q), so no flush is needed between steps.

--impl reference times the FP64 CPU oracle (tests' reference implementation) on a bounded
sample of the same workload on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import re
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "chi0 complex MAC/s (split-precision chi0, FP64 Dyson/S/F, whole response path)"
UNIT = "cMAC/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default="fp16x3", choices=["fp16x3", "bf16x3", "fp64"])
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64-form slice, the accuracy check and the CPU baseline")
    ap.add_argument("--nq", type=int, default=0, help="use the first nq q vectors (0 = all)")
    ap.add_argument("--kmesh", type=int, default=0,
                    help="k mesh n^3 instead of 12^3 (small cases for profiler captures)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--autotune", action="store_true", help="let the library time its kernel variants")
    ap.add_argument("--variant", type=int, default=-1, help="force a tensor-kernel variant (0, 1)")
    ap.add_argument("--unit-stages", type=int, default=0, help="force the stages per work unit")
    ap.add_argument("--fine-accum", action="store_true",
                    help="flush the FP32 tensor-core accumulators every 32 stages instead of 64")
    ap.add_argument("--workload", default="al1",
                    choices=["al1", "al4_adjoint", "al64_slice", "al32_k1", "al1_q_fp64"],
                    help="al1: the timed 8-q workload (default); the others measure the other "
                         "configurations once and print one JSON line each (al1_q_fp64: the "
                         "largest |q| of the timed workload at full size in the FP64 and the "
                         "split form)")
    return ap.parse_args()


def workload(nq=0, kmesh=0):
    from paper_2510_01875_gb300 import workloads as W
    wl = W.al1_fcc_k12_b120()
    if nq:
        wl = wl.replace(q=wl.q[:nq], nG=wl.nG[:nq])
    if kmesh:
        wl = wl.replace(kmesh=(kmesh, kmesh, kmesh), name=wl.name.replace("k12", f"k{kmesh}"))
    return wl


def cmac_per_q(ctx, wl):
    return float(int(wl.nG[0]) ** 2) * wl.nw * float(ctx.nk) * ctx.nb * ctx.nb


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(busy)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------- distributed plumbing
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(pg, value):
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if pg.get_backend() == "nccl" else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, value):
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if pg.get_backend() == "nccl" else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


# ---------------------------------------------------------------- our implementation
def run_ours(args, world, rank, local, pg):
    import torch
    from paper_2510_01875_gb300 import binding, build
    build.build()
    binding.load()
    torch.cuda.set_device(local)
    wl = workload(args.nq, args.kmesh)
    t0 = time.time()
    ctx = binding.Context(wl, args.precision, device=local)
    setup_s = time.time() - t0
    if args.precision != "fp64":
        ctx.set_tuning(auto=args.autotune, variant=args.variant, unit_stages=args.unit_stages,
                       fine_accum=args.fine_accum)
    dev = torch.device("cuda", local)
    ntau = wl.ntau
    tau = torch.linspace(0.0, 0.5 / wl.T, ntau, dtype=torch.float64, device=dev)
    F = torch.zeros((wl.nq, ntau), dtype=torch.float64, device=dev)
    M = torch.zeros((wl.nq, 5), dtype=torch.float64, device=dev)
    S = torch.zeros((wl.nq, wl.nw), dtype=torch.float64, device=dev)
    params = binding.atten_params()

    def step():
        # every call on the legacy default stream (0), which torch's events also use
        ctx.chi0_assemble()
        ctx.dyson_solve()
        ctx.dsf_device(S.data_ptr())
        ctx.itcf_device(ntau, tau.data_ptr(), F.data_ptr(), M.data_ptr())
        ctx.attenuate(params)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ctx.profile(True)
    barrier(pg)
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    barrier(pg)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    prof = ctx.profile_read()
    ctx.profile(False)
    ms_max = max_over_ranks(pg, ms)
    cmac_step = cmac_per_q(ctx, wl) * wl.nq
    value = sum_over_ranks(pg, cmac_step) / (ms_max / 1e3)

    # roofline of the dominant kernel (the chi0 contraction)
    peaks, src = measured_peaks()
    if args.precision == "fp64":
        bound, unit = "fp64", "TFLOP/s"
        flops_per_cmac = 4.0
        peak = max(binding.measure_fp64(local), fp64_peak()["tflops"])
        peak_note = "measured: the larger of an FP64 FMA loop (lrtddft_measure_fp64) and cuBLAS DGEMM"
    else:
        bound, unit = "tensor", "TFLOP/s"
        flops_per_cmac = 12.0      # 2 real MACs per complex MAC (Hermitian split) x 3 products
        peak = peaks["bf16_tflops_sustained"]
        peak_note = f"bf16 dense sustained, {src} (fp16 runs at the bf16 rate)"
    chi0_ms = prof["chi0_ms"] / max(prof["chi0_launches"], 1)
    chi0_tflops = flops_per_cmac * prof["chi0_cmac"] / (prof["chi0_ms"] / 1e3) / 1e12
    roofline = {"bound": bound, "achieved": chi0_tflops, "peak": peak, "unit": unit,
                "frac": chi0_tflops / peak,
                # one launch covers every q of a chi0_assemble call when they fit together
                "traffic": profiled_traffic(args.precision, ctx.nk * ctx.nb * ctx.nb * wl.nq * args.steps
                                            / max(prof["chi0_launches"], 1)),
                "kernel": "chi0_tc_kernel" if args.precision != "fp64" else "chi0_fp64_kernel",
                "launch_ms": chi0_ms, "peak_source": peak_note,
                "chi0_launches_per_step": prof["chi0_launches"] / args.steps,
                "kernel_variant_and_unit_stages": list(ctx.get_tuning()) if args.precision != "fp64" else None,
                "pair_density_ms_per_launch": prof["rho_ms"] / max(prof["rho_launches"], 1),
                "chi0_share_of_step": prof["chi0_ms"] / (ms * args.steps)}

    print(json.dumps({"progress": "device-timed", "ms_per_step": ms_max, "value": value,
                      "roofline": roofline, "launches": prof["launches"], "clocks": clk,
                      "setup_s": setup_s}), file=sys.stderr, flush=True)

    # end to end through the C ABI with host buffers: per step the orbitals, eigenvalues and
    # occupations of every q go host -> device, and S, F, the metrics and S_p come back
    try:
        e2e = (run_e2e(ctx, wl, args, cmac_step, pg, world) if not args.no_e2e
               else {"value": None, "unit": UNIT, "skipped": "--no-e2e"})
    except Exception as exc:  # reported, not hidden: the line carries the failure
        e2e = {"value": None, "unit": UNIT, "error": repr(exc)}
    print(json.dumps({"progress": "e2e", "e2e": e2e}), file=sys.stderr, flush=True)

    extras = {}
    if not args.no_extras and rank == 0:
        try:
            extras = run_extras(args, ctx, wl, S.cpu().numpy(), F.cpu().numpy())
        except Exception as exc:
            extras = {"extras_error": repr(exc)}
    ctx.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f16x3/f32-accumulate chi0, f64 elsewhere" if args.precision == "fp16x3"
            else ("bf16x3/f32-accumulate chi0, f64 elsewhere" if args.precision == "bf16x3" else "f64"),
            "data": "synthetic (seeded empty-core Al, no external data)",
            "config": {"workload": wl.name, "precision": args.precision, "nq": wl.nq,
                       "nk": ctx.nk, "nbands": ctx.nb, "nG": int(wl.nG[0]), "nw": wl.nw,
                       "np_per_q": ctx.nk * ctx.nb * ctx.nb, "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (pair densities %.2f GB per q)" % (
                           ctx.nk * ctx.nb * ctx.nb * int(wl.nG[0])
                           * (16 if args.precision == "fp64" else 8) / 1e9)},
            "q_spectra_per_s": sum_over_ranks(None, wl.nq * world) / (ms_max / 1e3),
            "setup_s": setup_s,
            # setup = one dense eigensolve per k point of both meshes of every q (+ refinement)
            "setup_ms_per_eigensolve": 1e3 * setup_s / (2 * ctx.nk * wl.nq),
            "roofline": roofline,
            "e2e": e2e,
            "gpu_launches": prof["launches"],
            "clocks": clk,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)


def chi0_kernel_digest(path):
    """sha256 of the contraction kernel's source (the text from its template header to the unpack
    kernel that follows it), so that host-side edits of the file keep a capture valid."""
    import hashlib
    text = open(path, "rb").read()
    a = text.find(b"template <bool BF, int NS, int NSR, bool ME>")
    b = text.find(b"// chi0[i][G][G'] from the FP64 sums", a)
    return hashlib.sha256(text[a:b] if a >= 0 and b > a else text).hexdigest()


def profiled_traffic(precision, np_per_q):
    """DRAM bytes per contraction launch from the committed ncu summary of the kernel
    (dram__bytes_read.sum + dram__bytes_write.sum on a 4^3-k case, per pair, scaled by this
    launch's pair count), or None when the kernel source has changed since the capture or the
    precision was not the profiled one."""
    import glob
    if precision != "fp16x3":
        return None
    here = os.path.dirname(os.path.abspath(__file__))
    digest = chi0_kernel_digest(os.path.join(here, "paper_2510_01875_gb300", "csrc", "chi0_tc.cu"))
    for path in sorted(glob.glob(os.path.join(here, "profiles", "chi0_tc_kernel_*.md"))):
        text = open(path).read()
        m = re.search(r"sha256 prefix `([0-9a-f]+)`", text)
        t = re.search(r"^traffic_bytes_per_pair: ([0-9.eE+]+)", text, re.M)
        if m and t and digest.startswith(m.group(1)):
            return float(t.group(1)) * float(np_per_q)
    return None


def run_e2e(ctx, wl, args, cmac_step, pg, world):
    import torch
    from paper_2510_01875_gb300 import binding
    nk, nb, npw = ctx.nk, ctx.nb, ctx.npw
    # pinned host copies of every q's inputs (taken once, outside the timed region)
    coeff = [torch.empty((2, nk, nb, npw, 2), dtype=torch.float64).pin_memory() for _ in range(wl.nq)]
    eps = [torch.empty((2, nk, nb), dtype=torch.float64).pin_memory() for _ in range(wl.nq)]
    occ = [torch.empty((2, nk, nb), dtype=torch.float64).pin_memory() for _ in range(wl.nq)]
    for iq in range(wl.nq):
        ctx.get_orbitals(iq, coeff[iq].numpy().view(np.complex128).reshape(2, nk, nb, npw))
        e, f, _, _ = ctx.get_ground_state(iq)
        eps[iq].numpy()[:] = e
        occ[iq].numpy()[:] = f
    tau = np.linspace(0.0, 0.5 / wl.T, wl.ntau)
    params = binding.atten_params()
    h2d = sum(c.numel() * 8 + e.numel() * 8 + o.numel() * 8 for c, e, o in zip(coeff, eps, occ))
    d2h = (wl.nq * wl.nw * 8) * 2 + wl.nq * wl.ntau * 8 + wl.nq * 5 * 8

    def upload():
        for iq in range(wl.nq):
            ctx.set_orbitals_async(iq, eps[iq].numpy(), coeff[iq].numpy().view(np.complex128).reshape(2, nk, nb, npw),
                                   occ[iq].numpy())

    def steps(n):
        # pipelined: the first step's inputs are copied before it, every later step's while the
        # step before it runs its contraction (the copies of all n steps are in the region)
        upload()
        for i in range(n):
            ctx.chi0_assemble()          # waits for this step's copies
            if i + 1 < n:
                upload()
            ctx.dyson_solve()
            S = ctx.dsf()
            F, m = ctx.itcf(tau)
            Sp, _ = ctx.attenuate(params)
        return S, F, m, Sp

    steps(1)
    torch.cuda.synchronize()
    barrier(pg)
    t0 = time.perf_counter()
    n = max(1, min(args.steps, 3))
    steps(n)
    torch.cuda.synchronize()
    barrier(pg)
    dt = (time.perf_counter() - t0) / n
    dt = max_over_ranks(pg, dt)
    return {"value": sum_over_ranks(pg, cmac_step) / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3, "steps": n,
            "pipeline": "orbitals of step i+1 copied from pinned host memory during step i's "
                        "contraction (lrtddft_set_orbitals_async); step 1's before it, in the region"}


def run_extras(args, ctx_main, wl, S_direct, F_direct):
    """The spectral chi0 engine on the timed workload against the direct engine's S and F of the
    timed steps; the FP64 form on a slice (1 q, 63 frequencies) beside the split form; the split
    form's error against the FP64 form at the timed workload's shape on a 4^3 k mesh; the eta
    scan; the CPU oracle."""
    from paper_2510_01875_gb300 import binding
    from paper_2510_01875_gb300 import workloads as W
    out = {}
    if args.precision != "fp64":
        out["spectral_engine"] = spectral_extra(ctx_main, wl, S_direct, F_direct)
    # slice: q[0], 63 frequencies from 15 eV; with the w = 0 column that S(q,0) needs they fill
    # one whole 64-frequency tile of the FP64 kernel, as the 1025 columns of the full grid
    # nearly fill 17
    j0 = int(np.searchsorted(wl.omega, W.ev(15.0)))
    sl = wl.replace(q=wl.q[:1], nG=wl.nG[:1], omega=wl.omega[j0:j0 + 63])
    forms = {}
    for prec in ("fp64", args.precision if args.precision != "fp64" else "fp16x3"):
        c = binding.Context(sl, prec)
        c.chi0_assemble()
        c.profile(True)
        c.chi0_assemble()
        p = c.profile_read()
        forms[prec] = {"chi0": c.get_chi0(0), "ms": p["chi0_ms"], "cmac": p["chi0_cmac"]}
        c.close()
    fp = forms["fp64"]
    sp = forms[[k for k in forms if k != "fp64"][0]]
    err = float(np.abs(sp["chi0"] - fp["chi0"]).max() / np.abs(fp["chi0"]).max())
    peak64 = fp64_peak()
    dfma = binding.measure_fp64(0)
    tf64 = 4.0 * fp["cmac"] / (fp["ms"] / 1e3) / 1e12
    peak = max(dfma, peak64["tflops"])
    out["fp64_form"] = {"value": fp["cmac"] / (fp["ms"] / 1e3), "unit": UNIT,
                        "chi0_tflops": tf64,
                        "roofline": {"bound": "fp64", "achieved": tf64, "peak": peak,
                                     "unit": "TFLOP/s", "frac": tf64 / peak,
                                     "peak_source": "measured: the larger of an FP64 FMA loop on "
                                                    "every SM (lrtddft_measure_fp64, %.3f) and cuBLAS "
                                                    "DGEMM (%.3f)" % (dfma, peak64["tflops"])},
                        "dgemm_peak": {"tflops": peak64["tflops"], "frac": tf64 / peak64["tflops"],
                                       "how": peak64["how"]},
                        "sample": f"1 q, 63 frequencies (15-25 eV) and w = 0, all {ctx_main.nk * ctx_main.nb ** 2:.3g} "
                                  "pairs; the rate is set by the pair sum, so it extrapolates "
                                  "linearly to the full workload",
                        "split_rate_same_slice": sp["cmac"] / (sp["ms"] / 1e3),
                        "split_vs_fp64_chi0_err": err}
    # accuracy of the split form against the FP64 form at the shape of the timed workload
    # (same cell, 120 bands, 59 G, 1024 frequencies, T, eta), smallest and largest |q|, on a
    # 4^3 k mesh (the FP64 form takes tens of seconds per q there)
    acc = wl.replace(kmesh=(4, 4, 4), q=wl.q[[0, wl.nq - 1]], nG=wl.nG[[0, wl.nq - 1]],
                     name=wl.name.replace("k12", "k4").replace(f"q{wl.nq}", "q2"))
    res = {}
    for prec in ("fp64", args.precision if args.precision != "fp64" else "fp16x3"):
        c = binding.Context(acc, prec)
        c.chi0_assemble()
        c.dyson_solve()
        S = c.dsf()
        F, m = c.itcf(np.linspace(0.0, 0.5 / acc.T, acc.ntau))
        res[prec] = ([c.get_chi0(i) for i in range(acc.nq)], S, F)
        c.close()
    a = res["fp64"]
    b = res[[k for k in res if k != "fp64"][0]]
    per_q = []
    for i in range(acc.nq):
        Sa, Sb = a[1][i], b[1][i]
        peaks = [j for j in range(1, acc.nw - 1) if Sa[j] > Sa[j - 1] and Sa[j] >= Sa[j + 1]
                 and Sa[j] > 0.1 * Sa.max()]
        per_q.append({
            "q_inv_bohr": float(np.linalg.norm(acc.q[i])),
            "chi0_maxnorm_rel": float(np.abs(b[0][i] - a[0][i]).max() / np.abs(a[0][i]).max()),
            "S_maxnorm_rel": float(np.abs(Sb - Sa).max() / np.abs(Sa).max()),
            "S_peak_rel": float(max(abs(Sb[j] / Sa[j] - 1) for j in peaks)) if peaks else None,
            "F_pointwise_rel": float(np.abs(b[2][i] / a[2][i] - 1).max())})
    out["split_accuracy"] = {
        "workload": acc.name, "against": "the library's FP64 form (parity-tested against the oracle)",
        "per_q": per_q,
        "F_pointwise_rel": max(x["F_pointwise_rel"] for x in per_q),
        "S_peak_rel": max(x["S_peak_rel"] or 0.0 for x in per_q),
        "bounds": {"F": 1e-5, "S_peaks": 1e-4}}
    out["eta_scan"] = eta_scan_extra(args, wl)
    out["cpu_baseline"] = cpu_baseline(wl)
    return out


def spectral_extra(ctx, wl, S_direct, F_direct, order=3, hdiv=16):
    """All q of the timed workload through the spectral chi0 engine (bin width eta/hdiv,
    Lagrange order 3; same context, orbitals and split precision), Dyson, S and F, device-timed
    after one untimed pass, against the direct engine's S and F of the timed steps."""
    tau = np.linspace(0.0, 0.5 / wl.T, wl.ntau)
    chi_direct = ctx.get_chi0(0)
    h = wl.eta / hdiv
    ctx.set_spectral(h, order)

    def fwd():
        ctx.chi0_assemble()
        ctx.dyson_solve()
        return ctx.dsf(), ctx.itcf(tau)[0]

    fwd()
    ms, (S, F) = _timed(fwd)
    chi = ctx.get_chi0(0)
    grids = [ctx.get_spectral_grid(i) for i in range(wl.nq)]
    ctx.set_spectral(0.0)
    pk = []
    for i in range(wl.nq):
        Sa = S_direct[i]
        pk += [abs(S[i][j] / Sa[j] - 1) for j in range(1, wl.nw - 1)
               if Sa[j] > Sa[j - 1] and Sa[j] >= Sa[j + 1] and Sa[j] > 0.1 * Sa.max()]
    return {"h_eV": h * 27.211386245988, "order": order, "bins_per_q": [int(g[1]) for g in grids],
            "ms_per_step": ms, "q_spectra_per_s": wl.nq / (ms / 1e3),
            "timed": "chi0_assemble (spectral) + dyson_solve + dsf + itcf for all q",
            "vs_direct_engine": {
                "chi0_maxnorm_rel_q0": float(np.abs(chi - chi_direct).max() / np.abs(chi_direct).max()),
                "S_maxnorm_rel": float(max(np.abs(S[i] - S_direct[i]).max() / np.abs(S_direct[i]).max()
                                           for i in range(wl.nq))),
                "S_peak_rel": float(max(pk)) if pk else None,
                "F_pointwise_rel": float(np.abs(F / F_direct - 1).max())}}


def eta_scan_extra(args, wl, n_eta=8, tol=5e-3):
    """The eta-convergence test (Sec. 2) on q[0] of the timed workload: n_eta broadenings in one
    assembly (the (eta, w) pairs as columns of one contraction launch) against n_eta separate
    single-eta passes, both through Dyson, S, F and the metrics; device-timed with CUDA events
    on the legacy stream the library uses."""
    import torch
    from paper_2510_01875_gb300 import binding
    from paper_2510_01875_gb300 import workloads as W
    one = wl.replace(q=wl.q[:1], nG=wl.nG[:1], name=wl.name.replace(f"q{wl.nq}", "q1"))
    etas = [W.ev(x) for x in np.linspace(0.1, 0.8, n_eta)]
    tau = np.linspace(0.0, 0.5 / one.T, one.ntau)
    prec = args.precision
    c = binding.Context(one, prec)

    def timed(fn):
        fn()                              # warm-up (plans, buffers)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    def batched():
        c.chi0_assemble()
        c.dyson_solve()
        return c.eta_scan(tau, tol)

    def separate():
        ms = []
        for e in etas:
            c.set_params(one.T, e)
            c.chi0_assemble()
            c.dyson_solve()
            ms.append(c.itcf(tau)[1][0])
        return np.array(ms)

    c.set_eta_list(etas)
    t_b, (_, m, ref) = timed(batched)
    t_s, m_sep = timed(separate)
    c.close()
    return {"workload": one.name, "precision": prec, "etas_eV": [float(x) for x in np.linspace(0.1, 0.8, n_eta)],
            "one_assembly_ms": t_b, "separate_ms": t_s, "speedup": t_s / t_b,
            "Ftilde_half_beta": [float(x) for x in m[0, :, 2]],
            "int_Ftilde": [float(x) for x in m[0, :, 3]],
            "metrics_max_rel_diff_vs_separate": float(np.abs(m[0] / m_sep - 1).max()),
            "tol": tol, "reference_eta_index": int(ref[0])}


def fp64_peak():
    """Measured FP64 rate of this GPU: cuBLAS DGEMM (torch.matmul in float64, 2 N^3 flops per
    product), best of 5 after a warm-up, CUDA events; the same method as the measured bf16
    peak.  The FP64 chi0 kernel is SIMT FP64 (4 flops per complex MAC of the Hermitian split)."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return {"tflops": 2.0 * n ** 3 / best / 1e12,
            "how": f"measured: torch.matmul float64 {n}^3 (cuBLAS DGEMM), best of 5, CUDA events"}


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(wl, seconds=15.0):
    """The FP64 oracle on a bounded sample of the workload: q[0], the first k point of the mesh
    (all N_b^2 = 14400 band pairs), N_G = 59, as many of the 1025 internal frequencies as fit in
    about `seconds`: pair densities, chi0, Dyson, S.  The eigensolves of the sample are not
    timed (the GPU's setup is not timed either).  Returns (cMAC/s, description)."""
    from oracle import crystal, occupations, response
    q = wl.q[0]
    gset = crystal.response_gset(wl.lattice, q, int(wl.nG[0]))
    kp, kqp = crystal.pair_meshes(wl.lattice, wl.kmesh, q, wl.kscheme)
    ek, Ck, bk = [], [], []
    for kv in (kp[0], kqp[0]):
        b = response.basis_for(wl, kv)
        e, C = crystal.eigenstates(wl.lattice, wl.positions, wl.Z, wl.r_c, kv, b, wl.nbands)
        ek.append(e)
        Ck.append(C)
        bk.append(b)
    mu = occupations.chemical_potential(ek[0][None, :], wl.T, wl.Z * wl.natoms, 1)
    f0, f1 = occupations.fermi(ek[0], mu, wl.T), occupations.fermi(ek[1], mu, wl.T)
    freqs, _ = response.internal_frequencies(wl.omega)
    om = crystal.volume(wl.lattice)
    K = response.kernel_diag(wl, q, gset)
    t0 = time.perf_counter()
    rho = response.pair_density(Ck[0], bk[0], Ck[1], bk[1], gset).reshape(-1, len(gset))
    d = (ek[0][:, None] - ek[1][None, :]).reshape(-1)
    df = (f0[:, None] - f1[None, :]).reshape(-1)
    t_rho = time.perf_counter() - t0
    # probe the per-frequency cost, then size the sample
    t0 = time.perf_counter()
    response.chi0(rho, d, df, freqs[:4], wl.eta, 1, om)
    per_w = (time.perf_counter() - t0) / 4
    nw = int(max(4, min(len(freqs), seconds / max(per_w, 1e-6))))
    t0 = time.perf_counter()
    chi0s = response.chi0(rho, d, df, freqs[:nw], wl.eta, 1, om)
    x = response.dyson_column0(chi0s, K)
    S = -x[:, 0].imag
    dt = time.perf_counter() - t0 + t_rho
    cmac = float(len(gset)) ** 2 * nw * len(d)
    desc = (f"{wl.name}: q[0], 1 of {wl.nk} k points ({len(d)} pairs), {len(gset)} G, {nw} of "
            f"{len(freqs)} frequencies; pair densities + chi0 + Dyson + S, FP64 numpy")
    return cmac / dt, desc, dt


def blas_threads():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count() or 1


def cpu_baseline(wl):
    v, desc, dt = oracle_sample(wl)
    return {"value": v, "unit": UNIT, "cores": blas_threads(), "kind": "oracle", "sample": desc,
            "seconds": dt}


def run_reference(args, world, rank, pg):
    if rank != 0:
        return
    wl = workload(args.nq, args.kmesh)
    for _ in range(args.warmup):
        oracle_sample(wl, seconds=2.0)
    vals, times, desc = [], [], ""
    for _ in range(args.steps):
        v, desc, dt = oracle_sample(wl, seconds=10.0)
        vals.append(v)
        times.append(dt)
    value = float(np.mean(vals))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded empty-core Al, no external data)",
            "config": {"workload": wl.name, "precision": "fp64 (CPU oracle)"},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- other configurations
def _split_vs_fp64(wl, prec, tau):
    """Split form against the FP64 form on the same workload: chi0 (max norm), S (max norm and
    peaks), F (pointwise)."""
    from paper_2510_01875_gb300 import binding
    res = {}
    for p in ("fp64", prec):
        c = binding.Context(wl, p)
        c.chi0_assemble()
        c.dyson_solve()
        S = c.dsf()
        F, _ = c.itcf(tau)
        res[p] = ([c.get_chi0(i) for i in range(wl.nq)], S, F)
        c.close()
    a, b = res["fp64"], res[prec]
    out = {"chi0_maxnorm_rel": max(float(np.abs(b[0][i] - a[0][i]).max() / np.abs(a[0][i]).max())
                                   for i in range(wl.nq)),
           "S_maxnorm_rel": float(max(np.abs(b[1][i] - a[1][i]).max() / np.abs(a[1][i]).max()
                                      for i in range(wl.nq))),
           "F_pointwise_rel": float(np.abs(b[2] / a[2] - 1).max())}
    pk = []
    for i in range(wl.nq):
        Sa = a[1][i]
        pk += [abs(b[1][i][j] / Sa[j] - 1) for j in range(1, wl.nw - 1)
               if Sa[j] > Sa[j - 1] and Sa[j] >= Sa[j + 1] and Sa[j] > 0.1 * Sa.max()]
    out["S_peak_rel"] = float(max(pk)) if pk else None
    return out


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    r = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), r


def run_workload(args):
    """One measurement of another configuration, one JSON line: setup time, the response path
    timed with CUDA events (after one untimed pass), the chi0 rate, and accuracy against the
    FP64 form on a reduced case of the same shape."""
    from paper_2510_01875_gb300 import binding, build
    from paper_2510_01875_gb300 import workloads as W
    build.build()
    binding.load()
    prec = args.precision if args.precision != "fp64" else "fp16x3"
    line = {"workload_kind": args.workload, "precision": prec}
    if args.workload == "al4_adjoint":
        wl = W.al4_cubic_k6_b200()
    elif args.workload == "al64_slice":
        full = W.al64_k2_b1600()
        wl = full.replace(q=full.q[:1], nG=full.nG[:1], name=full.name.replace("q48", "q1of48"))
    else:
        full = W.al32_k4_b400()
        wl = full.replace(kmesh=(1, 1, 1), name=full.name.replace("k4", "k1"))
    tau = np.linspace(0.0, 0.5 / wl.T, wl.ntau)
    t0 = time.time()
    c = binding.Context(wl, prec)
    line["setup_s"] = time.time() - t0
    line["setup_ms_per_eigensolve"] = 1e3 * line["setup_s"] / (2 * c.nk * wl.nq)
    line["workload"] = wl.name
    line.update({"nq": wl.nq, "nk": c.nk, "nbands": c.nb, "nG": [int(x) for x in wl.nG][:48],
                 "nw": wl.nw, "np_per_q": c.nk * c.nb * c.nb})

    def forward():
        c.chi0_assemble()
        c.dyson_solve()
        return c.itcf(tau)

    forward()
    c.profile(True)
    ms, _ = _timed(forward)
    prof = c.profile_read()
    cmac = sum(float(g) ** 2 for g in wl.nG) * wl.nw * c.nk * c.nb * c.nb
    line.update({"forward_ms": ms, "chi0_ms": prof["chi0_ms"], "chi0_launches": prof["chi0_launches"],
                 "pair_density_ms": prof["rho_ms"], "cmac_per_s": cmac / (ms / 1e3),
                 "chi0_tflops": 12.0 * cmac / (prof["chi0_ms"] / 1e3) / 1e12})
    if args.workload == "al4_adjoint":
        gms, (dS, dF) = _timed(lambda: c.jacobian(tau))
        line["gradient_ms"] = gms
        line["gradient"] = "dF(q, tau)/d(T, eta, A, B, C), 16 q x 64 tau, hand-written adjoint"
    else:
        ams, _ = _timed(lambda: c.attenuate(binding.atten_params()))
        line["attenuation_ms"] = ams
    c.close()
    # accuracy on a reduced case of the same shape
    if args.workload == "al4_adjoint":
        red = wl.replace(kmesh=(2, 2, 2), q=wl.q[[0, wl.nq - 1]], nG=wl.nG[[0, wl.nq - 1]],
                         name=wl.name.replace("k6", "k2"))
        acc = _split_vs_fp64(red, prec, tau)
        jac = {}
        for p in ("fp64", prec):
            cc = binding.Context(red, p)
            cc.chi0_assemble()
            cc.dyson_solve()
            jac[p] = cc.jacobian(tau)[1]
            cc.close()
        acc["gradient_maxnorm_rel_per_theta"] = [
            float(np.abs(jac[prec][..., j] - jac["fp64"][..., j]).max() / np.abs(jac["fp64"][..., j]).max())
            for j in range(5)]
        acc["reduced_case"] = red.name + " (against the FP64 form and the FP64 adjoint)"
    elif args.workload == "al64_slice":
        j0 = int(np.searchsorted(wl.omega, 0.0))
        red = wl.replace(omega=wl.omega[j0:j0 + 4], name=wl.name + "_4w")
        chi = {}
        for p in ("fp64", prec):
            cc = binding.Context(red, p)
            cc.chi0_assemble()
            chi[p] = cc.get_chi0(0)
            cc.close()
        acc = {"chi0_maxnorm_rel": float(np.abs(chi[prec] - chi["fp64"]).max() / np.abs(chi["fp64"]).max()),
               "reduced_case": red.name + " (4 frequencies, all pairs, against the FP64 form)"}
    else:
        i = int(np.argmin(wl.nG))
        red = wl.replace(q=wl.q[i:i + 1], nG=wl.nG[i:i + 1], name=wl.name + f"_q{i}")
        acc = _split_vs_fp64(red, prec, tau)
        acc["reduced_case"] = red.name + " (against the FP64 form)"
    line["accuracy"] = acc
    print(json.dumps(line), flush=True)


def run_full_q_fp64(args):
    """The largest |q| of the timed workload at its full size (12^3 k, 121 bands, 59 G, 1024
    frequencies) in the FP64 form and in the split form: the split form's error at exactly the
    timed configuration, and the FP64 form's rate and roofline on a whole q."""
    from paper_2510_01875_gb300 import binding, build
    build.build()
    binding.load()
    full = workload(0, 0)
    wl = full.replace(q=full.q[-1:], nG=full.nG[-1:], name=full.name.replace(f"q{full.nq}", "q1last"))
    tau = np.linspace(0.0, 0.5 / wl.T, wl.ntau)
    prec = args.precision if args.precision != "fp64" else "fp16x3"
    res = {}
    for p in ("fp64", prec):
        t0 = time.time()
        c = binding.Context(wl, p)
        setup = time.time() - t0
        c.profile(True)

        def fwd():
            c.chi0_assemble()
            c.dyson_solve()
            return c.dsf(), c.itcf(tau)[0]

        ms, (S, F) = _timed(fwd)
        pr = c.profile_read()
        res[p] = {"S": S[0], "F": F[0], "chi0": c.get_chi0(0), "ms": ms, "chi0_ms": pr["chi0_ms"],
                  "cmac": pr["chi0_cmac"], "setup_s": setup}
        c.close()
    a, b = res["fp64"], res[prec]
    Sa, Sb = a["S"], b["S"]
    peaks = [j for j in range(1, wl.nw - 1) if Sa[j] > Sa[j - 1] and Sa[j] >= Sa[j + 1] and Sa[j] > 0.1 * Sa.max()]
    tf64 = 4.0 * a["cmac"] / (a["chi0_ms"] / 1e3) / 1e12
    dfma = max(binding.measure_fp64(0), fp64_peak()["tflops"])
    line = {"workload_kind": "al1_q_fp64", "workload": wl.name, "precision": prec,
            "q_inv_bohr": float(np.linalg.norm(wl.q[0])),
            "fp64_form": {"forward_ms": a["ms"], "chi0_ms": a["chi0_ms"],
                          "cmac_per_s": a["cmac"] / (a["chi0_ms"] / 1e3), "chi0_tflops": tf64,
                          "roofline": {"bound": "fp64", "achieved": tf64, "peak": dfma, "unit": "TFLOP/s",
                                       "frac": tf64 / dfma,
                                       "peak_source": "measured: the larger of an FP64 FMA loop "
                                                      "(lrtddft_measure_fp64) and cuBLAS DGEMM"},
                          "setup_s": a["setup_s"]},
            "split_form": {"forward_ms": b["ms"], "chi0_ms": b["chi0_ms"],
                           "cmac_per_s": b["cmac"] / (b["chi0_ms"] / 1e3), "setup_s": b["setup_s"]},
            "split_vs_fp64": {
                "chi0_maxnorm_rel": float(np.abs(b["chi0"] - a["chi0"]).max() / np.abs(a["chi0"]).max()),
                "S_maxnorm_rel": float(np.abs(Sb - Sa).max() / np.abs(Sa).max()),
                "S_peak_rel": float(max(abs(Sb[j] / Sa[j] - 1) for j in peaks)) if peaks else None,
                "F_pointwise_rel": float(np.abs(b["F"] / a["F"] - 1).max()),
                "bounds": {"F": 1e-5, "S_peaks": 1e-4}}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "al1_q_fp64":
        run_full_q_fp64(args)
        return
    if args.workload != "al1":
        run_workload(args)
        return
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank, pg)
    else:
        run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
