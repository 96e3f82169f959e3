#!/usr/bin/env python
"""Benchmark of the screened periodic LRI exchange build on GB300.

One step = one full hfx_build (block norms, screen, staged contractions,
deterministic Sigma reduction, E_X) over the 64-atom Si-like supercell
(2x2x2 diamond, 13 NAOs / 60 ABFs per atom, C and D blocks within 16 bohr,
V within 20 bohr, theta = 1e-6) with its inputs resident in HBM.

value     canonical TFLOP/s = Algorithm 3 flop count of the build / device time
e2e       the same through the C ABI with host buffers: set C, V, D from host
          memory, build, copy every Sigma block back
roofline  the kernel with the most device time in the timed region
cpu_baseline  the CPU oracle on this host's cores, on a bounded sample of the
          same workload, extrapolated by surviving-term count

--impl reference times the CPU oracle alone (rank 0) on bounded samples.
Under torchrun each rank builds its own independent cell (weak scaling, no
collective on the data path; one all-reduce of the elapsed time).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HFX build s & TFLOP/s on 1 GB300, split-prec vs FP64 at max|ΔH|≤1e-8 Ha"
THETA = 1e-6
# FP64 on CUDA cores: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


# name: (supercell, cells per edge, seed, generator options).  The last two are
# the second workload: full-range Coulomb V out to 50 bohr, and a metallic D
# (polynomial decay) out to 24 bohr.
WORKLOADS = {"si64": ("2x2x2", 2, 2, {}), "si8": ("1x1x1", 1, 1, {}),
             "si512": ("4x4x4", 4, 3, {}),
             "si8_fullrange": ("1x1x1", 1, 5, {"cut_V": 50.0, "mu": 0.0}),
             "si8_metal": ("1x1x1", 1, 6, {"cut_D": 24.0, "d_decay": "power"})}


def workload(name: str, rank: int):
    import synth
    cells, ncell, seed, opts = WORKLOADS[name]
    return synth.make_workload(synth.si_diamond(ncell), seed=seed + 1000 * rank, name=name,
                               **opts)


def workload_desc(wl) -> str:
    cells, _, _, opts = WORKLOADS[wl.name]
    kind = ""
    if opts.get("mu") == 0.0:
        kind += ", full-range Coulomb V"
    if opts.get("d_decay") == "power":
        kind += ", metallic D (polynomial decay)"
    return (f"{wl.name}: Si-like diamond {cells} supercell, {wl.system.natoms} atoms, 13 NAO / "
            f"60 ABF per atom, C <= {wl.cut_C:g} bohr, D <= {wl.cut_D:g} bohr, "
            f"V <= {wl.cut_V:g} bohr{kind}, theta = {THETA:g}, seed {wl.seed}")


# dram__bytes_read.sum + dram__bytes_write.sum of one k_zc<6,16,4,8,1> launch on the
# 8-atom cell (30.71 GB + 0.52 GB) over its issued bf16 tensor flops (14.99 TFLOP),
# captured from hfx_zc.cu with this sha256 prefix (see profiles/k_zc_split_si8.md)
ZC_BYTES_PER_TENSOR_FLOP = (30.712555e9 + 0.524244e9) / 14.988985761792e12
ZC_CAPTURED_SHA = "1cef9b93b0076611"


def zc_traffic(tensor_flops_per_launch):
    import hashlib
    src = os.path.join(ROOT, "paper_2009_12505_gb300", "csrc", "hfx_zc.cu")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if sha != ZC_CAPTURED_SHA:
        return None
    return ZC_BYTES_PER_TENSOR_FLOP * tensor_flops_per_launch


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(wl, theta: float, seconds: float, canonical_flops: float, o=None,
                      keys=None, counts=None):
    """Time the CPU oracle on a bounded, deterministic sample of Sigma blocks
    and extrapolate to the whole build by surviving-term count."""
    import numpy as np

    import oracle
    if o is None:
        o = oracle.Oracle.of(wl)
    if keys is None:
        keys, counts = o.keys(theta)
    total_terms = int(counts.sum())
    k0 = keys[keys[:, 0] == 0]
    order = np.random.default_rng(1).permutation(len(k0))
    cores = os.cpu_count() or 1
    # grow the sample until it takes about `seconds`
    done, t_used, terms = 0, 0.0, 0
    batch = max(cores, 8)
    while done < len(order) and t_used < seconds:
        sel = k0[np.sort(order[done:done + batch])]
        t0 = time.perf_counter()
        _, _, nt = o.blocks(theta, sel, nthreads=cores, terms=True)
        t_used += time.perf_counter() - t0
        terms += int(nt.sum())
        done += len(sel)
        batch *= 2
    t_full = t_used * total_terms / max(terms, 1)
    return {"value": canonical_flops / t_full / 1e12, "unit": "TFLOP/s", "cores": cores,
            "kind": "oracle",
            "sample": (f"{done} Sigma blocks of atom 0 ({terms} of {total_terms} surviving terms, "
                       f"{t_used:.1f} s); full build extrapolated by term count to "
                       f"{t_full:.0f} s"),
            "est_build_s": t_full}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    wl = workload(args.workload, 0)
    o = oracle.Oracle.of(wl)
    keys, counts, extra = o.keys(THETA, extra=True)
    flops = extra["canonical_flops"]
    vals = []
    for step in range(args.warmup + args.steps):
        r = cpu_oracle_sample(wl, THETA, args.ref_seconds, flops, o, keys, counts)
        if step >= args.warmup:
            vals.append(r)
    value = statistics.median(v["value"] for v in vals)
    last = vals[-1]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(v["est_build_s"] for v in vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(wl), "theta": THETA,
                                            "prec": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": last["cores"],
                             "kind": "oracle", "sample": last["sample"]},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    import paper_2009_12505_gb300 as hfx

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = workload(args.workload, rank)
    stream = torch.cuda.Stream()
    ctx = hfx.Context(wl.system.nao, wl.system.nabf, stream=stream.cuda_stream,
                      lattice=wl.system.lattice, pos=wl.system.positions)
    for k in "CVD":
        ctx.set_blocks(k, getattr(wl, k))
    prec, nsl = args.prec, args.nslices

    def barrier():
        if dist:
            dist.barrier()

    for _ in range(args.warmup):
        ctx.build(THETA, prec, nsl)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kms, kfl = {}, {}
    launches = 0
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            ctx.build(THETA, prec, nsl)
            st = ctx.stats()
            launches += st["n_launches"]
            for k, v in st["kernel_ms"].items():
                kms[k] = kms.get(k, 0.0) + v
                kfl[k] = kfl.get(k, 0.0) + st["kernel_flops"][k]
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    st = ctx.stats()
    flops = st["canonical_flops"]
    value = world * flops / (ms / 1e3) / 1e12

    # the plain FP64 GPU build of the same cell, and the split build's deviation from it
    fp64 = None
    if prec != "fp64" and not args.no_fp64:
        ex_split = ctx.build(THETA, prec, nsl)
        sig_split = ctx.sigma()
        ctx.build(THETA, "fp64")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            ex64 = ctx.build(THETA, "fp64")
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        sig64 = ctx.sigma()
        fp64 = {"build_s": ms64 / 1e3, "value": flops / (ms64 / 1e3) / 1e12, "unit": "TFLOP/s",
                "split_speedup": ms64 / ms,
                "max_abs_dsigma_split_vs_fp64_Ha": float(abs(sig_split - sig64).max()),
                "abs_dex_per_atom_Ha": abs(ex_split - ex64) / wl.system.natoms}
        # two digits per operand (hi*hi + hi*lo + lo*hi): faster, but misses the bar
        e0.record(stream)
        exb = ctx.build(THETA, "bf16x3")
        e1.record(stream)
        torch.cuda.synchronize()
        dsb = float(abs(ctx.sigma() - sig64).max())
        fp64["bf16x3"] = {"build_s": e0.elapsed_time(e1) / 1e3,
                          "max_abs_dsigma_vs_fp64_Ha": dsb,
                          "abs_dex_per_atom_Ha": abs(exb - ex64) / wl.system.natoms,
                          "meets_1e-8_Ha": dsb <= 1e-8}
        ctx.build(THETA, prec, nsl)  # leave the context on the split result

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        h2d = sum(getattr(wl, k).data.nbytes + getattr(wl, k).keys.nbytes +
                  getattr(wl, k).offs.nbytes for k in "CVD")
        nsig = int(ctx.offsets()[-1])
        out = np.empty(nsig, np.float64)
        times = []
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in "CVD":
                ctx.set_blocks(k, getattr(wl, k))
            ctx.build(THETA, prec, nsl)
            ctx.sigma(out)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        te = statistics.median(times)
        if dist:
            t = torch.tensor([te], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        e2e = {"value": world * flops / te / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 8 * nsig + 8, "s_per_step": te}

    # roofline of the kernel with the most device time
    top = max(kms, key=kms.get)
    nwaves = max(1, int(st["n_waves"]))
    achieved = kfl[top] / (kms[top] / 1e3) / 1e12
    pk, src = peaks()
    tfl = st.get("kernel_tensor_flops", {}).get(top, 0.0)
    cp = st["canonical_flops_piece"]
    # canonical (Algorithm 3) flops of the pieces each tensor-core kernel computes;
    # with the mirror pieces the D_FG / D_FB kernel also yields the D_AG piece
    canon = {"v1_DFG": cp[0] + cp[1] + (cp[2] if st["mirror"] else 0.0),
             "Y": st["canonical_flops_y"], "v4_DAB": cp[3]}
    desc = {"v1_DFG": "D_FG + D_FB pieces (k_zc: tcgen05 digit products, double-float Y contraction)",
            "Y": "Y = V C (k_pgemm job 0: tcgen05 digit products)",
            "v4_DAB": "D_AB piece (k_pgemm job 1: tcgen05 digit products)"}
    if tfl == 0 or top not in canon:
        roof = {"kernel": top, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                "traffic": None}
    else:
        bf16 = pk["bf16_tflops_sustained"] if "bf16_tflops_sustained" in pk else pk["bf16_tflops"]
        prods = nsl * (nsl + 1) // 2 if prec == "ozaki" else 3
        speak = bf16 / prods
        ach = canon[top] * args.steps / (kms[top] / 1e3) / 1e12
        issued = tfl * args.steps / (kms[top] / 1e3) / 1e12
        roof = {"kernel": top, "kernel_desc": desc[top], "bound": "tensor", "achieved": ach,
                "peak": speak, "unit": "TFLOP/s", "frac": ach / speak,
                "peak_source": f"split roofline: bf16 sustained ({src}) / {prods} digit products",
                "achieved_is": "canonical FP64-equivalent flops of the pieces the kernel computes "
                               "per build / its device time",
                "tensor_issued": {"achieved": issued, "peak": bf16, "frac": issued / bf16,
                                  "unit": "TFLOP/s"},
                "traffic": zc_traffic(tfl / nwaves) if top == "v1_DFG" else None,
                "traffic_note": ("DRAM bytes per launch (one launch per wave): bytes per issued "
                                 "tensor flop from one ncu capture of this kernel on the 8-atom "
                                 "cell, times this launch's issued flops; null once the kernel "
                                 "source differs from the captured one") if top == "v1_DFG" else None}
    roof["kernel_ms_per_step"] = {k: v / args.steps for k, v in kms.items()}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_sample(wl, THETA, args.cpu_seconds, flops)
        cpu.pop("est_build_s", None)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if prec == "fp64" else "bf16", "data": "synthetic",
                "config": {"workload": workload_desc(wl), "theta": THETA, "prec": prec,
                           "nslices": nsl if prec == "ozaki" else None,
                           "arithmetic": ("Y, D_FG, D_FB and D_AB products: exact products of "
                                          "7-bit bf16 digits on tcgen05 (exact f32 group sums "
                                          "per digit order, added in int64 for D_AB and in "
                                          "double-float for Y, D_FG and D_FB); Y contraction "
                                          "of the D_FG / D_FB pieces and P of the D_AB piece "
                                          "in double-float; Sigma in 128-bit fixed point")
                           if prec == "ozaki" else "FP64 CUDA cores; Sigma in 128-bit fixed point",
                           "l2": f"inputs {sum(getattr(wl, k).data.nbytes for k in 'CVD') / 1e9:.2f} GB per cell (L2 is 129 MB)",
                           "parallelism": f"{world} independent cells" if world > 1 else "1 cell"},
                "build_s": ms / 1e3, "canonical_tflop": flops / 1e12,
                "executed_tflop": st["executed_flops"] / 1e12,
                "sigma_blocks": st["n_sigma_blocks"], "survivors": st["survivors"],
                "fp64_gpu": fp64, "mirror_pieces": bool(st["mirror"]),
                "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--prec", choices=["fp64", "ozaki"], default="ozaki")
    ap.add_argument("--nslices", type=int, default=6)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison build")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="si64")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
