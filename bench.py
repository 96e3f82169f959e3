#!/usr/bin/env python
"""Benchmark of the screened periodic LRI exchange build on GB300.

One step = one full hfx_build (block norms, screen, staged contractions,
deterministic Sigma reduction, E_X) over the 512-atom Si-like supercell
(4x4x4 diamond, 13 NAOs / 60 ABFs per atom, C and D blocks within 16 bohr,
V within 20 bohr, theta = 1e-6) with its inputs resident in HBM, in the
6-digit split precision (HFX_OZAKI).

value     canonical TFLOP/s = Algorithm 3 flop count of the build / device time
fp64_gpu  the plain FP64 GPU build of the same cell: time, its split speed-up,
          max |dSigma| split vs FP64, its own roofline on executed FP64 flops
eri_screen  a build with the Cauchy-Schwarz ERI screen added (Eq. CS-ERI): its
          time, the terms it removes and its change of Sigma
e2e       the same metric through the C ABI with host buffers (pinned): set C,
          V, D, build, copy every Sigma block back; e2e_d_only re-sets only D
          (the cached-plan path of an SCF iteration)
roofline  the kernel with the most device time: issued bf16 tensor flops
          against the measured bf16 peak, plus the FP64-equivalent products
          without padding and the canonical (effective) rate
cpu_baseline  the CPU oracle on this host's cores, on a bounded sample of the
          same workload (Sigma blocks of atom 0), extrapolated by surviving-term
          count; the same sample gives a parity check of the GPU blocks

--impl reference times the CPU oracle alone (rank 0) on bounded samples.
Under torchrun (N > 1) the ranks share one cell: each contracts the pairs of
its central atoms (machine scheduling, Algorithm 6) and the fixed-point Sigma
accumulators are summed with one int64 all-reduce over NCCL, the build's one
exchange step (strong scaling; value = the cell's canonical flops / time).
--replicas instead gives every rank its own independent cell (weak scaling,
no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HFX build s & TFLOP/s on 1 GB300, split-prec vs FP64 at max|ΔH|≤1e-8 Ha"
THETA = 1e-6
PARITY_BAR = {"ozaki": 1e-8, "fp64": 1e-10}
# FP64 on CUDA cores: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


# name: (lattice, cells per edge, seed, generator options).  The Si-like
# diamond cells and the two-element rocksalt-like cell carry the paper's
# shapes; the last two are the second workload: full-range Coulomb V out to
# 50 bohr, and a metallic D (polynomial decay) out to 24 bohr.
WORKLOADS = {"si512": ("si", 4, 3, {}), "si64": ("si", 2, 2, {}), "si8": ("si", 1, 1, {}),
             "ab216": ("ab", 3, 4, {}),
             "si8_fullrange": ("si", 1, 5, {"cut_V": 50.0, "mu": 0.0}),
             "si8_metal": ("si", 1, 6, {"cut_D": 24.0, "d_decay": "power"})}


# The batched form: cells drawn (seeded) from Si-like 1x1x1 and 2x2x2 cells and the
# two-element 1x1x1 cell, each with a threshold drawn from {1e-5, 1e-6, 1e-7}.
BATCHES = {"batch12": 12}


def batch_cells(name: str, rank: int):
    """[(workload, theta)] of a batch; cell i has seed 1000 + i."""
    import numpy as np

    import synth
    rng = np.random.default_rng(12345 + rank)
    out = []
    for i in range(BATCHES[name]):
        kind = ["si8", "si64", "ab8"][int(rng.integers(3))]
        theta = [1e-5, 1e-6, 1e-7][int(rng.integers(3))]
        seed = 1000 + i + 100000 * rank
        if kind == "si8":
            system = synth.si_diamond(1)
        elif kind == "si64":
            system = synth.si_diamond(2)
        else:
            system = synth.two_element_rocksalt(1, seed=seed)
        out.append((synth.make_workload(system, seed=seed, name=kind), theta))
    return out


def workload(name: str, rank: int):
    import synth
    kind, ncell, seed, opts = WORKLOADS[name]
    s = seed + 1000 * rank
    system = synth.si_diamond(ncell) if kind == "si" else synth.two_element_rocksalt(ncell, seed=s)
    return synth.make_workload(system, seed=s, name=name, **opts)


def workload_desc(wl) -> str:
    kind, ncell, _, opts = WORKLOADS[wl.name]
    extra = ""
    if opts.get("mu") == 0.0:
        extra += ", full-range Coulomb V"
    if opts.get("d_decay") == "power":
        extra += ", metallic D (polynomial decay)"
    cells = f"{ncell}x{ncell}x{ncell}"
    if kind == "si":
        lat = f"Si-like diamond {cells} supercell, {wl.system.natoms} atoms, 13 NAO / 60 ABF per atom"
    else:
        lat = (f"two-element rocksalt-like {cells} supercell (a = 8 bohr), {wl.system.natoms} "
               f"atoms, half 13 NAO / 60 ABF and half 27 NAO / 90 ABF")
    return (f"{wl.name}: {lat}, C <= {wl.cut_C:g} bohr, D <= {wl.cut_D:g} bohr, "
            f"V <= {wl.cut_V:g} bohr{extra}, theta = {THETA:g}, seed {wl.seed}")


# dram__bytes_read.sum + dram__bytes_write.sum of one k_zc launch on the 8-atom
# cell over its issued bf16 tensor flops, captured from the hfx_zc.cu whose code
# (comments and blank space removed) has this sha256 prefix (see the k_zc
# profile summary under profiles/)
ZC_BYTES_PER_TENSOR_FLOP = (30.483057e9 + 0.469812e9) / 14.988985761792e12
ZC_CAPTURED_SHA = "efee46cbd3e070ad"


def source_digest(path):
    """sha256 prefix of a C++/CUDA source's code: comments and blank space
    removed, so an edit of comments alone keeps the digest."""
    import hashlib
    import re
    text = open(path, encoding="utf-8").read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    text = " ".join(text.split())
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def zc_traffic(tensor_flops_per_launch):
    src = os.path.join(ROOT, "paper_2009_12505_gb300", "csrc", "hfx_zc.cu")
    try:
        sha = source_digest(src)
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
    """nvidia-smi clocks and throttle reasons sampled every 200 ms into a
    temporary file that is removed after the summary is taken."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="hfx_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
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

    def close(self):
        try:
            os.remove(self.path)
        except OSError:
            pass


def sample_atoms(natoms: int, n: int = 8):
    """Central atoms whose oracle key sets stand for the whole cell: all of
    them for small cells, else n evenly spaced ones."""
    if natoms <= n:
        return list(range(natoms))
    return [round(i * natoms / n) for i in range(n)]


def oracle_term_total(o, natoms: int, theta: float):
    """Surviving terms of the whole build, from the oracle's per-atom key
    enumeration on sample_atoms (scaled by natoms / number sampled)."""
    atoms = sample_atoms(natoms)
    tot = 0
    for a in atoms:
        _, c = o.keys(theta, atoms=(a, a + 1))
        tot += int(c.sum())
    return tot * natoms / len(atoms), atoms


def cpu_oracle_sample(wl, theta: float, seconds: float, canonical_flops: float, o=None,
                      totals=None):
    """Time the CPU oracle on a bounded, deterministic sample of atom 0's
    Sigma blocks and extrapolate to the whole build by surviving-term count
    (``totals`` = oracle_term_total's result, computed here when None).
    Returns the baseline record and the sampled (keys, blocks, offsets)."""
    import numpy as np

    import oracle
    if o is None:
        o = oracle.Oracle.of(wl)
    total_terms, atoms = totals or oracle_term_total(o, wl.system.natoms, theta)
    k0, _ = o.keys(theta, atoms=(0, 1))
    order = np.random.default_rng(1).permutation(len(k0))
    cores = os.cpu_count() or 1
    # grow the sample until it takes about `seconds`
    done, t_used, terms = 0, 0.0, 0
    batch = max(cores, 8)
    sk, sd, so = [], [], []
    while done < len(order) and t_used < seconds:
        sel = k0[np.sort(order[done:done + batch])]
        t0 = time.perf_counter()
        data, offs, nt = o.blocks(theta, sel, nthreads=cores, terms=True)
        t_used += time.perf_counter() - t0
        terms += int(nt.sum())
        done += len(sel)
        batch *= 2
        sk.append(sel)
        sd.append(data)
        so.append(offs)
    t_full = t_used * total_terms / max(terms, 1)
    rec = {"value": canonical_flops / t_full / 1e12, "unit": "TFLOP/s", "cores": cores,
           "kind": "oracle",
           "sample": (f"{done} Sigma blocks of atom 0 ({terms} surviving terms, {t_used:.1f} s on "
                      f"{cores} threads); the build's {total_terms:.4g} surviving terms counted by "
                      f"the oracle on central atoms {atoms} and scaled to all "
                      f"{wl.system.natoms}; full build extrapolated by term count to "
                      f"{t_full:.0f} s"),
           "est_build_s": t_full}
    return rec, (sk, sd, so)


def sampled_parity(ctx, sample, nao, bar):
    """max |dSigma| of the GPU blocks against the oracle's sampled blocks."""
    import numpy as np
    sk, sd, so = sample
    keys = ctx.keys()
    offs = ctx.offsets()
    sig = ctx.sigma()
    index = {tuple(k): e for e, k in enumerate(keys.tolist())}
    err, nblk, missing = 0.0, 0, 0
    for sel, data, o in zip(sk, sd, so):
        for e, k in enumerate(sel.tolist()):
            g = index.get(tuple(k))
            if g is None:
                missing += 1
                continue
            d = np.abs(sig[offs[g]:offs[g + 1]] - data[o[e]:o[e + 1]])
            err = max(err, float(d.max()) if d.size else 0.0)
            nblk += 1
    return {"blocks": nblk, "missing_keys": missing, "max_abs_dsigma_Ha": err, "bar_Ha": bar,
            "pass": missing == 0 and err <= bar}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    wl = workload(args.workload, 0)
    o = oracle.Oracle.of(wl)
    # canonical flops of the whole build, counted by the oracle over the
    # sampled central atoms and scaled (the same sampling as the term count)
    atoms = sample_atoms(wl.system.natoms)
    fl = 0.0
    for a in atoms:
        _, _, ex = o.keys(THETA, atoms=(a, a + 1), extra=True)
        fl += ex["canonical_flops"]
    flops = fl * wl.system.natoms / len(atoms)
    totals = oracle_term_total(o, wl.system.natoms, THETA)
    vals = []
    for step in range(args.warmup + args.steps):
        r, _ = cpu_oracle_sample(wl, THETA, args.ref_seconds, flops, o, totals)
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


def pinned_copy(blocks):
    """The block set's keys, data and offsets with the data in page-locked
    host memory (so host-to-device copies run at full speed)."""
    import numpy as np
    import torch
    t = torch.from_numpy(np.ascontiguousarray(blocks.data)).pin_memory()
    return (np.ascontiguousarray(blocks.keys, np.int32), t.numpy(),
            np.ascontiguousarray(blocks.offs, np.int64), t)


def run_batch(args):
    """Many independent cells of uneven size with their own thresholds, built
    by one hfx_build_batch (one merged build: per wave one launch of each
    persistent kernel for all cells), against the same cells built one by
    one."""
    import torch

    import paper_2009_12505_gb300 as hfx
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    cells = batch_cells(args.workload, 0)
    stream = torch.cuda.Stream()
    ctxs = []
    for wl, _ in cells:
        c = hfx.Context(wl.system.nao, wl.system.nabf, stream=stream.cuda_stream)
        for k in "CVD":
            c.set_blocks(k, getattr(wl, k))
        ctxs.append(c)
    thetas = [th for _, th in cells]
    prec, nsl = args.prec, args.nslices
    for _ in range(args.warmup):
        hfx.build_batch(ctxs, thetas, prec, nsl)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    clk = ClockSampler(0)
    with clk:
        e0.record(stream)
        for _ in range(args.steps):
            hfx.build_batch(ctxs, thetas, prec, nsl)
            launches += ctxs[0].stats()["n_launches"]
        e1.record(stream)
        torch.cuda.synchronize()
    clocks = clk.summary()
    clk.close()
    ms = e0.elapsed_time(e1) / args.steps
    st = ctxs[0].stats()
    flops = st["canonical_flops"]
    # the same cells one by one, each on a fresh context freed after its build
    # (every context keeps its own scratch, so twelve at once would not fit)
    for c in ctxs:
        c.close()
    ctxs = []
    ms_seq = 0.0
    for wl, th in cells:
        c = hfx.Context(wl.system.nao, wl.system.nabf, stream=stream.cuda_stream)
        for k in "CVD":
            c.set_blocks(k, getattr(wl, k))
        c.build(th, prec, nsl)           # slicing and planning, not timed
        torch.cuda.synchronize()
        e0.record(stream)
        c.build(th, prec, nsl)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_seq += e0.elapsed_time(e1)
        c.close()
    kinds = {}
    for wl, th in cells:
        kinds[f"{wl.name}@{th:g}"] = kinds.get(f"{wl.name}@{th:g}", 0) + 1
    line = {"metric": METRIC, "value": flops / (ms / 1e3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if prec != "fp64" else "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {len(cells)} independent cells "
                                   f"(Si-like 8 and 64 atoms, two-element 8 atoms; seeds 1000+i), "
                                   f"theta per cell from {{1e-5, 1e-6, 1e-7}}: {kinds}",
                       "prec": prec, "nslices": nsl if prec == "ozaki" else None,
                       "parallelism": "one merged build (hfx_build_batch)"},
            "canonical_tflop": flops / 1e12, "batch_s": ms / 1e3,
            "cells_one_by_one_s": ms_seq / 1e3, "batch_speedup": ms_seq / ms,
            "one_by_one_is": "sum of each cell's second hfx_build on its own context (the "
                             "first slices and plans), CUDA events",
            "n_waves": st["n_waves"], "gpu_launches": launches,
            "kernel_ms_per_step": st["kernel_ms"], "clocks": clocks}
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
    if world > 1 or args.shard:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    shard = (world > 1 and not args.replicas) or args.shard
    world_measured = world
    wl = workload(args.workload, 0 if shard else rank)
    natoms = wl.system.natoms
    stream = torch.cuda.Stream()
    ctx = hfx.Context(wl.system.nao, wl.system.nabf, stream=stream.cuda_stream,
                      lattice=wl.system.lattice, pos=wl.system.positions)
    for k in "CVD":
        ctx.set_blocks(k, getattr(wl, k))
    prec, nsl = args.prec, args.nslices
    words = None
    if shard:
        from paper_2009_12505_gb300 import sharding
        owner = sharding.lpt(sharding.atom_costs(natoms, wl.C.keys, wl.V.keys), world)
        ctx.set_shard(owner, rank)

    def step():
        """One build; in the sharded form also the exchange of the fixed-point
        Sigma words and the final Sigma and E_X from their sum."""
        nonlocal words
        ctx.build(THETA, prec, nsl)
        if not shard:
            return
        if words is None:
            words = torch.empty((int(ctx.offsets()[-1]), 2), dtype=torch.int64, device="cuda")
        ctx.sigma_fixed(words, on_device=True)
        dist.all_reduce(words, op=dist.ReduceOp.SUM)
        torch.cuda.current_stream().synchronize()
        ctx.set_sigma_fixed(words, on_device=True)

    def barrier():
        if dist:
            dist.barrier()

    def max_over_ranks(x):
        if not dist:
            return x
        t = torch.tensor([x], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kms, kfl, ktf, kuf = {}, {}, {}, {}
    launches = 0
    clk = ClockSampler(local)
    with clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
            st = ctx.stats()
            launches += st["n_launches"]
            for k, v in st["kernel_ms"].items():
                kms[k] = kms.get(k, 0.0) + v
                kfl[k] = kfl.get(k, 0.0) + st["kernel_flops"][k]
                ktf[k] = ktf.get(k, 0.0) + st["kernel_tensor_flops"][k]
                kuf[k] = kuf.get(k, 0.0) + st["kernel_unpadded_flops"][k]
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    clocks = clk.summary()
    clk.close()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps)
    st = ctx.stats()
    flops = st["canonical_flops"]   # of the whole cell (every rank screens globally)
    cells = 1 if shard else world
    value = cells * flops / (ms / 1e3) / 1e12
    if shard:
        # the remaining measurements run on the unsharded cell, on rank 0 alone
        ctx.set_shard(None, 0)
        if rank != 0:
            dist.barrier()
            dist.destroy_process_group()
            return 0
        dist.barrier()
        dist.destroy_process_group()
        world, dist = 1, None
    pk, src = peaks()
    bf16 = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])

    def fp64_roof(kms_, kfl_, steps):
        top = max(kms_, key=kms_.get)
        ach = kfl_[top] / (kms_[top] / 1e3) / 1e12
        return {"kernel": top, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                "achieved_is": "executed FP64 multiply-adds x 2 of the kernel / its device time",
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                "kernel_ms_per_step": {k: v / steps for k, v in kms_.items()}}

    # the plain FP64 GPU build of the same cell, and the split build's deviation from it
    fp64 = None
    if prec != "fp64" and not args.no_fp64:
        ex_split = ctx.build(THETA, prec, nsl)
        sig_split = ctx.sigma()
        ctx.build(THETA, "fp64")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        km64, kf64 = {}, {}
        e0.record(stream)
        for _ in range(args.fp64_steps):
            ex64 = ctx.build(THETA, "fp64")
            s64 = ctx.stats()
            for k, v in s64["kernel_ms"].items():
                km64[k] = km64.get(k, 0.0) + v
                kf64[k] = kf64.get(k, 0.0) + s64["kernel_flops"][k]
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        sig64 = ctx.sigma()
        fp64 = {"build_s": ms64 / 1e3, "value": flops / (ms64 / 1e3) / 1e12, "unit": "TFLOP/s",
                "split_speedup": ms64 / ms,
                "max_abs_dsigma_split_vs_fp64_Ha": float(abs(sig_split - sig64).max()),
                "abs_dex_per_atom_Ha": abs(ex_split - ex64) / natoms,
                "roofline": fp64_roof(km64, kf64, args.fp64_steps)}
        # two digits per operand (hi*hi + hi*lo + lo*hi): faster, but misses the bar
        e0.record(stream)
        exb = ctx.build(THETA, "bf16x3")
        e1.record(stream)
        torch.cuda.synchronize()
        dsb = float(abs(ctx.sigma() - sig64).max())
        fp64["bf16x3"] = {"build_s": e0.elapsed_time(e1) / 1e3,
                          "max_abs_dsigma_vs_fp64_Ha": dsb,
                          "abs_dex_per_atom_Ha": abs(exb - ex64) / natoms,
                          "meets_1e-8_Ha": dsb <= 1e-8}
        ctx.build(THETA, prec, nsl)  # leave the context on the split result

    # the Cauchy-Schwarz ERI screen on top of the block screen (Eq. CS-ERI):
    # time saved and the change of Sigma against the build without it
    eri = None
    if prec != "fp64" and args.eps_eri > 0:
        ex_plain = ctx.build(THETA, prec, nsl)
        k_plain, o_plain, s_plain = ctx.keys(), ctx.offsets(), ctx.sigma()
        n_plain = sum(ctx.stats()["survivors"])
        ctx.set_eri_screen(args.eps_eri)
        ctx.build(THETA, prec, nsl)   # the per-C-block bounds are computed once here
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.eri_steps):
            ex_eri = ctx.build(THETA, prec, nsl)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_eri = e0.elapsed_time(e1) / args.eri_steps
        se = ctx.stats()
        k_eri, o_eri, s_eri = ctx.keys(), ctx.offsets(), ctx.sigma()

        def packed(k):
            k = k.astype(np.int64)
            return (k[:, 0] << 44) | (k[:, 1] << 24) | ((k[:, 2] + 128) << 16) | \
                ((k[:, 3] + 128) << 8) | (k[:, 4] + 128)
        pp, pe = packed(k_plain), packed(k_eri)
        pos = np.searchsorted(pp, pe)
        assert np.array_equal(pp[pos], pe), "screened key set is not a subset"
        diff = s_plain.copy()
        for e, q in enumerate(pos):   # screened blocks minus the plain ones
            diff[o_plain[q]:o_plain[q + 1]] -= s_eri[o_eri[e]:o_eri[e + 1]]
        eri = {"eps_eri": args.eps_eri, "build_s": ms_eri / 1e3, "speedup_vs_block_screen": ms / ms_eri,
               "surviving_terms": sum(se["survivors"]), "surviving_terms_block_screen": n_plain,
               "removed_quadruples": se["n_eri_removed"],
               "canonical_tflop": se["canonical_flops"] / 1e12,
               "max_abs_dsigma_vs_block_screen_Ha": float(np.abs(diff).max()),
               "abs_dex_per_atom_vs_block_screen_Ha": abs(ex_eri - ex_plain) / natoms}
        ctx.set_eri_screen(None)
        ctx.build(THETA, prec, nsl)

    # end to end through the C ABI with host buffers (page-locked staging)
    e2e = e2e_d = None
    if not args.no_e2e:
        staged = {k: pinned_copy(getattr(wl, k)) for k in "CVD"}
        h2d = {k: staged[k][1].nbytes + staged[k][0].nbytes + staged[k][2].nbytes for k in "CVD"}
        nsig = int(ctx.offsets()[-1])
        out = torch.empty(nsig, dtype=torch.float64).pin_memory().numpy()

        def e2e_steps(kinds, n):
            times = []
            for _ in range(n):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for k in kinds:
                    keys, data, offs, _ = staged[k]
                    ctx.set_many(k, keys, data, offs)
                ctx.build(THETA, prec, nsl)
                ctx.sigma(out)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            return max_over_ranks(statistics.median(times)), times

        te, times = e2e_steps("CVD", args.e2e_steps)
        e2e = {"value": world * flops / te / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": sum(h2d.values()), "d2h_bytes_per_step": 8 * nsig + 8,
               "s_per_step": te, "steps": len(times), "s_min": min(times), "s_max": max(times),
               "what": "median over steps of: set C, V and D from page-locked host memory "
                       "(hfx_set_many), hfx_build, read every Sigma block (hfx_get_H_all)"}
        td, times = e2e_steps("D", args.e2e_steps)
        e2e_d = {"value": world * flops / td / 1e12, "unit": "TFLOP/s",
                 "h2d_bytes_per_step": h2d["D"], "d2h_bytes_per_step": 8 * nsig + 8,
                 "s_per_step": td, "steps": len(times), "s_min": min(times),
                 "s_max": max(times),
                 "what": "as e2e with only D set again (C, V and their sliced operands and "
                         "plan cached): one SCF iteration's exchange build"}

    # roofline of the kernel with the most device time
    top = max(kms, key=kms.get)
    nwaves = max(1, int(st["n_waves"]))
    achieved = kfl[top] / (kms[top] / 1e3) / 1e12
    cp = st["canonical_flops_piece"]
    # canonical (Algorithm 3) flops of the pieces each tensor-core kernel computes;
    # with the mirror pieces the D_FG / D_FB kernel also yields the D_AG piece
    canon = {"v1_DFG": cp[0] + cp[1] + (cp[2] if st["mirror"] else 0.0),
             "Y": st["canonical_flops_y"], "v4_DAB": cp[3]}
    desc = {"v1_DFG": "k_zc: D_FG + D_FB pieces (tcgen05 digit products, double-float Y "
                      "contraction in the epilogue)",
            "Y": "k_pgemm job 0: Y = V C (tcgen05 digit products)",
            "v4_DAB": "k_pgemm job 1: D_AB piece (tcgen05 digit products)"}
    if ktf.get(top, 0.0) == 0 or top not in canon:
        roof = {"kernel": top, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                "traffic": None}
    else:
        prods = nsl * (nsl + 1) // 2 if prec == "ozaki" else 3
        t_s = kms[top] / 1e3
        issued = ktf[top] / t_s / 1e12
        unp = kuf[top] / t_s / 1e12
        roof = {"kernel": top, "kernel_desc": desc[top], "bound": "tensor",
                "achieved": issued, "peak": bf16, "unit": "TFLOP/s", "frac": issued / bf16,
                "peak_source": f"bf16 dense, sustained ({src} MEASURED_PEAKS.json)",
                "achieved_is": "bf16 tensor-core flops issued by the kernel (every digit "
                               "product, padding included) / its device time",
                "fp64_equivalent_unpadded": (
                    {"achieved": unp, "peak": bf16 / prods, "frac": unp * prods / bf16,
                     "unit": "TFLOP/s",
                     "what": f"FP64-equivalent products the kernel executes without padding or "
                             f"zero tiles, after the mirror and sum-over-F reassociations, / "
                             f"time; peak = bf16 / {prods} digit products"}
                    if unp > 0 else None),
                "effective_tflops": canon[top] * args.steps / t_s / 1e12,
                "effective_is": "canonical Algorithm 3 flops of the pieces the kernel yields "
                                "/ its device time (counts work the reassociations avoid)",
                "traffic": zc_traffic(ktf[top] / args.steps / nwaves) if top == "v1_DFG" else None,
                "traffic_note": ("DRAM bytes per launch (one launch per wave): bytes per issued "
                                 "tensor flop from one ncu capture of this kernel on the 8-atom "
                                 "cell, times this launch's issued flops; null once the kernel "
                                 "source differs from the captured one") if top == "v1_DFG" else None}
    roof["kernel_ms_per_step"] = {k: v / args.steps for k, v in kms.items()}
    roof["kernel_tensor_tflop_per_step"] = {k: v / args.steps / 1e12 for k, v in ktf.items() if v}
    roof["launches_per_step_of_top"] = nwaves
    if top == "v1_DFG" and st.get("zc_dt_max_over_avg"):
        roof["cta_dt_max_over_avg"] = st["zc_dt_max_over_avg"]

    cpu = parity = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, sample = cpu_oracle_sample(wl, THETA, args.cpu_seconds, flops)
        cpu.pop("est_build_s", None)
        parity = sampled_parity(ctx, sample, wl.system.nao, PARITY_BAR.get(prec, 1e-8))

    if rank == 0:
        nranks = world_measured if shard else world
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": nranks,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "strong" if shard else "weak",
                "vs_baseline": None,
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
                           "l2": f"no flush: inputs {sum(getattr(wl, k).data.nbytes for k in 'CVD') / 1e9:.2f} GB per cell and GBs of per-wave scratch exceed the 129 MB L2",
                           "parallelism": (f"{world_measured} ranks share the cell: central atoms "
                                           "by machine scheduling, one int64 all-reduce of the "
                                           "fixed-point Sigma" if shard else
                                           f"{world} independent cells" if world > 1 else "1 cell")},
                "build_s": ms / 1e3, "canonical_tflop": flops / 1e12,
                "executed_tflop": st["executed_flops"] / 1e12,
                "sigma_blocks": st["n_sigma_blocks"], "survivors": st["survivors"],
                "parity_vs_oracle_sampled": parity,
                "fp64_gpu": fp64, "eri_screen": eri, "mirror_pieces": bool(st["mirror"]),
                "e2e": e2e, "e2e_d_only": e2e_d, "gpu_launches": launches, "roofline": roof,
                "cpu_baseline": cpu, "clocks": clocks}
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
    ap.add_argument("--shard", action="store_true",
                    help="the sharded form even on one rank (under torchrun)")
    ap.add_argument("--replicas", action="store_true",
                    help="under torchrun: one independent cell per rank instead of one shared, "
                         "sharded cell")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + sorted(BATCHES), default="si512")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--eps-eri", type=float, default=1e-3,
                    help="also time a build with the Cauchy-Schwarz ERI screen at this "
                         "threshold (0 skips it); the headline build does not use it")
    ap.add_argument("--eri-steps", type=int, default=2)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=4.0)
    args = ap.parse_args()
    if args.workload in BATCHES:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched cells have no "
                              "reference arm; use a single-cell workload"}))
            return 0
        return run_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
