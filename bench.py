"""Benchmark of the seed-location filter on GB300.

Three forms of the hot path, each on its synthetic workload:
  gather   (default line): 100 Mbp repeat-rich reference (70% i.i.d. ACGT +
           30% planted repeat families at 10-20% divergence), q=5, 256 bp
           bins + 150 bp overlap; 1M reads of 150 bp (4% substitutions, 1%
           indels), E=7; candidates = bins of all exact 12-mer seed hits from
           a CPU index, capped at 1,000 per read.  One step = one grim_filter
           over the whole batch.
  batched: 100 Mbp repeat-rich reference, q=6, 256 + 300 bp; 2M reads of
           50-300 bp (3% + 1%), E = floor(0.05 L); true bin + log-uniform
           1-5,000 candidates.  One step = one grim_filter_batched (one
           cost-balanced launch per 262,144 reads, replayed CUDA graph,
           autotuned launch shape).
  fullscan: 3.1 Gbp repeat-rich reference, q=5, 256 + 100 bp (12.1M bins);
           a batch of 65,536 reads of 100 bp, E=5, every bin scored on the
           tensor cores.  One step = one grim_scan.
The bank is built once per reference beforehand (the paper also leaves
bitvector generation out of its runtime, Sec. 6.1) and timed on its own.
`--workload` picks the form of the JSON line; the other two are measured
after it and reported as sub-objects unless disabled.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "(read,bin) checks/s & reads/s at E=0.05·L; frac of HBM/INT8 roofline vs plain"
UNIT = "checks/s"
L2_FLUSH_BYTES = 256 << 20

# dram__bytes_read.sum + dram__bytes_write.sum of one full-size launch, from
# an ncu capture, valid only for the kernel source it was taken on.
TRAFFIC_BY_SOURCE: dict[str, dict] = {
    # gather_kernel<5,8>, 1M reads, 74.8M checks: 660.20 MB read + 74.78 MB written
    "0b92bfcdafdb14db": {"bytes": 734_982_656, "reads": 1_000_000},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gather", choices=["gather", "batched", "fullscan", "mixed"])
    ap.add_argument("--reads", type=int, default=1_000_000, help="gather: reads per GPU (weak scaling)")
    ap.add_argument("--ref-bp", type=int, default=100_000_000, help="gather: reference length")
    ap.add_argument("--batched-reads", type=int, default=2_000_000)
    ap.add_argument("--scan-ref-bp", type=int, default=3_100_000_000)
    ap.add_argument("--scan-reads", type=int, default=65_536)
    ap.add_argument("--sub-steps", type=int, default=3, help="timed steps of the sub-measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="--impl reference: target CPU time of the whole run (warm-up + timed steps)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched sub-measurement")
    ap.add_argument("--no-full-scan", action="store_true", help="skip the full-scan sub-measurement")
    ap.add_argument("--no-mixed", action="store_true", help="skip the dispatcher (mixed) sub-measurement")
    ap.add_argument("--mixed-reads", type=int, default=10_000_000)
    ap.add_argument("--no-q-sweep", action="store_true", help="skip the token-size sweep (q = 4, 5, 6)")
    ap.add_argument("--q-sweep-reads", type=int, default=262_144)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def load_fp8_peak():
    """Dense e4m3 tensor peak: the measured bf16 cuBLAS peak x the nominal
    fp8 / bf16 ratio (4.5 / 2.25 PFLOP/s); burst and sustained."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return (float(d["bf16_tflops"]) * 2.0, float(d.get("bf16_tflops_sustained", d["bf16_tflops"])) * 2.0,
                "measured bf16 x 2")
    return 1900.0 * 2.0, 1700.0 * 2.0, "fallback bf16 x 2"


def source_sha(files=("gather.cu", "grim_internal.cuh", "tokens.cuh")):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1711_01177_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks + throttle reasons sampled during a timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.rows = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for ln in out.splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) >= 9:
                self.rows.append(f)

    def summary(self):
        if not self.rows:
            return None
        num = lambda x: x.replace(".", "", 1).isdigit()
        sm = [float(r[1]) for r in self.rows if num(r[1])]
        mx = [float(r[2]) for r in self.rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# --------------------------------------------------------------- workloads

def make_gather(args, rank):
    import synth
    return synth.gather_seeds(ref_len=args.ref_bp, n_reads=args.reads, read_seed=synth.SEED_READS + 1000 * rank)


def make_batched(args, rank):
    import synth
    return synth.batched_varlen(n_reads=args.batched_reads, read_seed=synth.SEED_READS + 1000 * rank)


def make_fullscan(args, rank):
    import synth
    return synth.fullscan(ref_len=args.scan_ref_bp, n_reads=args.scan_reads,
                          read_seed=synth.SEED_READS + 1000 * rank)


def make_mixed(args, rank, cand_reads=0):
    """Candidates come from the GPU seed table; cand_reads > 0 also builds
    CPU lists for the first reads (the oracle's sample)."""
    import synth
    return synth.mixed_seeds(ref_len=args.scan_ref_bp, n_reads=args.mixed_reads,
                             read_seed=synth.SEED_READS + 1000 * rank, cand_reads=cand_reads)


def describe(form, w):
    L = np.diff(w.read_offsets)
    base = {"ref_bp": w.ref_len, "q": w.q, "bin_len": w.bin_len, "overlap": w.overlap, "n_bins": w.n_bins,
            "reads_per_gpu": w.n_reads, "read_len": [int(L.min()), int(L.max())],
            "E": [int(w.E.min()), int(w.E.max())], "sub": w.meta["sub"], "indel": w.meta["indel"],
            "repeat_frac": w.meta["repeat_frac"],
            "l2": "flushed between timed steps (256 MiB write, outside the events)"}
    rep = f"{int(w.meta['repeat_frac'] * 100)}% repeats"
    if form == "gather":
        c = np.diff(w.cand_offsets)
        base.update(workload=f"gather, {w.ref_len / 1e6:g} Mbp repeat-rich reference ({rep}), q={w.q}, "
                             f"{w.n_reads} x {int(L[0])} bp reads/GPU, 12-mer seed candidates (cap 1000)",
                    checks_per_gpu_step=w.n_checks, cands_per_read_mean=round(float(c.mean()), 2),
                    cands_per_read_max=int(c.max()))
    elif form == "batched":
        base.update(workload=f"batched gather, {w.ref_len / 1e6:g} Mbp repeat-rich reference ({rep}), q={w.q}, "
                             f"{w.n_reads} reads of {int(L.min())}-{int(L.max())} bp/GPU, E=floor(0.05 L), "
                             f"log-uniform 1-5000 candidates (mean {w.n_checks / w.n_reads:.0f})",
                    checks_per_gpu_step=w.n_checks)
    elif form == "mixed":
        base.update(workload=f"dispatcher, {w.ref_len / 1e9:g} Gbp reference ({rep} at 5-20% divergence), q={w.q}, "
                             f"{w.n_reads} x {int(L[0])} bp reads/GPU, 12-mer seed candidates (cap 10000), "
                             f"gather vs full scan chosen per batch")
        if w.cand_offsets is not None and len(w.cand_offsets) == w.n_reads + 1:
            c = np.diff(w.cand_offsets)
            base.update(checks_per_gpu_step=w.n_checks, cands_per_read_mean=round(float(c.mean()), 2),
                        cands_per_read_max=int(c.max()))
    else:
        base.update(workload=f"full scan, {w.ref_len / 1e9:g} Gbp repeat-rich reference ({rep}), q={w.q}, "
                             f"{w.n_bins} bins, batch of {w.n_reads} x {int(L[0])} bp reads/GPU, every bin",
                    checks_per_gpu_step=w.n_reads * w.n_bins)
    return base


def gather_bytes(w, row_bytes):
    """Bytes one gather pass must move: per check the bin row, the candidate
    id and the pass byte; per read its bases, two offsets and E."""
    return w.n_checks * (row_bytes + 4 + 1) + int(w.read_offsets[-1]) + (w.n_reads + 1) * 16 + w.n_reads * 2


# --------------------------------------------------------------- one form

def max_over_ranks(x, world):
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Ctx:
    def __init__(self, rank, world, local):
        import torch
        self.rank, self.world, self.local = rank, world, local
        self.stream = torch.cuda.Stream()
        self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    @staticmethod
    def dev(a):
        import torch
        a = np.ascontiguousarray(a)
        view = {np.dtype(np.uint32): np.int32, np.dtype(np.uint16): np.int16}.get(a.dtype)
        return torch.from_numpy(a.view(view) if view else a).cuda()

    @staticmethod
    def pin(a):
        import torch
        a = np.ascontiguousarray(a)
        view = {np.dtype(np.uint32): np.int32, np.dtype(np.uint16): np.int16}.get(a.dtype)
        return torch.from_numpy(a.view(view) if view else a).pin_memory()

    def max_over_ranks(self, x):
        return max_over_ranks(x, self.world)

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(self, fn, steps, warmup, clocks=False):
        """Per-step CUDA-event times on the launching stream, L2 flushed
        between steps outside the events; returns (list of ms, clock summary)."""
        import torch
        s = self.stream
        for i in range(warmup):
            with torch.cuda.stream(s):
                self.flush.fill_(i)
                fn()
        s.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        self.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(self.local) if clocks else None
        if sampler:
            sampler.__enter__()
        for i in range(steps):
            with torch.cuda.stream(s):
                self.flush.fill_(i)
                ev[i][0].record(s)
                fn()
                ev[i][1].record(s)
        torch.cuda.synchronize()
        if sampler:
            sampler.__exit__(None, None, None)
        self.barrier()
        return [a.elapsed_time(b) for a, b in ev], (sampler.summary() if sampler else None)


def run_form(form, args, ctx, primary):
    """Measure one form; returns its JSON dict (contract keys if primary)."""
    import torch

    import paper_1711_01177_gb300 as grim
    w = {"gather": make_gather, "batched": make_batched, "fullscan": make_fullscan,
         "mixed": make_mixed}[form](args, ctx.rank)
    dev, s = ctx.dev, ctx.stream
    steps = args.steps if primary else args.sub_steps
    warmup = args.warmup if primary else 2

    ref_d = dev(w.ref2bit)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        e0.record(s)
        bank = grim.grim_build_bank(ref_d, w.ref_len, w.q, w.bin_len, w.overlap, stream=s)
        e1.record(s)
    s.synchronize()
    bank_ms = e0.elapsed_time(e1)
    st, flags = grim.grim_bank_status(bank, s)
    assert st == grim.GRIM_OK, (st, flags)
    row = bank.row_words * 4
    bank_info = {"ms": bank_ms, "mbp_per_s": w.ref_len / 1e6 / (bank_ms / 1e3),
                 "gb_per_s": (bank.n_bins * row + len(w.ref2bit)) / 1e9 / (bank_ms / 1e3),
                 "bank_bytes": bank.n_bins * row}
    del ref_d

    out = {"form": form}
    if form == "mixed":
        # the mapper's side of the filter on the GPU: seed table, candidates,
        # then the dispatcher over every read, then the Seed Location Checker
        torch.cuda.empty_cache()  # the library allocates from the CUDA pool, not torch's cache
        ref_d = dev(w.ref2bit)
        reads_d, offs_d, E_d = dev(w.bases), dev(w.read_offsets), dev(w.E)
        s.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s):
            idx = grim.grim_seed_index_build(ref_d, w.ref_len, w.meta["seed_k"], stream=s)
        s.synchronize()
        index_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        with torch.cuda.stream(s):
            cb_d, co_d = grim.grim_seed_candidates(idx, reads_d, offs_d, w.bin_len, w.n_bins, w.meta["cap"],
                                                   capacity=w.n_reads * 2048, stream=s)
        s.synchronize()
        cand_s = time.perf_counter() - t0
        del ref_d
        n_checks = int(cb_d.numel())
        launches = -(-w.n_reads // 262144)
        per_read = torch.diff(co_d)
        ins = [reads_d, offs_d, cb_d, co_d, E_d]
        pass_d = torch.empty(n_checks, dtype=torch.uint8, device="cuda")
        with torch.cuda.stream(s):
            tune = grim.grim_autotune(bank, *ins, pass_out=pass_d, stream=s)
        s.synchronize()
        choice = grim.grim_choose_form(bank, w.n_reads, n_checks)
        scanned = []

        def call():
            _, n_sc = grim.grim_filter_auto(bank, *ins, pass_out=pass_d, stream=s)
            scanned.append(n_sc)

        ms, clk = ctx.timed(call, steps, warmup, clocks=primary)
        ms_g, _ = ctx.timed(lambda: grim.grim_filter_batched(bank, *ins, pass_out=pass_d, tune=tune, stream=s),
                            args.sub_steps, 1)
        nb = min(w.n_reads, 65_536)  # the full scan is timed on one batch of reads
        scan_ins = (reads_d, offs_d[:nb + 1], E_d[:nb])
        res = grim.grim_scan(bank, *scan_ins, cap=1 << 24, stream=s)
        ms_s, _ = ctx.timed(lambda: grim.grim_scan(bank, *scan_ins, out=res, stream=s), 1, 1)
        n_pass = int(torch.count_nonzero(pass_d).item())
        ms_l, _ = ctx.timed(lambda: grim.grim_locate(bank, cb_d, co_d, pass_d, capacity=n_pass, stream=s), 1, 1)
        loc = grim.grim_locate(bank, cb_d, co_d, pass_d, capacity=n_pass, stream=s)
        st, flags = grim.grim_bank_status(bank, s)
        assert st == grim.GRIM_OK, (st, flags)
        units = n_checks
        avg = float(np.mean(ms))
        g, sc, lc = float(np.mean(ms_g)), float(np.mean(ms_s)), float(np.mean(ms_l))
        alg = n_checks * (row + 4 + 1) + int(w.read_offsets[-1]) + (w.n_reads + 1) * 16 + w.n_reads * 2
        peak, peak_kind = load_peaks()
        roof = {"bound": "hbm", "achieved": alg / (avg / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                "frac": alg / (avg / 1e3) / 1e9 / peak, "traffic": None, "peak_source": f"{peak_kind} hbm_gbs",
                "kernel": "dispatcher -> gather_kernel<5,8>", "avg_step_ms": avg}
        out["config_extra"] = {"checks_per_gpu_step": n_checks,
                               "cands_per_read_mean": round(n_checks / w.n_reads, 2),
                               "cands_per_read_max": int(per_read.max().item()),
                               "candidates": "GPU seed table + grim_seed_candidates (12-mer seeds, cap 10000)"}
        out["dispatch"] = {"choice": "scan" if choice == grim.GRIM_FORM_SCAN else "gather",
                           "reads_scanned_per_step": scanned[-1] if scanned else 0}
        out["gather_form"] = {"ms_per_step": g, "checks_per_s": units / (g / 1e3), "reads_per_s": w.n_reads / (g / 1e3)}
        out["scan_form"] = {"ms_per_batch": sc, "batch_reads": nb,
                            "checks_per_s_all_bins": nb * w.n_bins / (sc / 1e3), "reads_per_s": nb / (sc / 1e3),
                            "pairs_passing": res.n_pairs,
                            "note": "one batch of reads timed; the dispatcher's choice runs every read"}
        out["seed_pipeline"] = {"seed_table_s": index_s, "candidates_s": cand_s,
                                "candidates_reads_per_s": w.n_reads / cand_s, "locate_ms": lc,
                                "locations_passing": loc.n,
                                "reads_per_s_serial": w.n_reads / (cand_s + avg / 1e3 + lc / 1e3)}
        out["pass_rate"] = n_pass / max(1, n_checks)
        # the paper's metrics (Sec. 5, 6.1): every passing location aligned
        # against its bin's span; every candidate of the first reads too, to
        # count misses (rejected locations that map)
        ref_d = dev(w.ref2bit)
        ms_v, _ = ctx.timed(lambda: grim.grim_verify(bank, ref_d, reads_d, offs_d, loc.read, loc.bin, stream=s), 1, 1)
        dist = grim.grim_verify(bank, ref_d, reads_d, offs_d, loc.read, loc.bin, stream=s)
        st_pass = grim.grim_verify_stats(dist, loc.read, E_d, stream=s)
        nz = min(w.n_reads, 65_536)
        nz_c = int(co_d[nz].item())
        every = grim.grim_locate(bank, cb_d[:nz_c], co_d[:nz + 1], torch.ones(nz_c, dtype=torch.uint8, device="cuda"),
                                 capacity=nz_c, stream=s)
        dist_all = grim.grim_verify(bank, ref_d, reads_d, offs_d, every.read, every.bin, stream=s)
        st_all = grim.grim_verify_stats(dist_all, every.read, E_d, pass_=pass_d[:nz_c], stream=s)
        out["verification"] = {
            "false_negative_rate": st_pass["passed_unmapped"] / max(1, st_pass["passed"]),
            "locations_passing": st_pass["passed"], "passing_without_mapping": st_pass["passed_unmapped"],
            "average_read_existence": st_pass["passed"] / (w.n_reads * w.n_bins),
            "verify_ms": float(np.mean(ms_v)), "verify_locations_per_s": st_pass["passed"] / (np.mean(ms_v) / 1e3),
            "zero_miss_check": {"reads": nz, "candidates": nz_c, "rejected_with_mapping": st_all["rejected_mapped"],
                                "passing_with_mapping": st_all["passed"] - st_all["passed_unmapped"]},
            "note": "mapping = semi-global edit distance <= E of the read into the bin's span (grim_verify); "
                    "false negative rate in the paper's sense: passing locations without a mapping / passing"}
        del loc, res, ins, cb_d, co_d, dist, dist_all, every  # the end-to-end steps make their own lists
        torch.cuda.empty_cache()
        # the whole path around the filter, alignment overlapping the next
        # batch's filtering (grim_map, 1M-read batches): once to warm, once timed
        align = torch.cuda.Stream()
        cap_loc = int(n_pass * 1.25) + 1024
        with torch.cuda.stream(s):
            grim.grim_map(bank, idx, ref_d, reads_d, offs_d, E_d, cap=w.meta["cap"], batch_reads=1 << 20,
                          capacity=cap_loc, stream=s, align_stream=align)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s):
            mp = grim.grim_map(bank, idx, ref_d, reads_d, offs_d, E_d, cap=w.meta["cap"], batch_reads=1 << 20,
                               capacity=cap_loc, stream=s, align_stream=align)
        torch.cuda.synchronize()
        map_s = time.perf_counter() - t0
        serial_s = cand_s + avg / 1e3 + lc / 1e3 + float(np.mean(ms_v)) / 1e3
        out["seed_pipeline"].update({"overlapped_s": map_s, "overlapped_reads_per_s": w.n_reads / map_s,
                                     "serial_sum_s": serial_s, "overlapped_locations": mp.n,
                                     "overlapped_mapped": int(((mp.dist.to(torch.int32) & 0xFFFF) <= (
                                         E_d.to(torch.int32) & 0xFFFF)[mp.read.long()]).sum().item())})
        del mp, ref_d
        torch.cuda.empty_cache()
        if primary:
            # end to end through the public calls: reads in from pinned host
            # memory, candidates, filter, pass bytes back
            h_in = [ctx.pin(w.bases), ctx.pin(w.read_offsets), ctx.pin(w.E)]
            h_out = torch.empty(n_checks, dtype=torch.uint8).pin_memory()

            def e2e_step():
                for h, d in zip(h_in, (reads_d, offs_d, E_d)):
                    d.copy_(h, non_blocking=True)
                cb2, co2 = grim.grim_seed_candidates(idx, reads_d, offs_d, w.bin_len, w.n_bins, w.meta["cap"],
                                                     capacity=n_checks, stream=s)
                grim.grim_filter_auto(bank, reads_d, offs_d, cb2, co2, E_d, pass_out=pass_d, stream=s)
                h_out.copy_(pass_d, non_blocking=True)

            e2e_ms, _ = ctx.timed(e2e_step, steps, warmup)
            out["e2e"] = {"value": units * ctx.world * steps / (ctx.max_over_ranks(sum(e2e_ms)) / 1e3), "unit": UNIT,
                          "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in h_in),
                          "d2h_bytes_per_step": h_out.numel(),
                          "includes": "seed candidates on the GPU (synchronising), dispatcher, pass bytes to host"}
        idx.free()
        del pass_d, reads_d, offs_d, E_d
        torch.cuda.empty_cache()
    elif form in ("gather", "batched"):
        ins = [dev(w.bases), dev(w.read_offsets), dev(w.cand_bins), dev(w.cand_offsets), dev(w.E)]
        pass_d = torch.empty(w.n_checks, dtype=torch.uint8, device="cuda")
        tune = None
        if form == "batched":
            with torch.cuda.stream(s):
                tune = grim.grim_autotune(bank, *ins, pass_out=pass_d, stream=s)
            s.synchronize()
            call = lambda: grim.grim_filter_batched(bank, *ins, pass_out=pass_d, tune=tune, stream=s)
            launches = -(-w.n_reads // int(tune.batch_reads))
            kernel = f"gather_kernel<{w.q},{int(tune.warps_per_cta)}>"
        else:
            call = lambda: grim.grim_filter(bank, *ins, pass_out=pass_d, stream=s)
            launches = 1
            kernel = f"gather_kernel<{w.q},8>"
        ms, clk = ctx.timed(call, steps, warmup, clocks=primary)
        units = w.n_checks
        alg = gather_bytes(w, row)
        peak, peak_kind = load_peaks()
        avg = float(np.mean(ms))
        roof = {"bound": "hbm", "achieved": alg / (avg / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                "frac": alg / (avg / 1e3) / 1e9 / peak, "traffic": None, "peak_source": f"{peak_kind} hbm_gbs",
                "kernel": kernel, "algorithmic_bytes_per_launch": alg // launches, "launches_per_step": launches,
                "avg_step_ms": avg}
        if form == "gather":
            sha = source_sha()
            roof["source_sha"] = sha
            rec = TRAFFIC_BY_SOURCE.get(sha, {})
            roof["traffic"] = rec.get("bytes") if rec.get("reads") == w.n_reads else None
            if w.q == 5:
                roof["note"] = ("the 50 MB bank stays in the 129 MB L2, so algorithmic bytes exceed DRAM "
                                "traffic; frac counts algorithmic bytes")
        if form == "batched":
            out["tune"] = tune.as_dict()
            ms_plain, _ = ctx.timed(lambda: grim.grim_filter(bank, *ins, pass_out=pass_d, stream=s),
                                    args.sub_steps, 2)
            ap = float(np.mean(ms_plain))
            out["plain_gather_same_workload"] = {
                "value": units * ctx.world * len(ms_plain) / (ctx.max_over_ranks(sum(ms_plain)) / 1e3),
                "ms_per_step": ap, "frac": alg / (ap / 1e3) / 1e9 / peak}
        st, flags = grim.grim_bank_status(bank, s)
        assert st == grim.GRIM_OK, (st, flags)
        out["pass_rate"] = float(pass_d.float().mean().item())
        if primary:
            # end to end through grim_filter_host: page-locked host buffers in,
            # chunks copied in / filtered / copied out on overlapping streams
            h_in = [ctx.pin(w.bases), ctx.pin(w.read_offsets), ctx.pin(w.cand_bins), ctx.pin(w.cand_offsets),
                    ctx.pin(w.E)]
            h_out = torch.empty(w.n_checks, dtype=torch.uint8).pin_memory()

            def e2e_step():
                grim.grim_filter_host(bank, *h_in, pass_out=h_out, stream=s)

            e2e_ms, _ = ctx.timed(e2e_step, steps, warmup)
            assert torch.equal(h_out, pass_d.cpu()), "grim_filter_host differs from the device call"
            out["e2e"] = {"value": units * ctx.world * steps / (ctx.max_over_ranks(sum(e2e_ms)) / 1e3), "unit": UNIT,
                          "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in h_in),
                          "d2h_bytes_per_step": h_out.numel(), "call": "grim_filter_host (host buffers)"}
            if ctx.rank == 0 and ctx.world == 1 and not args.no_cpu_baseline:
                out["cpu_baseline"] = cpu_baseline_filter(w, args.cpu_seconds)
        del ins, pass_d
    else:
        ins = [dev(w.bases), dev(w.read_offsets), dev(w.E)]
        cap = 1 << 24
        res = grim.grim_scan(bank, *ins, cap=cap, stream=s)
        call = lambda: grim.grim_scan(bank, *ins, out=res, stream=s)
        ms, clk = ctx.timed(call, steps, warmup, clocks=primary)
        st, flags = grim.grim_bank_status(bank, s)
        assert st == grim.GRIM_OK, (st, flags)
        n_pairs = res.n_pairs
        units = w.n_reads * w.n_bins
        launches = 2  # scan_prep_kernel + scan_kernel
        avg = float(np.mean(ms))
        flops = 2.0 * units * (4 ** w.q)
        peak, peak_sust, src = load_fp8_peak()
        roof = {"bound": "tensor", "achieved": flops / (avg / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": flops / (avg / 1e3) / 1e12 / peak, "traffic": None,
                "peak_source": f"{src} (e4m3 dense), burst", "kernel": f"scan_kernel<{w.q}> (+ scan_prep_kernel)",
                "algorithmic_flops_per_launch": flops, "avg_step_ms": avg,
                "frac_of_sustained": flops / (avg / 1e3) / 1e12 / peak_sust}
        out["pairs_passing"] = n_pairs
        if primary:
            h_in = [ctx.pin(w.bases), ctx.pin(w.read_offsets), ctx.pin(w.E)]
            h_read = torch.empty(n_pairs + 1, dtype=torch.int32).pin_memory()
            h_bin = torch.empty(n_pairs + 1, dtype=torch.int32).pin_memory()
            h_n = torch.empty(1, dtype=torch.int64).pin_memory()

            def e2e_step():
                for h, d in zip(h_in, ins):
                    d.copy_(h, non_blocking=True)
                call()
                h_n.copy_(res.n_pairs_dev, non_blocking=True)
                h_read.copy_(res.pair_read[:n_pairs + 1], non_blocking=True)
                h_bin.copy_(res.pair_bin[:n_pairs + 1], non_blocking=True)

            e2e_ms, _ = ctx.timed(e2e_step, steps, warmup)
            out["e2e"] = {"value": units * ctx.world * steps / (ctx.max_over_ranks(sum(e2e_ms)) / 1e3), "unit": UNIT,
                          "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in h_in),
                          "d2h_bytes_per_step": 8 + 8 * (n_pairs + 1)}
        if ctx.rank == 0 and ctx.world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_scan(w)
        del ins, res
    total_ms = ctx.max_over_ranks(float(sum(ms)))
    out.update({"value": units * ctx.world * steps / (total_ms / 1e3), "unit": UNIT,
                "reads_per_s": w.n_reads * ctx.world * steps / (total_ms / 1e3), "ms_per_step": total_ms / steps,
                "steps": steps, "roofline": roof, "gpu_launches": launches * steps, "clocks": clk,
                "bank_build": bank_info, "config": describe(form, w)})
    out["config"].update(out.pop("config_extra", {}))
    bank.free()
    del w
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    grim.grim_release_scratch()
    return out


def q_sweep(args, ctx):
    """Token sizes 4-6 on the same 100 Mbp reads and seed candidates (the
    paper sweeps them in Sec. 6.1): bank size and build time, gather time,
    checks/s, fraction of HBM and the share of candidates that pass."""
    import torch

    import paper_1711_01177_gb300 as grim
    import synth
    w = synth.gather_seeds(ref_len=args.ref_bp, n_reads=args.q_sweep_reads,
                           read_seed=synth.SEED_READS + 1000 * ctx.rank + 7)
    dev, s = ctx.dev, ctx.stream
    ref_d = dev(w.ref2bit)
    ins = [dev(w.bases), dev(w.read_offsets), dev(w.cand_bins), dev(w.cand_offsets), dev(w.E)]
    pass_d = torch.empty(w.n_checks, dtype=torch.uint8, device="cuda")
    peak, _ = load_peaks()
    out = {"workload": f"{args.ref_bp / 1e6:g} Mbp repeat-rich reference, {w.n_reads} x 150 bp reads, "
                       f"12-mer seed candidates ({w.n_checks} checks), E = 7 for every q", "by_q": {}}
    for q in (4, 5, 6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            e0.record(s)
            bank = grim.grim_build_bank(ref_d, w.ref_len, q, w.bin_len, w.overlap, stream=s)
            e1.record(s)
        s.synchronize()
        ms, _ = ctx.timed(lambda: grim.grim_filter(bank, *ins, pass_out=pass_d, stream=s), args.sub_steps, 2)
        st, flags = grim.grim_bank_status(bank, s)
        assert st == grim.GRIM_OK, (st, flags)
        avg = float(np.mean(ms))
        row = bank.row_words * 4
        alg = gather_bytes(w, row)
        out["by_q"][str(q)] = {"bank_bytes": bank.n_bins * row, "bank_build_ms": e0.elapsed_time(e1),
                               "ms_per_step": avg, "checks_per_s": w.n_checks / (avg / 1e3),
                               "hbm_frac": alg / (avg / 1e3) / 1e9 / peak,
                               "pass_rate": float(pass_d.float().mean().item())}
        bank.free()
    del ins, pass_d, ref_d
    torch.cuda.empty_cache()
    return out


# --------------------------------------------------------------- CPU oracle

def cpu_baseline_filter(w, seconds):
    """The oracle, single-threaded, on the first reads of the same workload."""
    import oracle
    o = oracle.Oracle()
    t0 = time.perf_counter()
    ob = o.build_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    t_bank = time.perf_counter() - t0

    def run(n):
        co, ro = w.cand_offsets[:n + 1], w.read_offsets[:n + 1]
        t = time.perf_counter()
        o.filter(ob, w.q, w.bases[:ro[-1]], ro, w.cand_bins[:co[-1]], co, w.E[:n])
        return time.perf_counter() - t, int(co[-1])

    dt, nc = run(min(500, w.n_reads))
    n = min(w.n_reads, max(500, int(500 * seconds / max(dt, 1e-6))))
    dt, nc = run(n)
    return {"value": nc / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n} reads ({nc} checks) of the same workload, oracle bank prebuilt "
                      f"({t_bank:.1f} s, not timed), single thread",
            "reads_per_s": n / dt, "seconds": round(dt, 2)}


def cpu_baseline_rows(w, seconds):
    """The oracle on a genome-scale candidate list: each candidate's bitvector
    built straight from the reference (oracle_bin_row), then summed
    (oracle_sum_one); single-threaded, on the first candidates of the same
    workload (a byte-per-bit oracle bank of 12.1M bins would not fit)."""
    import oracle
    o = oracle.Oracle()
    t0 = time.perf_counter()
    done = 0
    r = 0
    while time.perf_counter() - t0 < seconds and r < w.n_reads:
        read = w.bases[w.read_offsets[r]:w.read_offsets[r + 1]]
        for c in range(w.cand_offsets[r], w.cand_offsets[r + 1]):
            row = o.bin_row(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap, int(w.cand_bins[c]))
            o.sum_one(row, w.q, read)
            done += 1
        r += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {r} reads ({done} checks) of the same workload, rows built per check, single thread",
            "seconds": round(dt, 2)}


def cpu_baseline_scan(w, n_reads=64, n_bins=20_000):
    """The oracle's full scan, single-threaded, on the first reads x the first
    bins of the same workload (the oracle bank of a reference prefix: its
    first n_bins bins equal the full reference's)."""
    import oracle
    import synth
    o = oracle.Oracle()
    prefix = n_bins * w.bin_len + w.overlap
    ob = o.build_bank(synth.pack2bit(w.codes[:prefix]), prefix, w.q, w.bin_len, w.overlap)[:n_bins]
    t = time.perf_counter()
    o.scan(ob, w.q, w.bases[:w.read_offsets[n_reads]], w.read_offsets[:n_reads + 1], w.E[:n_reads])
    dt = time.perf_counter() - t
    return {"value": n_reads * n_bins / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n_reads} reads x first {n_bins} bins of the same workload, single thread",
            "seconds": round(dt, 2)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    per_step = min(20.0, max(0.05, args.ref_seconds / max(1, args.steps + args.warmup)))
    o = oracle.Oracle()
    if args.workload == "fullscan":
        import synth
        w = make_fullscan(args, 0)
        nb = 20_000
        prefix = nb * w.bin_len + w.overlap
        ob = o.build_bank(synth.pack2bit(w.codes[:prefix]), prefix, w.q, w.bin_len, w.overlap)[:nb]

        def step(n):
            t = time.perf_counter()
            o.scan(ob, w.q, w.bases[:w.read_offsets[n]], w.read_offsets[:n + 1], w.E[:n])
            return time.perf_counter() - t, n * nb

        sample = f"first n reads x first {nb} bins per step"
    elif args.workload == "mixed":
        w = make_mixed(args, 0, cand_reads=4096)

        def step(n):
            t = time.perf_counter()
            done = 0
            for r in range(n):
                read = w.bases[w.read_offsets[r]:w.read_offsets[r + 1]]
                for c in range(w.cand_offsets[r], w.cand_offsets[r + 1]):
                    o.sum_one(o.bin_row(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap, int(w.cand_bins[c])),
                              w.q, read)
                    done += 1
            return time.perf_counter() - t, done

        sample = "first n reads per step, rows built per check"
    else:
        w = make_gather(args, 0) if args.workload == "gather" else make_batched(args, 0)
        ob = o.build_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)

        def step(n):
            co, ro = w.cand_offsets[:n + 1], w.read_offsets[:n + 1]
            t = time.perf_counter()
            o.filter(ob, w.q, w.bases[:ro[-1]], ro, w.cand_bins[:co[-1]], co, w.E[:n])
            return time.perf_counter() - t, int(co[-1])

        sample = "first n reads per step"
    dt, _ = step(16)
    n_max = w.n_reads if w.cand_offsets is None else len(w.cand_offsets) - 1
    n = min(n_max, max(16, int(16 * per_step / max(dt, 1e-6))))
    for _ in range(args.warmup):
        step(n)
    times, units = [], 0
    for _ in range(args.steps):
        dt, u = step(n)
        times.append(dt)
        units += u
    value = units / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": describe(args.workload, w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample.replace("n reads", f"{n} reads") + ", single thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1711_01177_gb300 as grim

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    grim.build()
    grim.load()
    ctx = Ctx(rank, world, local)
    main_form = run_form(args.workload, args, ctx, primary=True)
    subs = {}
    if args.workload != "batched" and not args.no_batched:
        subs["batched"] = run_form("batched", args, ctx, primary=False)
    if args.workload != "fullscan" and not args.no_full_scan:
        subs["full_scan"] = run_form("fullscan", args, ctx, primary=False)
    if args.workload != "mixed" and not args.no_mixed:
        subs["mixed"] = run_form("mixed", args, ctx, primary=False)
    if not args.no_q_sweep:
        subs["q_sweep"] = q_sweep(args, ctx)
    if rank == 0:
        m = main_form
        line = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "e4m3" if args.workload == "fullscan" else "u32",
                "data": "synthetic",
                "config": dict(m["config"], parallelism=f"replicas x{world} (read batches per GPU, no collective)"),
                "reads_per_s": m["reads_per_s"], "roofline": m["roofline"], "e2e": m["e2e"],
                "gpu_launches": m["gpu_launches"], "clocks": m["clocks"], "cpu_baseline": m.get("cpu_baseline"),
                "bank_build": m["bank_build"]}
        for k in ("pass_rate", "tune", "plain_gather_same_workload", "pairs_passing", "dispatch", "gather_form",
                  "scan_form"):
            if k in m:
                line[k] = m[k]
        for k, v in subs.items():
            line[k] = {kk: vv for kk, vv in v.items() if kk != "clocks"}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    # ranks on one host share its cores for the synthetic inputs (OpenMP)
    local_world = int(os.environ.get("LOCAL_WORLD_SIZE", os.environ.get("WORLD_SIZE", "1")))
    if local_world > 1 and "OMP_NUM_THREADS" not in os.environ:
        os.environ["OMP_NUM_THREADS"] = str(max(1, (os.cpu_count() or 1) // local_world))
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
