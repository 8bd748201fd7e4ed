"""Benchmark of the seed-location filter on GB300.

Five synthetic workloads, each timed with the form of the hot path it is
meant for (inputs resident in HBM, L2 flushed between timed steps):
  1 plain gather, 1 Mbp: i.i.d. reference, q=5, 256 bp bins + 100 bp
           overlap; 10,000 reads of 100 bp (3% substitutions, 1% indels),
           E=5; the true bin + 31 uniform candidates.  Step: grim_filter.
  2 gather at scale, 100 Mbp: 70% i.i.d. + 30% planted repeat families at
           10-20% divergence, q=5, 256 + 150 bp; 1M reads of 150 bp (4% + 1%),
           E=7; bins of all exact 12-mer seed hits, capped at 1,000.
           Step: grim_filter.
  3 full scan, 3.1 Gbp: same mixture, q=5, 256 + 100 bp (12.1M bins); a
           batch of 65,536 reads of 100 bp, E=5, every bin scored on the
           tensor cores.  Step: grim_scan.
  4 batching, 100 Mbp, q=6, 256 + 300 bp; 2M reads of 50-300 bp (3% + 1%),
           E = floor(0.05 L); true bin + log-uniform 1-5,000 candidates.
           Step: grim_filter_batched (one launch per 262,144 reads in a
           replayed CUDA graph, autotuned launch shape).
  5 human-scale mixed, 3.1 Gbp, 40% repeats at 5-20% divergence, q=5,
           256 + 100 bp; 10M reads of 100 bp, E=5; 12-mer seed candidates
           built on the GPU, capped at 10,000.  Step: grim_filter_auto (the
           per-batch choice between the gather form and the full scan).
The default JSON line is workload 5 (the largest single-GPU configuration);
the other four are measured after it and summarised in the `configs` key,
the line's last.  The bank is built once per reference beforehand (the paper
also leaves bitvector generation out of its runtime, Sec. 6.1) and timed on
its own.  Roofline denominators: the measured HBM copy bandwidth
(MEASURED_PEAKS.json) and, measured here by the library's own kernels, the
L2 read bandwidth and the dense tensor rates (grim_peak).

--impl reference times the CPU oracle on bounded samples of the same
workload instead, on every host core.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "(read,bin) checks/s & reads/s at E=0.05·L; frac of HBM/INT8 roofline vs plain"
UNIT = "checks/s"
L2_FLUSH_BYTES = 256 << 20
CONFIG_OF_FORM = {"plain": "1", "gather": "2", "fullscan": "3", "batched": "4", "mixed": "5"}
SUMMARY_KEY = {"plain": "1_plain_1Mbp", "gather": "2_gather_100Mbp", "fullscan": "3_fullscan_3.1Gbp",
               "batched": "4_batched_q6_100Mbp", "mixed": "5_mixed_3.1Gbp"}

# dram__bytes_read.sum + dram__bytes_write.sum of one gather launch, from an
# ncu capture, valid only for the kernel source it was taken on:
# {source hash: {form: {"bytes": per launch, "reads": reads per launch,
#                       "checks": checks of the launch where it is scaled by checks}}}
TRAFFIC_BY_SOURCE: dict[str, dict] = {
    "1577e08671b4a735": {
        # gather_kernel<5,4,DEEP>, one 262,144-read batch of the 3.1 Gbp dispatcher
        # workload, 438,575,706 checks: 54,668,177,664 B read + 440,018,176 B written
        "mixed": {"bytes": 55_108_195_840, "reads": 262_144, "checks": 438_575_706},
        # gather_kernel<5,8>, 100 Mbp, 1M reads, 74.8M checks: 655,405,568 B read + 71,852,544 B written
        "gather": {"bytes": 727_258_112, "reads": 1_000_000},
        # gather_kernel<5,8>, 1 Mbp, 10,000 reads, 320,000 checks: 3,017,216 B read, the output stays in L2
        "plain": {"bytes": 3_017_216, "reads": 10_000},
        # gather_kernel<6,8>, one 262,144-read batch of the q=6 workload, 153,942,833 checks:
        # 47,292,314,112 B read + 163,915,776 B written
        "batched": {"bytes": 47_456_229_888, "reads": 262_144, "checks": 153_942_833},
    },
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed", choices=["plain", "gather", "batched", "fullscan", "mixed"])
    ap.add_argument("--plain-ref-bp", type=int, default=1_000_000)
    ap.add_argument("--plain-reads", type=int, default=10_000)
    ap.add_argument("--reads", type=int, default=1_000_000, help="gather: reads per GPU (weak scaling)")
    ap.add_argument("--ref-bp", type=int, default=100_000_000, help="gather / batched: reference length")
    ap.add_argument("--batched-reads", type=int, default=2_000_000)
    ap.add_argument("--scan-ref-bp", type=int, default=3_100_000_000, help="full scan / mixed: reference length")
    ap.add_argument("--scan-reads", type=int, default=65_536)
    ap.add_argument("--mixed-reads", type=int, default=10_000_000)
    ap.add_argument("--sub-steps", type=int, default=3, help="timed steps of the other workloads")
    ap.add_argument("--only", action="store_true", help="measure the --workload line alone")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=3.0, help="CPU time of each oracle sample leg")
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="--impl reference: target wall time of the whole run (warm-up + timed steps)")
    ap.add_argument("--no-q-sweep", action="store_true", help="skip the token-size sweep (q = 4, 5, 6)")
    ap.add_argument("--q-sweep-reads", type=int, default=262_144)
    ap.add_argument("--no-extras", action="store_true",
                    help="workload 5: skip the verification metrics and the overlapped pipeline")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def load_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["hbm_gbs"]), "measured hbm_gbs (MEASURED_PEAKS.json)"
    return 6800.0, "fallback hbm 6.8 TB/s"


def source_sha(files=("gather.cu", "grim_internal.cuh", "tokens.cuh")):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1711_01177_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def sig(x, n=4):
    """x rounded to n significant digits (compact JSON)."""
    if x is None or not isinstance(x, (int, float)) or x == 0 or not np.isfinite(x):
        return x
    return float(f"{x:.{n}g}")


def cpu_info():
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"cpu_model": model, "nproc": os.cpu_count() or 1}


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

def make_workload(form, args, rank, cand_reads=0):
    import synth
    rs = synth.SEED_READS + 1000 * rank
    if form == "plain":
        return synth.gather_iid(ref_len=args.plain_ref_bp, n_reads=args.plain_reads)
    if form == "gather":
        return synth.gather_seeds(ref_len=args.ref_bp, n_reads=args.reads, read_seed=rs)
    if form == "batched":
        return synth.batched_varlen(ref_len=args.ref_bp, n_reads=args.batched_reads, read_seed=rs)
    if form == "fullscan":
        return synth.fullscan(ref_len=args.scan_ref_bp, n_reads=args.scan_reads, read_seed=rs)
    # candidates come from the GPU seed table; cand_reads > 0 also builds CPU
    # lists for the first reads (the oracle's sample)
    return synth.mixed_seeds(ref_len=args.scan_ref_bp, n_reads=args.mixed_reads, read_seed=rs, cand_reads=cand_reads)


def describe(form, w, world=1):
    """The workload's defining parameters (identical for both arms)."""
    L = np.diff(w.read_offsets)
    base = {"ref_bp": w.ref_len, "q": w.q, "bin_len": w.bin_len, "overlap": w.overlap, "n_bins": w.n_bins,
            "reads_per_gpu": w.n_reads, "read_len": [int(L.min()), int(L.max())],
            "E": [int(w.E.min()), int(w.E.max())], "sub": w.meta["sub"], "indel": w.meta["indel"],
            "repeat_frac": w.meta["repeat_frac"],
            "l2": "flushed between timed steps (256 MiB write, outside the events)",
            "parallelism": f"replicas x{world} (read batches per GPU, no collective)"}
    rep = f"{int(w.meta['repeat_frac'] * 100)}% repeats"
    if form == "plain":
        wl = (f"plain gather, {w.ref_len / 1e6:g} Mbp i.i.d. reference, q={w.q}, {w.n_reads} x {int(L[0])} bp "
              f"reads/GPU, true bin + 31 uniform candidates")
    elif form == "gather":
        wl = (f"gather, {w.ref_len / 1e6:g} Mbp repeat-rich reference ({rep}), q={w.q}, {w.n_reads} x {int(L[0])} "
              f"bp reads/GPU, 12-mer seed candidates (cap 1000)")
    elif form == "batched":
        wl = (f"batched gather, {w.ref_len / 1e6:g} Mbp repeat-rich reference ({rep}), q={w.q}, {w.n_reads} reads "
              f"of {int(L.min())}-{int(L.max())} bp/GPU, E=floor(0.05 L), log-uniform 1-5000 candidates")
    elif form == "mixed":
        wl = (f"dispatcher, {w.ref_len / 1e9:g} Gbp reference ({rep} at 5-20% divergence), q={w.q}, {w.n_reads} x "
              f"{int(L[0])} bp reads/GPU, 12-mer seed candidates from the GPU seed table (cap 10000), gather vs full "
              f"scan chosen per batch")
    else:
        wl = (f"full scan, {w.ref_len / 1e9:g} Gbp repeat-rich reference ({rep}), q={w.q}, {w.n_bins} bins, batch "
              f"of {w.n_reads} x {int(L[0])} bp reads/GPU, every bin")
    base["workload"] = wl
    return base


def gather_bytes(n_checks, w, row_bytes):
    """Bytes one gather pass must move: per check the bin row, the candidate
    id and the pass byte; per read its bases, two offsets and E."""
    return n_checks * (row_bytes + 4 + 1) + int(w.read_offsets[-1]) + (w.n_reads + 1) * 16 + w.n_reads * 2


# --------------------------------------------------------------- CPU oracle

def oracle_rate(run_chunk, n_max, seconds, threads):
    """run_chunk(a, b) runs the oracle on units [a, b) and returns the checks
    done; the oracle's C calls release the GIL, so a thread pool runs them on
    `threads` cores.  Calibrated on a small prefix, the sample is sized for
    about `seconds` of wall time and cut into chunks that the threads take in
    turn.  Returns (checks/s, units used, checks, seconds)."""
    n0 = min(n_max, 8)
    t = time.perf_counter()
    run_chunk(0, n0)
    per = max((time.perf_counter() - t) / n0, 1e-7)
    n = int(min(n_max, max(threads, seconds * threads / per)))
    edges = np.unique(np.linspace(0, n, min(n, 8 * threads) + 1).astype(np.int64))
    t = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        done = sum(ex.map(lambda ab: run_chunk(int(ab[0]), int(ab[1])), zip(edges[:-1], edges[1:])))
    dt = time.perf_counter() - t
    return done / dt, n, done, dt


def oracle_sampler(form, w, sample_reads=16_384):
    """(run_chunk, n_max, what) for the oracle on this workload: read ranges
    [a, b) through the byte-per-bit bank (built beforehand, untimed), or, at
    genome scale, with each candidate's bitvector rebuilt from the reference
    (oracle_filter_rows), or the full scan over the first 20,000 bins."""
    import oracle
    import synth
    o = oracle.Oracle()
    ro, bases = w.read_offsets, w.bases
    if form == "fullscan":
        nb = 20_000
        prefix = nb * w.bin_len + w.overlap
        ob = o.build_bank(synth.pack2bit(w.codes[:prefix]), prefix, w.q, w.bin_len, w.overlap)[:nb]

        def run(a, b):
            o.scan(ob, w.q, bases[ro[a]:ro[b]], ro[a:b + 1] - ro[a], w.E[a:b])
            return (b - a) * nb

        return run, w.n_reads, f"reads x the first {nb} bins"
    if form == "mixed":
        if w.cand_offsets is None or len(w.cand_offsets) - 1 < min(sample_reads, w.n_reads):
            m = min(sample_reads, w.n_reads)
            sub_off = ro[:m + 1]
            idx = synth.seed_index_for_reads(w.codes, bases[:sub_off[-1]], sub_off, w.meta["seed_k"])
            cb, co = synth.cands_seeds(idx, bases[:sub_off[-1]], sub_off, w.bin_len, w.n_bins, w.meta["cap"],
                                       w.meta["seed_k"])
            del idx
        else:
            cb, co = w.cand_bins, w.cand_offsets

        def run(a, b):
            o.filter_rows(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap, bases[ro[a]:ro[b]], ro[a:b + 1],
                          cb[co[a]:co[b]], co[a:b + 1], w.E[a:b])
            return int(co[b] - co[a])

        return run, len(co) - 1, "reads (CPU seed candidates), each candidate's bitvector rebuilt from the reference"
    ob = o.build_bank(w.ref2bit, w.ref_len, w.q, w.bin_len, w.overlap)
    cb, co = w.cand_bins, w.cand_offsets

    def run(a, b):
        o.filter(ob, w.q, bases[ro[a]:ro[b]], ro[a:b + 1] - ro[a], cb[co[a]:co[b]], co[a:b + 1] - co[a], w.E[a:b])
        return int(co[b] - co[a])

    return run, w.n_reads, "reads, oracle bank prebuilt (not timed)"


def cpu_baseline(form, w, seconds):
    """The oracle on a bounded sample of the same workload: single-threaded,
    then on every host core."""
    run, n_max, what = oracle_sampler(form, w)
    info = cpu_info()
    v1, n1, c1, t1 = oracle_rate(run, n_max, seconds, 1)
    vn, nn, cn, tn = oracle_rate(run, n_max, seconds, info["nproc"])
    return {"value": vn, "unit": UNIT, "cores": info["nproc"], "kind": "oracle",
            "sample": f"first {nn} {what}: {cn} checks in {tn:.1f} s on {info['nproc']} threads; single thread: "
                      f"first {n1}, {c1} checks in {t1:.1f} s",
            "single_thread": v1, "cpu_model": info["cpu_model"], "nproc": info["nproc"]}


# --------------------------------------------------------------- GPU context

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

    def timed(self, fn, steps, warmup, clocks=True):
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


def measure_peaks(ctx):
    """Roofline denominators: the driver's HBM copy figure and, measured
    here by the library's kernels, the L2 read bandwidth, the dense tensor
    rates (burst: one launch of a few ms; sustained: launches back to back
    for about a second) and the legacy mma.sync INT8 rate."""
    import paper_1711_01177_gb300 as grim
    hbm, hbm_src = load_hbm_peak()
    out = {"hbm_gbs": hbm, "hbm_source": hbm_src}

    def best(kind, work, n=3):
        r = [grim.grim_peak(kind, work, stream=ctx.stream) for _ in range(n)]
        return max(u / (ms / 1e3) for u, ms in r)

    out["l2_read_gbs"] = best(grim.GRIM_PEAK_L2_READ, 32 << 20) / 1e9
    for name, kind, work in (("e4m3", grim.GRIM_PEAK_E4M3, 65536), ("mxf4", grim.GRIM_PEAK_MXF4, 131072),
                             ("e4m3_tmem_a", grim.GRIM_PEAK_E4M3_TMEM_A, 65536),
                             ("mxf4_tmem_a", grim.GRIM_PEAK_MXF4_TMEM_A, 131072)):
        out[f"{name}_tflops"] = best(kind, work) / 1e12
    # sustained: the full scan's kind for about a second, the last launches
    t0, rates = time.perf_counter(), []
    while time.perf_counter() - t0 < 1.0:
        u, ms = grim.grim_peak(grim.GRIM_PEAK_MXF4_TMEM_A, 1 << 20, stream=ctx.stream)
        rates.append(u / (ms / 1e3))
    out["mxf4_tmem_a_tflops_sustained"] = float(np.median(rates[len(rates) // 2:])) / 1e12
    out["int8_mma_sync_tops"] = best(grim.GRIM_PEAK_INT8_MMA_SYNC, 4000) / 1e12
    # this box's copy bandwidth, taken the way the HBM figure above was
    # (b.copy_(a) over 1 Gi bf16 elements, read + write bytes, best of 10):
    # context for the spread of DRAM-bound lines between boxes; the
    # roofline keeps hbm_gbs
    import torch
    a = torch.empty(1 << 30, dtype=torch.bfloat16, device="cuda")
    b = torch.empty_like(a)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bw = []
    with torch.cuda.stream(ctx.stream):
        for _ in range(10):
            e0.record(ctx.stream)
            b.copy_(a)
            e1.record(ctx.stream)
            ctx.stream.synchronize()
            bw.append(4.0 * a.numel() / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del a, b
    out["hbm_copy_gbs_this_box"] = max(bw)
    out["how"] = ("grim_peak: L2 = 32 MiB read 40x with ld.global.cg.v4 on every SM; tensor = one CTA per SM "
                  "issuing dense tcgen05.mma 128x256 (e4m3 K=32 / mxf4 e2m1 K=64, unit scales) back to back, "
                  "operands in shared (or A in tensor) memory; best of 3 launches; int8 = mma.sync m16n8k32 s8; "
                  "hbm_copy_gbs_this_box = torch copy on this box")
    return {k: (sig(v) if isinstance(v, float) else v) for k, v in out.items()}


# --------------------------------------------------------------- one form

def build_bank_timed(grim, ctx, w):
    """Builds the bank once; the build kernel's time is taken on a second
    build into the same bank (grim_build_bank_into), which allocates nothing."""
    import torch
    s = ctx.stream
    ref_d = ctx.dev(w.ref2bit)
    with torch.cuda.stream(s):
        bank = grim.grim_build_bank(ref_d, w.ref_len, w.q, w.bin_len, w.overlap, stream=s)
    ms, _ = ctx.timed(lambda: grim.grim_build_bank_into(bank, ref_d, stream=s), 3, 1, clocks=False)
    st, flags = grim.grim_bank_status(bank, s)
    assert st == grim.GRIM_OK, (st, flags)
    row = bank.row_words * 4
    alg = bank.n_bins * row + len(w.ref2bit)
    m = float(np.median(ms))
    hbm, _ = load_hbm_peak()
    info = {"ms": sig(m), "mbp_per_s": sig(w.ref_len / 1e6 / (m / 1e3)), "gb_per_s": sig(alg / 1e9 / (m / 1e3)),
            "hbm_frac": sig(alg / 1e9 / (m / 1e3) / hbm, 3), "bank_bytes": bank.n_bins * row,
            "algorithmic_bytes": alg}
    del ref_d
    return bank, info


def finish(out, form, ctx, w, units, ms, steps, roof, launches, clk, bank_info):
    total_ms = ctx.max_over_ranks(float(sum(ms)))
    out.update({"value": units * ctx.world * steps / (total_ms / 1e3), "unit": UNIT,
                "reads_per_s": w.n_reads * ctx.world * steps / (total_ms / 1e3), "ms_per_step": total_ms / steps,
                "steps": steps, "roofline": roof, "gpu_launches": launches * steps, "clocks": clk,
                "bank_build": bank_info})
    return out


def run_plain_or_gather(form, args, ctx, primary, peaks):
    import torch

    import paper_1711_01177_gb300 as grim
    w = make_workload(form, args, ctx.rank)
    steps = args.steps if primary else args.sub_steps
    warmup = args.warmup if primary else 2
    bank, bank_info = build_bank_timed(grim, ctx, w)
    s = ctx.stream
    ins = [ctx.dev(w.bases), ctx.dev(w.read_offsets), ctx.dev(w.cand_bins), ctx.dev(w.cand_offsets), ctx.dev(w.E)]
    pass_d = torch.empty(w.n_checks, dtype=torch.uint8, device="cuda")
    ms, clk = ctx.timed(lambda: grim.grim_filter(bank, *ins, pass_out=pass_d, stream=s), steps, warmup)
    st, flags = grim.grim_bank_status(bank, s)
    assert st == grim.GRIM_OK, (st, flags)
    row = bank.row_words * 4
    alg = gather_bytes(w.n_checks, w, row)
    avg = float(np.mean(ms))
    ach = alg / (avg / 1e3) / 1e9
    hbm, hbm_src = load_hbm_peak()
    bank_bytes = bank.n_bins * row
    roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": None,
            "peak_source": hbm_src, "kernel": f"gather_kernel<{w.q},8>", "algorithmic_bytes_per_launch": alg,
            "launches_per_step": 1, "avg_step_ms": avg}
    sha = source_sha()
    rec = TRAFFIC_BY_SOURCE.get(sha, {}).get(form, {})
    roof["source_sha"] = sha
    roof["traffic"] = rec.get("bytes") if rec.get("reads") == w.n_reads else None
    if bank_bytes < 100e6 and peaks.get("l2_read_gbs"):
        roof["l2_frac"] = ach / peaks["l2_read_gbs"]
        roof["l2_peak"] = peaks["l2_read_gbs"]
        roof["note"] = (f"the {bank_bytes / 1e6:.1f} MB bank stays in the 129 MB L2: frac counts algorithmic bytes "
                        f"against HBM, l2_frac against the measured L2 read bandwidth")
        roof["summary_frac"], roof["summary_peak"] = roof["l2_frac"], "measured l2_read_gbs"
    out = {"form": form, "pass_rate": float(pass_d.float().mean().item()),
           "workload_stats": {"checks_per_gpu_step": w.n_checks,
                              "cands_per_read_mean": round(w.n_checks / w.n_reads, 2),
                              "cands_per_read_max": int(np.diff(w.cand_offsets).max())}}
    if primary:
        # end to end through grim_filter_host: page-locked host buffers in,
        # chunks copied in / filtered / copied out on overlapping streams
        h_in = [ctx.pin(w.bases), ctx.pin(w.read_offsets), ctx.pin(w.cand_bins), ctx.pin(w.cand_offsets),
                ctx.pin(w.E)]
        h_out = torch.empty(w.n_checks, dtype=torch.uint8).pin_memory()
        e2e_ms, _ = ctx.timed(lambda: grim.grim_filter_host(bank, *h_in, pass_out=h_out, stream=s), steps, warmup,
                              clocks=False)
        assert torch.equal(h_out, pass_d.cpu()), "grim_filter_host differs from the device call"
        out["e2e"] = {"value": w.n_checks * ctx.world * steps / (ctx.max_over_ranks(sum(e2e_ms)) / 1e3),
                      "unit": UNIT, "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in h_in),
                      "d2h_bytes_per_step": h_out.numel(), "call": "grim_filter_host (host buffers)"}
    if ctx.rank == 0 and ctx.world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(form, w, args.cpu_seconds)
    del ins, pass_d
    bank.free()
    return finish(out, form, ctx, w, w.n_checks, ms, steps, roof, 1, clk, bank_info), w


def run_batched(args, ctx, primary, peaks):
    import torch

    import paper_1711_01177_gb300 as grim
    form = "batched"
    w = make_workload(form, args, ctx.rank)
    steps = args.steps if primary else args.sub_steps
    warmup = args.warmup if primary else 2
    bank, bank_info = build_bank_timed(grim, ctx, w)
    s = ctx.stream
    ins = [ctx.dev(w.bases), ctx.dev(w.read_offsets), ctx.dev(w.cand_bins), ctx.dev(w.cand_offsets), ctx.dev(w.E)]
    pass_d = torch.empty(w.n_checks, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(s):
        tune = grim.grim_autotune(bank, *ins, pass_out=pass_d, stream=s)
    s.synchronize()
    ms, clk = ctx.timed(lambda: grim.grim_filter_batched(bank, *ins, pass_out=pass_d, tune=tune, stream=s), steps,
                        warmup)
    launches = -(-w.n_reads // int(tune.batch_reads))
    ms_plain, _ = ctx.timed(lambda: grim.grim_filter(bank, *ins, pass_out=pass_d, stream=s), args.sub_steps, 2,
                            clocks=False)
    st, flags = grim.grim_bank_status(bank, s)
    assert st == grim.GRIM_OK, (st, flags)
    row = bank.row_words * 4
    alg = gather_bytes(w.n_checks, w, row)
    avg, ap = float(np.mean(ms)), float(np.mean(ms_plain))
    hbm, hbm_src = load_hbm_peak()
    ach = alg / (avg / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": None,
            "peak_source": hbm_src, "kernel": f"gather_kernel<{w.q},{int(tune.warps_per_cta)}>",
            "algorithmic_bytes_per_launch": alg // launches, "launches_per_step": launches, "avg_step_ms": avg}
    sha = source_sha()
    rec = TRAFFIC_BY_SOURCE.get(sha, {}).get(form, {})
    roof["source_sha"] = sha
    if rec.get("reads"):
        # measured on one batch launch; scaled to the average launch by checks
        roof["traffic"] = int(rec["bytes"] * (w.n_checks / launches) / rec["checks"])
        roof["traffic_note"] = (f"ncu DRAM bytes of one {rec['reads']}-read batch launch ({rec['checks']} checks), "
                                f"scaled to the average launch by its checks")
    out = {"form": form, "tune": tune.as_dict(), "pass_rate": float(pass_d.float().mean().item()),
           "workload_stats": {"checks_per_gpu_step": w.n_checks,
                              "cands_per_read_mean": round(w.n_checks / w.n_reads, 2)},
           "plain_gather_same_workload": {"value": w.n_checks / (ap / 1e3), "ms_per_step": ap,
                                          "frac": alg / (ap / 1e3) / 1e9 / hbm}}
    if ctx.rank == 0 and ctx.world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(form, w, args.cpu_seconds)
    del ins, pass_d
    bank.free()
    return finish(out, form, ctx, w, w.n_checks, ms, steps, roof, launches, clk, bank_info), w


def run_fullscan(args, ctx, primary, peaks):
    import torch

    import paper_1711_01177_gb300 as grim
    form = "fullscan"
    w = make_workload(form, args, ctx.rank)
    steps = args.steps if primary else args.sub_steps
    warmup = args.warmup if primary else 1
    bank, bank_info = build_bank_timed(grim, ctx, w)
    s = ctx.stream
    ins = [ctx.dev(w.bases), ctx.dev(w.read_offsets), ctx.dev(w.E)]
    res = grim.grim_scan(bank, *ins, cap=1 << 24, stream=s)
    call = lambda: grim.grim_scan(bank, *ins, out=res, stream=s)
    ms, clk = ctx.timed(call, steps, warmup)
    st, flags = grim.grim_bank_status(bank, s)
    assert st == grim.GRIM_OK, (st, flags)
    units = w.n_reads * w.n_bins
    avg = float(np.mean(ms))
    flops = 2.0 * units * (4 ** w.q)
    tf = flops / (avg / 1e3) / 1e12
    kind = grim.grim_scan_kind()
    burst = peaks.get(f"{kind}_tflops")
    roof = {"bound": "tensor", "achieved": tf, "peak": burst, "unit": "TFLOP/s",
            "frac": tf / burst if burst else None, "traffic": None,
            "peak_source": f"measured {kind}_tflops (grim_peak, operands in shared memory, burst)",
            "kernel": f"scan_kernel<{w.q}> (+ scan_prep_kernel), tcgen05 kind::{kind}",
            "algorithmic_flops_per_launch": flops, "avg_step_ms": avg}
    for k in (f"{kind}_tmem_a_tflops", f"{kind}_tmem_a_tflops_sustained"):
        if peaks.get(k):
            roof["frac_of_" + k] = tf / peaks[k]
    out = {"form": form, "pairs_passing": res.n_pairs}
    if primary:
        h_in = [ctx.pin(w.bases), ctx.pin(w.read_offsets), ctx.pin(w.E)]
        n_pairs = res.n_pairs
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

        e2e_ms, _ = ctx.timed(e2e_step, steps, warmup, clocks=False)
        out["e2e"] = {"value": units * ctx.world * steps / (ctx.max_over_ranks(sum(e2e_ms)) / 1e3), "unit": UNIT,
                      "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in h_in),
                      "d2h_bytes_per_step": 8 + 8 * (n_pairs + 1)}
    if ctx.rank == 0 and ctx.world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(form, w, args.cpu_seconds)
    del ins, res
    bank.free()
    return finish(out, form, ctx, w, units, ms, steps, roof, 2, clk, bank_info), w


def run_mixed(args, ctx, primary, peaks):
    import torch

    import paper_1711_01177_gb300 as grim
    form = "mixed"
    w = make_workload(form, args, ctx.rank)
    steps = args.steps if primary else args.sub_steps
    warmup = args.warmup if primary else 1
    bank, bank_info = build_bank_timed(grim, ctx, w)
    s, dev = ctx.stream, ctx.dev
    torch.cuda.empty_cache()  # the library allocates from its own pool, not torch's cache
    ref_d = dev(w.ref2bit)
    reads_d, offs_d, E_d = dev(w.bases), dev(w.read_offsets), dev(w.E)
    s.synchronize()
    # the mapper's side of the filter on the GPU: seed table, then candidates
    t0 = time.perf_counter()
    with torch.cuda.stream(s):
        idx = grim.grim_seed_index_build(ref_d, w.ref_len, w.meta["seed_k"], stream=s)
    s.synchronize()
    index_s = time.perf_counter() - t0
    # candidates twice: the first call also grows the library's memory pool,
    # the second (output sized to the first's count) is the warm figure
    cand_runs = []
    for capacity in (w.n_reads * 2048, None):
        if capacity is None:
            capacity = int(cb_d.numel())
            del cb_d, co_d
        t0 = time.perf_counter()
        with torch.cuda.stream(s):
            cb_d, co_d = grim.grim_seed_candidates(idx, reads_d, offs_d, w.bin_len, w.n_bins, w.meta["cap"],
                                                   capacity=capacity, stream=s)
        s.synchronize()
        cand_runs.append(time.perf_counter() - t0)
    cand_s = cand_runs[-1]
    n_checks = int(cb_d.numel())
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

    ms, clk = ctx.timed(call, steps, warmup)
    # the dispatcher's kernels per step: the batch-bounds gather, one launch
    # per run of gathered batches (here all of them: one), and per scanned
    # batch the prep, scan and the two join kernels
    n_sc = scanned[-1] if scanned else 0
    sc_batches = -(-n_sc // 262_144)
    launches = 1 if n_sc < w.n_reads else sc_batches
    kernels_per_step = 1 + (1 if n_sc < w.n_reads else 0) + 4 * sc_batches
    ms_g, _ = ctx.timed(lambda: grim.grim_filter_batched(bank, *ins, pass_out=pass_d, tune=tune, stream=s),
                        args.sub_steps, 1, clocks=False)
    nb = min(w.n_reads, 65_536)  # the full scan is timed on one batch of reads
    scan_ins = (reads_d, offs_d[:nb + 1], E_d[:nb])
    res = grim.grim_scan(bank, *scan_ins, cap=1 << 24, stream=s)
    ms_s, _ = ctx.timed(lambda: grim.grim_scan(bank, *scan_ins, out=res, stream=s), 1, 1, clocks=False)
    n_pass = int(torch.count_nonzero(pass_d).item())
    ms_l, _ = ctx.timed(lambda: grim.grim_locate(bank, cb_d, co_d, pass_d, capacity=n_pass, stream=s), 1, 1,
                        clocks=False)
    loc = grim.grim_locate(bank, cb_d, co_d, pass_d, capacity=n_pass, stream=s)
    st, flags = grim.grim_bank_status(bank, s)
    assert st == grim.GRIM_OK, (st, flags)
    avg = float(np.mean(ms))
    g, sc, lc = float(np.mean(ms_g)), float(np.mean(ms_s)), float(np.mean(ms_l))
    row = bank.row_words * 4
    alg = gather_bytes(n_checks, w, row)
    hbm, hbm_src = load_hbm_peak()
    ach = alg / (avg / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": None,
            "peak_source": hbm_src, "kernel": "dispatcher -> gather_kernel<5,*,DEEP>", "algorithmic_bytes_per_launch":
            alg // launches, "launches_per_step": launches, "avg_step_ms": avg}
    if peaks.get("hbm_copy_gbs_this_box"):
        # context: boxes differ by several percent on this DRAM-bound line
        roof["this_box_copy_gbs"] = peaks["hbm_copy_gbs_this_box"]
        roof["frac_of_this_box_copy"] = ach / peaks["hbm_copy_gbs_this_box"]
    sha = source_sha()
    rec = TRAFFIC_BY_SOURCE.get(sha, {}).get(form, {})
    roof["source_sha"] = sha
    if rec.get("reads"):
        # measured on one batch launch; scaled to the average launch by checks
        roof["traffic"] = int(rec["bytes"] * (n_checks / launches) / rec["checks"])
        roof["traffic_note"] = (f"ncu DRAM bytes of one {rec['reads']}-read batch launch ({rec['checks']} checks), "
                                f"scaled to the average launch by its checks")
    out = {"form": form,
           "workload_stats": {"checks_per_gpu_step": n_checks, "cands_per_read_mean": round(n_checks / w.n_reads, 2),
                              "cands_per_read_max": int(per_read.max().item()),
                              "candidates": "GPU seed table + grim_seed_candidates (12-mer seeds, cap 10000)"},
           "dispatch": {"choice": "scan" if choice == grim.GRIM_FORM_SCAN else "gather",
                        "reads_scanned_per_step": scanned[-1] if scanned else 0},
           "gather_form": {"ms_per_step": g, "checks_per_s": n_checks / (g / 1e3),
                           "reads_per_s": w.n_reads / (g / 1e3)},
           "scan_form": {"ms_per_batch": sc, "batch_reads": nb, "checks_per_s_all_bins": nb * w.n_bins / (sc / 1e3),
                         "reads_per_s": nb / (sc / 1e3), "pairs_passing": res.n_pairs,
                         "note": "one batch of reads timed; the dispatcher's choice runs every read"},
           "seed_pipeline": {"seed_table_s": index_s, "candidates_s": cand_s, "candidates_first_call_s": cand_runs[0],
                             "candidates_reads_per_s": w.n_reads / cand_s, "locate_ms": lc,
                             "locations_passing": loc.n,
                             "reads_per_s_serial": w.n_reads / (cand_s + avg / 1e3 + lc / 1e3)},
           "pass_rate": n_pass / max(1, n_checks)}
    del res
    if not args.no_extras:
        # the paper's metrics (Sec. 5, 6.1): every passing location aligned
        # against its bin's span; every candidate of the first reads too, to
        # count misses (rejected locations that map)
        ms_v, _ = ctx.timed(lambda: grim.grim_verify(bank, ref_d, reads_d, offs_d, loc.read, loc.bin, stream=s), 1, 1,
                            clocks=False)
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
        del dist, dist_all, every
        serial_s = cand_s + avg / 1e3 + lc / 1e3 + float(np.mean(ms_v)) / 1e3
    del loc, ins
    if primary:
        # end to end through the public calls: reads in from pinned host
        # memory, candidates on the GPU, the dispatcher, pass bytes back
        del cb_d, co_d
        torch.cuda.empty_cache()
        h_in = [ctx.pin(w.bases), ctx.pin(w.read_offsets), ctx.pin(w.E)]
        bits_d = torch.empty((n_checks + 31) // 32, dtype=torch.int32, device="cuda")
        h_out = torch.empty(bits_d.numel(), dtype=torch.int32).pin_memory()

        def e2e_step():
            for h, d in zip(h_in, (reads_d, offs_d, E_d)):
                d.copy_(h, non_blocking=True)
            cb2, co2 = grim.grim_seed_candidates(idx, reads_d, offs_d, w.bin_len, w.n_bins, w.meta["cap"],
                                                 capacity=n_checks, stream=s)
            grim.grim_filter_auto(bank, reads_d, offs_d, cb2, co2, E_d, pass_out=pass_d, stream=s)
            # the filter bitmask (Sec. 3.3): one bit per (read, candidate bin)
            grim.grim_pack_mask(pass_d, bits_d, stream=s)
            h_out.copy_(bits_d, non_blocking=True)

        e2e_ms, _ = ctx.timed(e2e_step, steps, warmup, clocks=False)
        out["e2e"] = {"value": n_checks * ctx.world * steps / (ctx.max_over_ranks(sum(e2e_ms)) / 1e3), "unit": UNIT,
                      "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in h_in),
                      "d2h_bytes_per_step": h_out.numel() * h_out.element_size(),
                      "includes": "reads copied in from pinned memory, seed candidates on the GPU (synchronising), "
                                  "dispatcher, the pass bitmask (one bit per check, grim_pack_mask) to pinned host "
                                  "memory"}
        del h_in, h_out, bits_d
    else:
        del cb_d, co_d
    del pass_d
    torch.cuda.empty_cache()
    if not args.no_extras:
        # the whole path around the filter, alignment overlapping the next
        # batch's filtering (grim_map, 1M-read batches): once to warm, once timed
        # the filter's stream ahead of the aligner's when both have work
        filt, align = torch.cuda.Stream(priority=-1), torch.cuda.Stream(priority=0)
        cap_loc = int(n_pass * 1.25) + 1024

        def map_time(align_stream):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(filt):
                m = grim.grim_map(bank, idx, ref_d, reads_d, offs_d, E_d, cap=w.meta["cap"], batch_reads=1 << 20,
                                  capacity=cap_loc, stream=filt, align_stream=align_stream)
            torch.cuda.synchronize()
            return time.perf_counter() - t0, m

        map_time(align)  # warm: slot sizes, pools
        map_s, mp = map_time(align)
        # the same batches with the aligner on the filter's stream: no overlap
        same_s, mp_same = map_time(filt)
        assert mp_same.n == mp.n
        out["seed_pipeline"].update({"overlapped_s": map_s, "overlapped_reads_per_s": w.n_reads / map_s,
                                     "serial_sum_s": serial_s, "same_batches_one_stream_s": same_s,
                                     "overlapped_locations": mp.n})
        del mp, mp_same
    idx.free()
    del reads_d, offs_d, E_d, ref_d
    torch.cuda.empty_cache()
    if ctx.rank == 0 and ctx.world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(form, w, args.cpu_seconds)
    bank.free()
    return finish(out, form, ctx, w, n_checks, ms, steps, roof, kernels_per_step, clk, bank_info), w


def q_sweep(args, ctx):
    """Token sizes 4-6 on the same 100 Mbp reads and seed candidates (the
    paper sweeps them in Sec. 6.1): bank size and build time, gather time,
    checks/s, fraction of HBM and the share of candidates that pass; then
    bin counts of 3, 6 and 12 x 2^16 at q = 5."""
    import torch

    import paper_1711_01177_gb300 as grim
    import synth
    w = synth.gather_seeds(ref_len=args.ref_bp, n_reads=args.q_sweep_reads,
                           read_seed=synth.SEED_READS + 1000 * ctx.rank + 7)
    dev, s = ctx.dev, ctx.stream
    ref_d = dev(w.ref2bit)
    ins = [dev(w.bases), dev(w.read_offsets), dev(w.cand_bins), dev(w.cand_offsets), dev(w.E)]
    pass_d = torch.empty(w.n_checks, dtype=torch.uint8, device="cuda")
    hbm, _ = load_hbm_peak()
    out = {"workload": f"{args.ref_bp / 1e6:g} Mbp repeat-rich reference, {w.n_reads} x 150 bp reads, "
                       f"12-mer seed candidates ({w.n_checks} checks), E = 7 for every q", "by_q": {}}
    for q in (4, 5, 6):
        bank = grim.grim_build_bank(ref_d, w.ref_len, q, w.bin_len, w.overlap, stream=s)
        bms, _ = ctx.timed(lambda: grim.grim_build_bank_into(bank, ref_d, stream=s), 2, 1, clocks=False)
        ms, _ = ctx.timed(lambda: grim.grim_filter(bank, *ins, pass_out=pass_d, stream=s), args.sub_steps, 2,
                          clocks=False)
        st, flags = grim.grim_bank_status(bank, s)
        assert st == grim.GRIM_OK, (st, flags)
        avg = float(np.mean(ms))
        row = bank.row_words * 4
        alg = gather_bytes(w.n_checks, w, row)
        out["by_q"][str(q)] = {"bank_bytes": bank.n_bins * row, "bank_build_ms": sig(float(np.median(bms))),
                               "ms_per_step": sig(avg), "checks_per_s": sig(w.n_checks / (avg / 1e3)),
                               "hbm_frac": sig(alg / (avg / 1e3) / 1e9 / hbm, 3),
                               "pass_rate": sig(float(pass_d.float().mean().item()), 3)}
        bank.free()
    del pass_d
    # bin counts as multiples of 2^16 (the paper's banks hold 450 x 2^16
    # bins, Sec. 6.1): q = 5, the bin length that gives k x 2^16 bins, the
    # candidates rebuilt for it from the GPU seed table
    out["bin_count_workload"] = (f"same reads, q=5, overlap {w.overlap} bp, 12-mer seed candidates (cap 1000) "
                                 f"rebuilt on the GPU for each bin length")
    out["by_bin_count"] = {}
    idx = grim.grim_seed_index_build(ref_d, w.ref_len, 12, stream=s)
    for k in (3, 6, 12):
        bin_len = -(-w.ref_len // (k << 16))
        bank = grim.grim_build_bank(ref_d, w.ref_len, 5, bin_len, w.overlap, stream=s)
        bms, _ = ctx.timed(lambda: grim.grim_build_bank_into(bank, ref_d, stream=s), 2, 1, clocks=False)
        with torch.cuda.stream(s):
            cb, co = grim.grim_seed_candidates(idx, ins[0], ins[1], bin_len, bank.n_bins, 1000,
                                               capacity=w.n_reads * 1000, stream=s)
        n_checks = int(cb.numel())
        pd = torch.empty(max(n_checks, 1), dtype=torch.uint8, device="cuda")
        kins = [ins[0], ins[1], cb, co, ins[4]]
        ms, _ = ctx.timed(lambda: grim.grim_filter(bank, *kins, pass_out=pd, stream=s), args.sub_steps, 2,
                          clocks=False)
        st, flags = grim.grim_bank_status(bank, s)
        assert st == grim.GRIM_OK, (st, flags)
        avg = float(np.mean(ms))
        row = bank.row_words * 4
        alg = gather_bytes(n_checks, w, row)
        out["by_bin_count"][f"{k}x2^16"] = {
            "n_bins": bank.n_bins, "bin_len": bin_len, "bank_bytes": bank.n_bins * row,
            "bank_build_ms": sig(float(np.median(bms))), "checks": n_checks,
            "cands_per_read": sig(n_checks / w.n_reads, 3), "ms_per_step": sig(avg),
            "checks_per_s": sig(n_checks / (avg / 1e3)), "reads_per_s": sig(w.n_reads / (avg / 1e3)),
            "hbm_frac": sig(alg / (avg / 1e3) / 1e9 / hbm, 3),
            "pass_rate": sig(float(pd[:n_checks].float().mean().item()), 3)}
        bank.free()
        del cb, co, pd, kins
    idx.free()
    del ins, ref_d
    torch.cuda.empty_cache()
    return out


RUNNERS = {"plain": lambda a, c, p, k: run_plain_or_gather("plain", a, c, p, k),
           "gather": lambda a, c, p, k: run_plain_or_gather("gather", a, c, p, k),
           "batched": run_batched, "fullscan": run_fullscan, "mixed": run_mixed}


def summary(m):
    """The compact record of one workload kept at the end of the line."""
    r = m["roofline"]
    frac = r.get("summary_frac", r.get("frac"))
    peak_src = r.get("summary_peak", r.get("peak_source", ""))
    cpu = m.get("cpu_baseline") or {}
    clk = m.get("clocks") or {}
    roof = {"bound": r.get("bound"), "frac": sig(frac, 3),
            "peak": sig(r.get("l2_peak") if "summary_frac" in r else r["peak"]), "peak_source": peak_src.split(" (")[0]}
    if r.get("bound") == "hbm":
        roof["hbm_frac"] = sig(r["frac"], 3)  # algorithmic bytes against HBM, also for L2-resident banks
    return {"value": sig(m["value"]), "ms_per_step": sig(m["ms_per_step"]), "reads_per_s": sig(m["reads_per_s"]),
            "roofline": roof,
            "cpu_baseline": sig(cpu.get("value")),
            "clocks": {"sm_mhz": clk.get("sm_mhz"), "reasons": clk.get("reasons")}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    form = args.workload
    w = make_workload(form, args, 0, cand_reads=16_384 if form == "mixed" else 0)
    run, n_max, what = oracle_sampler(form, w)
    info = cpu_info()
    threads = info["nproc"]
    per_step = min(20.0, max(0.05, args.ref_seconds / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_rate(run, n_max, per_step, threads)
    times, units, used = [], 0, 0
    for _ in range(args.steps):
        rate, n, done, dt = oracle_rate(run, n_max, per_step, threads)
        times.append(dt)
        units += done
        used = n
    value = units / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": describe(form, w, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"per step the first {used} {what}, on {threads} threads",
                             "cpu_model": info["cpu_model"]},
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
    peaks = measure_peaks(ctx)
    main_form, w = RUNNERS[args.workload](args, ctx, True, peaks)
    subs = {}
    if not args.only:
        for form in ("plain", "gather", "fullscan", "batched", "mixed"):
            if form != args.workload:
                subs[form], _ = RUNNERS[form](args, ctx, False, peaks)
    sweep = q_sweep(args, ctx) if not (args.no_q_sweep or args.only) else None
    if rank == 0:
        m = main_form
        line = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "e2m1" if args.workload == "fullscan" else "u32",
                "data": "synthetic", "config": describe(args.workload, w, world), "reads_per_s": m["reads_per_s"],
                "roofline": m["roofline"], "e2e": m.get("e2e"), "gpu_launches": m["gpu_launches"],
                "clocks": m["clocks"], "cpu_baseline": m.get("cpu_baseline"), "bank_build": m["bank_build"],
                "peaks": peaks}
        for k in ("workload_stats", "pass_rate", "tune", "plain_gather_same_workload", "pairs_passing", "dispatch",
                  "gather_form", "scan_form", "verification", "seed_pipeline"):
            if k in m:
                line[k] = m[k]
        if sweep:
            line["q_sweep"] = sweep
        if subs:
            # details of the other workloads, then their summaries as the
            # line's last key
            line["details"] = {SUMMARY_KEY[f]: {k: v for k, v in d.items()
                                                if k in ("bank_build", "workload_stats", "pass_rate", "tune",
                                                         "plain_gather_same_workload", "pairs_passing")}
                               for f, d in subs.items()}
            line["configs"] = {SUMMARY_KEY[f]: summary(d) for f, d in subs.items()}
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
