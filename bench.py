#!/usr/bin/env python3
"""Throughput of batched HQC.PKE decryption on GB300.

One step = one pass of the whole decryption path (product, XOR/truncate,
duplicated RM decode, RS decode) over one batch of synthetic ciphertexts
that are already resident in HBM.  Default workload: HQC-1 bulk, 65,536
ciphertexts under 256 registered keys, one fused keyed launch per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...     # the CPU oracle on host cores

Prints one JSON line (rank 0).  Under torchrun each rank decrypts its own
batch (weak scaling, no collective on the data path); the reported time is
the maximum over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "HQC-1/3/5 decryptions/sec per GB300 (batched vs plain) and p99 latency"
UNIT = "decryptions/s"
L2_BYTES = 129 * 2 ** 20

WORKLOADS = {
    # name: (level, count, nkeys, description)
    "hqc1-bulk": (1, 65536, 256, "HQC-1 bulk: 65536 ciphertexts under 256 keypairs, one batched keyed launch"),
    "hqc3": (3, 32768, 128, "HQC-3 batch: 32768 ciphertexts under 128 keypairs, one batched keyed launch"),
    "hqc5": (5, 32768, 128, "HQC-5 batch: 32768 ciphertexts under 128 keypairs, one batched keyed launch"),
    "hqc1-plain": (1, 256, 16, "HQC-1 plain path: 256 ciphertexts under 16 keypairs"),
    "mixed": (0, 100000, 384, "Mixed levels: 100000 ciphertexts, 40% HQC-1 / 35% HQC-3 / 25% HQC-5 shuffled, "
                              "384 keypairs (128 per level), one CUDA-graph plan with autotuned launch shapes"),
}
MIXED_SPLIT = ((1, 40000), (3, 35000), (5, 25000))
WORKLOADS["serving"] = (0, 0, 384, "Serving: open-loop Poisson bursts of 1-512 requests (log-uniform), levels 40/35/25 %, "
                                   "keys resident, 256 MiB device budget over 4 streams, continuous batching")
SERVE_LOADS = (1e5, 1e6, 1e7)
KEM_WORKLOADS = {
    "kem1-decaps": (1, 65536, 256, "HQC-1 KEM decapsulation: 65536 ciphertexts under 256 seeded keypairs "
                                   "(decrypt, re-derive, re-encrypt and compare, K with implicit rejection)"),
    "kem3-decaps": (3, 32768, 128, "HQC-3 KEM decapsulation: 32768 ciphertexts under 128 seeded keypairs"),
    "kem5-decaps": (5, 32768, 128, "HQC-5 KEM decapsulation: 32768 ciphertexts under 128 seeded keypairs"),
}
WORKLOADS.update(KEM_WORKLOADS)
KEM_UNIT = "decapsulations/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="hqc1-bulk")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="target CPU-baseline duration")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="trace length per offered load (serving): at most 30 s with --workload serving, 2 s inside the default line")
    ap.add_argument("--mixed-plan", default="auto",
                    help="mixed workload: 'auto' tunes the plan; FORM[:V1,V3,V5[:G1,G3,G5]] builds that configuration "
                         "(form 1-4, per-level variants by name, blocks per level)")
    ap.add_argument("--key-offset", type=int, default=0,
                    help="draw the seeded keys from this key index on (another key set, same recipe)")
    ap.add_argument("--configs", choices=["auto", "all", "none"], default="auto",
                    help="also measure every other benchmark configuration (auto: with the default workload at N=1)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU, launched by torchrun)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self, want_gpus: int):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            import torch
            torch.cuda.set_device(self.local)
            dist.init_process_group(backend="nccl", device_id=torch.device("cuda", self.local))
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 200):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.QUERY,
                                       "--format=csv,noheader,nounits", "-lms", str(int(interval_ms))],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload construction (on the device, with the library's own keygen and
# encryption kernels; randomness from the seeded generator)
# ---------------------------------------------------------------------------
KEY_OFFSET = 0  # --key-offset: the seeded key set starts at this key index


def make_workload(hqc, level, count, nkeys, rank, device):
    import torch
    import synth
    P = hqc.hqc_get_params(level)
    S = synth.Shape.of(P)
    h, x, y = synth.keys(S, nkeys, first=KEY_OFFSET + rank * nkeys)
    m, r1, r2, e = synth.ciphertext_randomness(S, count, first=rank * count)
    kidx = synth.key_assignment(count, nkeys, tag=100 + level)
    dev = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a if dt is None else a.view(dt))).to(device)
    h_d = dev(h, np.int64)
    s_d = hqc.hqc_keygen_batch(level, h_d, dev(x, np.int32), dev(y, np.int32))
    m_d = dev(m)
    k_d = dev(kidx.astype(np.int32))
    u_d, v_d = hqc.hqc_encrypt_batch(level, h_d, s_d, k_d, m_d, dev(r1, np.int32), dev(r2, np.int32),
                                     dev(e, np.int32))
    torch.cuda.synchronize()
    keys = hqc.Keyset(level, y)
    return P, keys, u_d, v_d, k_d, m_d, y, kidx


def pct(xs, q):
    s = sorted(xs)
    return s[min(len(s) - 1, int(round(q / 100.0 * (len(s) - 1))))]


def load_peaks():
    """On-chip peaks measured once in this run (libhqc_peaks.so)."""
    from paper_2512_12904_gb300 import _build
    lib = ctypes.CDLL(_build.PEAKS_LIB)
    for f in ("hqc_peak_smem_read_bytes_per_s", "hqc_peak_int_ops_per_s", "hqc_peak_int_issue_ops_per_s"):
        getattr(lib, f).restype = ctypes.c_double
    return {"smem_bytes_per_s": lib.hqc_peak_smem_read_bytes_per_s(),
            "alu_ops_per_s": lib.hqc_peak_int_ops_per_s(),
            "issue_ops_per_s": lib.hqc_peak_int_issue_ops_per_s()}


def measured_peaks_file():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def per_decryption_work(P):
    """Algorithmic work of one decryption (the per-unit figures of the roofline)."""
    W_v32 = P.n1 * P.n2 // 32
    nr, cap = 2 * P.delta, 2 * P.delta + 1
    smem = P.w * P.n1 * P.n2 // 8                  # rotated operand read once per support entry
    hbm = P.W_u_pitch * 8 + P.W_v * 8 + P.k + 4     # u row, v row, m row, key index
    gf_mults = nr * P.n1 + 2 * nr * cap + nr * nr // 2 + P.k * (2 * cap + nr)
    int_ops = 2 * P.w * W_v32 + P.n1 * (128 * P.mult + 896 + 256) + 4 * gf_mults
    return smem, hbm, int_ops


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(level, nkeys, count):
    import oracle
    import synth
    P = oracle.params(level)
    S = synth.Shape.of(P)
    h, x, y = synth.keys(S, nkeys)
    s = oracle.keygen(level, h, x, y)
    m, r1, r2, e = synth.ciphertext_randomness(S, count)
    kidx = synth.key_assignment(count, nkeys, tag=100 + level) % nkeys
    u, v = oracle.encrypt(level, h, s, kidx.astype(np.int32), m, r1, r2, e)
    return u, v, y[kidx], m


def oracle_rate(level, nkeys, target_s, cores):
    import oracle
    probe = max(2 * cores, 16)
    u, v, y, m = oracle_sample(level, nkeys, probe)
    t = time.perf_counter()
    oracle.decrypt(level, u, v, y, nthreads=cores)
    rate = probe / max(time.perf_counter() - t, 1e-6)
    n = int(max(probe, min(200000, rate * target_s)))
    u, v, y, m = oracle_sample(level, nkeys, n)
    t = time.perf_counter()
    got = oracle.decrypt(level, u, v, y, nthreads=cores)
    dt = time.perf_counter() - t
    assert (got == m).all(), "oracle sample failed to decrypt"
    return n / dt, n, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    if args.workload in KEM_WORKLOADS:
        return run_reference_kem(args)
    level, count, nkeys, desc = WORKLOADS[args.workload]
    if level == 0:
        level, nkeys = 1, nkeys // 3  # the mixed workload's reference arm times its HQC-1 share
    cores = os.cpu_count() or 1
    # calibrate, then size each step so the whole run takes ~2 minutes
    probe = max(2 * cores, 16)
    u, v, y, m = oracle_sample(level, nkeys, probe)
    t = time.perf_counter()
    oracle.decrypt(level, u, v, y, nthreads=cores)
    rate = probe / max(time.perf_counter() - t, 1e-6)
    per_step = int(max(cores, min(count, 120.0 * rate / max(1, args.steps + args.warmup))))
    u, v, y, m = oracle_sample(level, nkeys, per_step)
    for _ in range(args.warmup):
        oracle.decrypt(level, u, v, y, nthreads=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        got = oracle.decrypt(level, u, v, y, nthreads=cores)
    dt = time.perf_counter() - t
    assert (got == m).all()
    value = per_step * args.steps / dt
    sample = "%d of the workload's ciphertexts per step (oracle-encrypted, same seeds), %d threads" % (per_step, cores)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": {"workload": desc, "level": level, "count": count, "nkeys": nkeys},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def kem_oracle_sample(level, nkeys, count, tag):
    """Seeded key pairs and oracle-encapsulated ciphertexts for the KEM workloads."""
    import oracle
    import synth
    P = oracle.params(level)

    def rows(cnt, width, t):
        nw = (cnt * width + 7) // 8 + 1
        return synth.words(nw, tag=t).view(np.uint8)[:cnt * width].reshape(cnt, width).copy()

    h, x, y, s = oracle.kem_keygen(level, rows(nkeys, 32, tag), rows(nkeys, 32, tag + 1))
    sigma = rows(nkeys, P.k, tag + 2)
    kidx = synth.key_assignment(count, nkeys, tag=tag + 3)
    m, salt = rows(count, P.k, tag + 4), rows(count, 16, tag + 5)
    u, v, K = oracle.kem_encaps(level, h, s, kidx, m, salt)
    return (h, s, y, sigma, kidx, u, v, salt), K


def run_reference_kem(args):
    import oracle
    level, count, nkeys, desc = WORKLOADS[args.workload]
    nkeys = min(nkeys, 16)  # the oracle's key generation is slow; the sample reuses 16 of the key pairs
    cores = os.cpu_count() or 1
    probe_args, _ = kem_oracle_sample(level, nkeys, max(2 * cores, 16), tag=7000 + 100 * level)
    t = time.perf_counter()
    oracle.kem_decaps(level, *probe_args, nthreads=cores)
    rate = probe_args[4].size / max(time.perf_counter() - t, 1e-6)
    # the sample's encapsulation runs on one core: keep it to seconds
    per_step = int(max(cores, min(count, 2000, 120.0 * rate / max(1, args.steps + args.warmup))))
    dargs, K = kem_oracle_sample(level, nkeys, per_step, tag=7000 + 100 * level)
    for _ in range(args.warmup):
        oracle.kem_decaps(level, *dargs, nthreads=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        Kd, ok = oracle.kem_decaps(level, *dargs, nthreads=cores)
    dt = time.perf_counter() - t
    assert ok.all() and (Kd == K).all()
    value = per_step * args.steps / dt
    sample = "%d decapsulations per step (oracle-encapsulated, %d key pairs), %d threads" % (per_step, nkeys, cores)
    print(json.dumps({
        "impl": "reference", "metric": "HQC KEM decapsulations/sec per GB300", "value": value, "unit": KEM_UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": desc, "level": level, "count": count, "nkeys": nkeys},
        "cpu_baseline": {"value": value, "unit": KEM_UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": KEM_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
class Ctx:
    """What every GPU measurement of one bench process shares: the rank's
    device, the library, the on-chip peaks measured once in this run, and an
    L2 flush buffer for workloads smaller than L2."""

    def __init__(self, args):
        import torch
        import paper_2512_12904_gb300 as hqc
        self.args = args
        self.dist = Dist(args.gpus)
        self.device = torch.device("cuda", self.dist.local)
        torch.cuda.set_device(self.device)
        hqc.load()
        self.hqc = hqc
        self.peaks = load_peaks()
        self.hbm_peak = measured_peaks_file().get("hbm_gbs")
        self._flush = None

    def flush_l2(self):
        """Overwrite a buffer twice the size of L2 (on the current stream)."""
        import torch
        if self._flush is None:
            self._flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=self.device)
        self._flush.fill_(0x5A5A5A5A)

    def roofline(self, smem_b, int_ops, hbm_b, seconds, kernel, traffic=None):
        """Roofline of a measured launch: algorithmic work ÷ its time against
        the peaks measured in this run (ALU pipe, ALU+FMA issue, shared
        memory) and MEASURED_PEAKS.json's HBM bandwidth."""
        smem_peak = self.peaks["smem_bytes_per_s"] / 1e9
        alu_peak = self.peaks["alu_ops_per_s"] / 1e9
        issue_peak = self.peaks["issue_ops_per_s"] / 1e9
        smem_ach = smem_b / seconds / 1e9
        int_ach = int_ops / seconds / 1e9
        hbm_ach = hbm_b / seconds / 1e9
        blocks = {
            "smem": {"bound": "smem", "achieved": smem_ach, "peak": smem_peak, "unit": "GB/s",
                     "frac": smem_ach / smem_peak if smem_peak else None, "traffic": None,
                     "peak_source": "measured in this run: conflict-free 32-bit shared-memory loads, all SMs"},
            "alu": {"bound": "alu", "achieved": int_ach, "peak": alu_peak, "unit": "Gop/s",
                    "frac": int_ach / alu_peak if alu_peak else None,
                    "peak_source": "measured in this run: 32-bit funnel-shift + XOR issue rate, all SMs "
                                   "(the integer ALU pipe alone)",
                    "issue": {"peak": issue_peak, "frac": int_ach / issue_peak if issue_peak else None,
                              "peak_source": "measured in this run: half funnel-shift/XOR (ALU pipe), half "
                                             "IMAD (FMA pipe), all SMs: the integer issue ceiling of both pipes"}},
            "hbm": {"bound": "hbm", "achieved": hbm_ach, "peak": self.hbm_peak, "unit": "GB/s",
                    "frac": hbm_ach / self.hbm_peak if self.hbm_peak else None,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if self.hbm_peak else "absent"},
        }
        primary = max(("smem", "alu"), key=lambda k: blocks[k]["frac"] or 0)
        roof = dict(blocks[primary])
        roof["kernel"] = kernel
        roof["traffic"] = traffic
        roof["others"] = {k: v for k, v in blocks.items() if k != primary}
        return roof


def timed_steps(fn, steps, stream, dist, clocks_idx=None, flush=None):
    """Run fn() `steps` times between barriers; return (total_ms, per-step ms
    list, clocks).  With flush, flush() runs between steps outside the
    events, and total_ms is the sum of the steps' own times."""
    import torch
    dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(clocks_idx) if clocks_idx is not None else None
    with torch.cuda.stream(stream):
        if flush is None:
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
            evs[0].record(stream)
            for i in range(steps):
                fn()
                evs[i + 1].record(stream)
        else:
            pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                     for _ in range(steps)]
            for a, b in pairs:
                flush()
                a.record(stream)
                fn()
                b.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clocks = clk.stop() if clk else None
    if flush is None:
        per = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
        return evs[0].elapsed_time(evs[-1]), per, clocks
    per = [a.elapsed_time(b) for a, b in pairs]
    return sum(per), per, clocks


def warm(fn, n, stream):
    import torch
    with torch.cuda.stream(stream):
        for _ in range(n):
            fn()
    torch.cuda.synchronize()


def decrypt_kernel_name(level, count):
    """The kernel hqc_decrypt_batch_keyed runs for this batch (default shape)."""
    if count <= 8:
        return "k_decrypt_latency_cluster<%d,keyed,4,4>" % level
    if count <= 512:
        return "k_decrypt_latency<%d,keyed,4>" % level
    return ("k_decrypt_team<%d,keyed>" if level == 5 else "k_decrypt_fused<%d,keyed>") % level


def sub_steps(args):
    """Steps of a sub-configuration: the driver's K, bounded to keep the
    default run within a few minutes."""
    return max(5, min(args.steps, 50)), max(3, args.warmup)


def bench_single(ctx, wl_name, full):
    """One level: the fused batched form (the keyed entry point) against the
    plain per-stage form on the same inputs, every m checked."""
    import torch
    hqc, dist, args, device = ctx.hqc, ctx.dist, ctx.args, ctx.device
    level, count, nkeys, desc = WORKLOADS[wl_name]
    P, keys, u_d, v_d, k_d, m_ref, y_host, kidx = make_workload(hqc, level, count, nkeys, dist.rank, device)
    m_out = torch.empty_like(m_ref)
    stream = torch.cuda.Stream(device=device)
    in_bytes = (u_d.numel() + v_d.numel()) * 8
    flush = ctx.flush_l2 if in_bytes <= L2_BYTES else None
    l2 = ("inputs (%d MB) larger than L2 (129 MB); no flush" % (in_bytes // 2 ** 20) if flush is None else
          "inputs (%.1f MB) smaller than L2: a 258 MB buffer is overwritten between timed steps, outside the "
          "events; value = count x steps / sum of the steps' own times" % (in_bytes / 2 ** 20))
    steps, warmup = (args.steps, args.warmup) if full else sub_steps(args)

    def step():
        hqc.hqc_decrypt_batch_keyed(level, u_d, v_d, keys, k_d, m_out, stream=stream)

    warm(step, warmup, stream)
    total_ms, per, clocks = timed_steps(step, steps, stream, dist, clocks_idx=dist.local if full else None,
                                        flush=flush)
    max_ms = dist.max(total_ms)
    correct = bool((m_out == m_ref).all().item())
    wrong = int((m_out != m_ref).any(dim=1).sum().item())

    # plain one-kernel-per-stage form on the same inputs
    ws = torch.empty(hqc.hqc_staged_workspace_bytes(level, count), dtype=torch.uint8, device=device)
    m_plain = torch.empty_like(m_ref)

    def plain_step():
        hqc.hqc_decrypt_batch_staged(level, u_d, v_d, keys=keys, key_idx=k_d, workspace=ws, m_out=m_plain,
                                     stream=stream)

    plain_steps = max(5, min(steps, 200))
    warm(plain_step, 3, stream)
    plain_ms, _, _ = timed_steps(plain_step, plain_steps, stream, dist, flush=flush)
    plain_ms = dist.max(plain_ms)
    plain_ok = bool((m_plain == m_ref).all().item())

    # the same batch through an autotuned keyed plan (one graph launch of the
    # tuner's kernel variant and shape per step)
    tuned = None
    if count >= 4096:
        m_plan = torch.zeros_like(m_ref)
        plan = hqc.hqc_plan_create_keyed(level, u_d, v_d, keys, k_d, m_plan, autotune=True, stream=stream)
        d = plan.describe()
        fn = lambda: plan.launch(stream=stream)
        warm(fn, 3, stream)
        plan_ms, _, _ = timed_steps(fn, steps, stream, dist)
        plan_ms = dist.max(plan_ms)
        tuned = {"value": dist.sum(float(count)) * steps / (plan_ms * 1e-3), "unit": UNIT,
                 "ms_per_step": plan_ms / steps, "variant": d["variant"], "warps_per_cta": d["warps_per_cta"],
                 "ctas_per_sm": d["ctas_per_sm"], "candidates_timed": len(d["candidates"]),
                 "correct": bool((m_plan == m_ref).all().item()),
                 "api": "hqc_plan_create_keyed(autotune) + hqc_plan_launch"}
        plan.destroy()
    total_count = dist.sum(float(count))
    value = total_count * steps / (max_ms * 1e-3)
    plain_value = total_count * plain_steps / (plain_ms * 1e-3)
    smem_b, hbm_b, int_ops = per_decryption_work(P)
    launch_s = (total_ms / steps) * 1e-3  # one launch of the fused kernel per step
    kernel = decrypt_kernel_name(level, count)
    roofline = ctx.roofline(smem_b * count, int_ops * count, hbm_b * count, launch_s, kernel,
                            traffic=traffic_from_profile(level) if count == 65536 or count == 32768 else None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": steps,
        "warmup": warmup, "ms_per_step": max_ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": desc, "level": level, "count_per_gpu": count, "nkeys": nkeys,
                   "inputs_bytes_per_gpu": int(in_bytes), "l2": l2,
                   "launch": hqc.hqc_get_launch_shape(level, True),
                   "parallelism": "replicas" if dist.world > 1 else "single GPU"},
        "correct": correct and plain_ok, "wrong_messages": wrong,
        "latency_ms": {"p50": pct(per, 50), "p99": pct(per, 99), "max": max(per),
                       "what": "one batch of %d decryptions (launch to completion, device events)" % count},
        "plain_per_stage": {"value": plain_value, "unit": UNIT, "ms_per_step": plain_ms / plain_steps,
                            "launches_per_step": 3, "correct": plain_ok},
        "batched_over_per_stage": value / plain_value,
        "roofline": roofline,
        "gpu_launches": steps,
        "clocks": clocks,
    }
    if tuned is not None:
        line["tuned_plan"] = tuned
        line["correct"] = line["correct"] and tuned["correct"]
    if full:
        line["e2e"] = e2e_single(ctx, level, count, P, keys, u_d, v_d, k_d, m_ref, stream)
        line["correct"] = line["correct"] and line["e2e"].pop("correct")
    if full and count > 512:
        line["rm_stage"] = rm_stage_forms(ctx, level, count, stream)
        line["correct"] = (line["correct"] and line["rm_stage"]["equal"]
                           and line["rm_stage"]["tensor_core_timeouts"] == 0)
    if count <= 512:
        line["one_ciphertext_us"] = one_ciphertext_latency(ctx, stream)
        line["correct"] = line["correct"] and all(x["correct"] for x in line["one_ciphertext_us"].values())
    if full and dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        rate, n, dt = oracle_rate(level, nkeys, args.cpu_seconds, cores)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "%d ciphertexts of the same workload recipe (oracle-encrypted), %.1f s"
                                          % (n, dt)}
    keys.free()
    return line


def one_ciphertext_latency(ctx, stream, reps=200):
    """Device time of decrypting ONE ciphertext per level through the keyed
    entry point (the latency form: a four-warp team), median and p99 of
    `reps` launches, each timed alone with events on the launching stream;
    the L2 is flushed before each."""
    import torch
    hqc, dist, device = ctx.hqc, ctx.dist, ctx.device
    out = {}
    for level in (1, 3, 5):
        P, keys, u_d, v_d, k_d, m_ref, _, _ = make_workload(hqc, level, 1, 1, dist.rank, device)
        m = torch.zeros_like(m_ref)
        fn = lambda: hqc.hqc_decrypt_batch_keyed(level, u_d, v_d, keys, k_d, m, stream=stream)
        warm(fn, 5, stream)
        _, per, _ = timed_steps(fn, reps, stream, dist, flush=ctx.flush_l2)
        out[str(level)] = {"p50": 1e3 * pct(per, 50), "p99": 1e3 * pct(per, 99),
                           "correct": bool((m == m_ref).all().item()),
                           "kernel": decrypt_kernel_name(level, 1)}
        keys.free()
    return out


def rm_stage_forms(ctx, level, count, stream, reps=10):
    """S5-S7 alone on count received words (seeded random bits; the decoders'
    work does not depend on the bits): the register butterflies of the
    per-stage form against the tensor-core product (tcgen05), median device
    time of `reps` launches each, and whether their bytes agree."""
    import torch
    import synth
    hqc = ctx.hqc
    P = hqc.hqc_get_params(level)
    w = torch.from_numpy(synth.words(count * P.W_v, tag=990 + level).view(np.int64).reshape(count, P.W_v)).to(
        ctx.device)
    out, times = {}, {}
    for tc in (False, True):
        r = torch.zeros((count, P.n1), dtype=torch.uint8, device=ctx.device)
        fn = lambda: hqc.hqc_rm_decode_batch(level, w, r_out=r, tensor_cores=tc, stream=stream)
        warm(fn, 3, stream)
        _, per, _ = timed_steps(fn, reps, stream, ctx.dist)
        out[tc], times[tc] = r, 1e3 * pct(per, 50)
    return {"rm_blocks": count * P.n1, "butterflies_us": times[False], "tensor_cores_us": times[True],
            "equal": bool(torch.equal(out[False], out[True])), "tensor_core_timeouts": hqc.hqc_rm_tc_timeouts(),
            "what": "hqc_rm_decode_batch: k_stage_rm (register butterflies) vs k_rm_tc (tcgen05.mma kind::f16, "
                    "fp32 accumulators in tensor memory); median device time per launch"}


def e2e_single(ctx, level, count, P, keys, u_d, v_d, k_d, m_ref, stream):
    """End to end through hqc_decrypt_host_keyed: pinned host buffers in, m
    out, copies inside the timed region."""
    import torch
    hqc, dist, args, device = ctx.hqc, ctx.dist, ctx.args, ctx.device
    u_h = u_d.cpu().pin_memory()
    v_h = v_d.cpu().pin_memory()
    k_h = k_d.cpu().pin_memory()
    m_h = torch.empty(m_ref.shape, dtype=torch.uint8).pin_memory()
    u_e, v_e, k_e, m_e = torch.empty_like(u_d), torch.empty_like(v_d), torch.empty_like(k_d), torch.empty_like(m_ref)
    ws_host = torch.empty(hqc.hqc_host_workspace_bytes(level, min(count, 16384)), dtype=torch.uint8, device=device)

    def e2e_step():
        hqc.hqc_decrypt_host_keyed(level, u_h, v_h, keys, k_h, m_h, workspace=ws_host, stream=stream)

    def serial_step():
        u_e.copy_(u_h, non_blocking=True)
        v_e.copy_(v_h, non_blocking=True)
        k_e.copy_(k_h, non_blocking=True)
        hqc.hqc_decrypt_batch_keyed(level, u_e, v_e, keys, k_e, m_e, stream=stream)
        m_h.copy_(m_e, non_blocking=True)

    e2e_steps = max(5, min(args.steps, 100))
    m_cpu = m_ref.cpu()
    warm(serial_step, 3, stream)
    serial_ms, _, _ = timed_steps(serial_step, e2e_steps, stream, dist)
    serial_ms = dist.max(serial_ms)
    serial_ok = bool((m_h == m_cpu).all().item())
    m_h.zero_()
    warm(e2e_step, 3, stream)
    e2e_ms, _, _ = timed_steps(e2e_step, e2e_steps, stream, dist)
    e2e_ms = dist.max(e2e_ms)
    e2e_ok = bool((m_h == m_cpu).all().item()) and serial_ok

    # the host link alone: the same bytes copied up without decrypting
    def link_step():
        u_e.copy_(u_h, non_blocking=True)
        v_e.copy_(v_h, non_blocking=True)
        k_e.copy_(k_h, non_blocking=True)

    link_ms, _, _ = timed_steps(link_step, e2e_steps, stream, dist)
    link_ms = dist.max(link_ms)
    h2d = u_h.numel() * 8 + v_h.numel() * 8 + k_h.numel() * 4
    total = dist.sum(float(count))
    return {"value": total * e2e_steps / (e2e_ms * 1e-3), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": m_h.numel(), "steps": e2e_steps,
            "api": "hqc_decrypt_host_keyed: pinned host u, v, key_idx in, m out, chunked copies "
                   "overlapped with the fused kernel",
            "serial": {"value": total * e2e_steps / (serial_ms * 1e-3),
                       "api": "copy in, hqc_decrypt_batch_keyed, copy out, one after another"},
            "h2d_link_gbs": h2d * e2e_steps / (link_ms * 1e-3) / 1e9,
            "link_bound": total * e2e_steps / (link_ms * 1e-3),
            "link_what": "decryptions/s the host-to-device copy of the inputs alone allows",
            "correct": e2e_ok}


def bench_mixed(ctx, full):
    """Mixed-level batch: autotuned CUDA-graph plan vs the single mixed kernel,
    per-level fused launches and the plain per-stage form."""
    import torch
    import synth
    hqc, dist, args, device = ctx.hqc, ctx.dist, ctx.args, ctx.device
    _, count, nkeys_total, desc = WORKLOADS["mixed"]
    nk = nkeys_total // 3
    steps, warmup = (args.steps, args.warmup) if full else sub_steps(args)
    per = {}
    for lvl, cnt in MIXED_SPLIT:
        per[lvl] = make_workload(hqc, lvl, cnt, nk, dist.rank, device)
    # shuffled item order and arena layout (u row then v row per item)
    seq_lvl = np.concatenate([np.full(cnt, lvl, np.int32) for lvl, cnt in MIXED_SPLIT])
    seq_idx = np.concatenate([np.arange(cnt, dtype=np.int64) for _, cnt in MIXED_SPLIT])
    order = synth.shuffle(np.arange(count, dtype=np.int32), tag=77)
    seq_lvl, seq_idx = seq_lvl[order], seq_idx[order]
    P = {lvl: per[lvl][0] for lvl, _ in MIXED_SPLIT}
    wu = np.array([0, P[1].W_u_pitch, 0, P[3].W_u_pitch, 0, P[5].W_u_pitch])[seq_lvl]
    wv = np.array([0, P[1].W_v, 0, P[3].W_v, 0, P[5].W_v])[seq_lvl]
    kk = np.array([0, P[1].k, 0, P[3].k, 0, P[5].k])[seq_lvl]
    u_off = np.concatenate([[0], np.cumsum(wu + wv)[:-1]])
    v_off = u_off + wu
    m_off = np.concatenate([[0], np.cumsum(kk)[:-1]])
    words = int((wu + wv).sum())
    m_bytes = int(kk.sum())
    arena = torch.empty(words, dtype=torch.int64, device=device)
    m_expect = torch.empty(m_bytes, dtype=torch.uint8, device=device)
    items = np.zeros(count, dtype=hqc.ITEM_DTYPE)
    items["level"] = seq_lvl
    items["u_off"] = u_off
    items["v_off"] = v_off
    items["m_off"] = m_off
    for lvl, cnt in MIXED_SPLIT:
        Pl, keys, u_d, v_d, k_d, m_ref, y_host, kidx = per[lvl]
        sel = np.nonzero(seq_lvl == lvl)[0]
        src = torch.from_numpy(seq_idx[sel]).to(device)
        items["key"][sel] = kidx[seq_idx[sel]]
        ui = torch.from_numpy(u_off[sel]).to(device)[:, None] + torch.arange(Pl.W_u_pitch, device=device)
        vi = torch.from_numpy(v_off[sel]).to(device)[:, None] + torch.arange(Pl.W_v, device=device)
        mi = torch.from_numpy(m_off[sel]).to(device)[:, None] + torch.arange(Pl.k, device=device)
        arena[ui.reshape(-1)] = u_d[src].reshape(-1)
        arena[vi.reshape(-1)] = v_d[src].reshape(-1)
        m_expect[mi.reshape(-1)] = m_ref[src].reshape(-1)
    items_d = torch.from_numpy(items.view(np.uint8)).to(device)
    keys3 = [per[l][1] for l in (1, 3, 5)]
    m_out = torch.zeros(m_bytes, dtype=torch.uint8, device=device)
    stream = torch.cuda.Stream(device=device)
    torch.cuda.synchronize()

    t0 = time.perf_counter()
    if args.mixed_plan == "auto":
        plan = hqc.hqc_plan_create_mixed(items_d, arena, keys3, m_out, autotune=True, stream=stream)
    else:
        f = args.mixed_plan.split(":")
        plan = hqc.hqc_plan_create_mixed(items_d, arena, keys3, m_out, stream=stream, form=int(f[0]),
                                         variants=f[1].split(",") if len(f) > 1 else None,
                                         grids=[int(x) for x in f[2].split(",")] if len(f) > 2 else None)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    info = plan.info()
    desc = plan.describe()
    info["level_variants"] = desc["level_variants"]
    info["best_ms_per_form"] = {}
    for c in desc["candidates"]:  # fastest first; whole-batch runs only
        if c["whole_batch"]:
            info["best_ms_per_form"].setdefault(c["form"], c["ms"])
    info["candidates_timed"] = len(desc["candidates"])

    def step():
        plan.launch(stream=stream)

    warm(step, warmup, stream)
    total_ms, per_ms, clocks = timed_steps(step, steps, stream, dist, clocks_idx=dist.local if full else None)
    max_ms = dist.max(total_ms)
    correct = bool((m_out == m_expect).all().item())

    def arm(fn, n):
        warm(fn, 3, stream)
        ms, _, _ = timed_steps(fn, n, stream, dist)
        return dist.max(ms) / n

    arm_steps = max(5, min(steps, 100))
    ws_mixed = torch.zeros(hqc.hqc_mixed_workspace_bytes(), dtype=torch.uint8, device=device)
    m_single = torch.zeros_like(m_out)
    single_ms = arm(lambda: hqc.hqc_decrypt_mixed(items_d, arena, keys3, m_single, workspace=ws_mixed, stream=stream),
                    arm_steps)
    single_ok = bool((m_single == m_expect).all().item())
    outs = {lvl: torch.empty_like(per[lvl][5]) for lvl, _ in MIXED_SPLIT}

    def fused_levels():
        for lvl, _ in MIXED_SPLIT:
            Pl, keys, u_d, v_d, k_d, m_ref, _, _ = per[lvl]
            hqc.hqc_decrypt_batch_keyed(lvl, u_d, v_d, keys, k_d, outs[lvl], stream=stream)

    levels_ms = arm(fused_levels, arm_steps)
    levels_ok = all(bool((outs[l] == per[l][5]).all().item()) for l, _ in MIXED_SPLIT)
    wss = {lvl: torch.empty(hqc.hqc_staged_workspace_bytes(lvl, cnt), dtype=torch.uint8, device=device)
           for lvl, cnt in MIXED_SPLIT}
    outs2 = {lvl: torch.empty_like(per[lvl][5]) for lvl, _ in MIXED_SPLIT}

    def staged_levels():
        for lvl, _ in MIXED_SPLIT:
            Pl, keys, u_d, v_d, k_d, m_ref, _, _ = per[lvl]
            hqc.hqc_decrypt_batch_staged(lvl, u_d, v_d, keys=keys, key_idx=k_d, workspace=wss[lvl], m_out=outs2[lvl],
                                         stream=stream)

    staged_ms = arm(staged_levels, arm_steps)
    staged_ok = all(bool((outs2[l] == per[l][5]).all().item()) for l, _ in MIXED_SPLIT)

    total = dist.sum(float(count))
    value = total * steps / (max_ms * 1e-3)
    plain_value = total / (staged_ms * 1e-3)
    smem_b = sum(cnt * per_decryption_work(P[l])[0] for l, cnt in MIXED_SPLIT)
    int_ops = sum(cnt * per_decryption_work(P[l])[2] for l, cnt in MIXED_SPLIT)
    hbm_b = sum(cnt * per_decryption_work(P[l])[1] for l, cnt in MIXED_SPLIT)
    step_s = (total_ms / steps) * 1e-3
    roofline = ctx.roofline(smem_b, int_ops, hbm_b, step_s, "mixed plan (%s)" % info["form"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": steps,
        "warmup": warmup, "ms_per_step": max_ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": desc, "count_per_gpu": count, "split": dict((str(l), c) for l, c in MIXED_SPLIT),
                   "nkeys": nkeys_total, "plan": info, "autotune_s": tune_s,
                   "l2": "inputs (%d MB) larger than L2 (129 MB); no flush" % (words * 8 // 2 ** 20)},
        "correct": correct and single_ok and staged_ok and levels_ok,
        "wrong_messages": int((m_out != m_expect).sum().item()),
        "latency_ms": {"p50": pct(per_ms, 50), "p99": pct(per_ms, 99), "max": max(per_ms),
                       "what": "one mixed batch of %d decryptions (graph launch to completion)" % count},
        "single_mixed_kernel": {"value": total / (single_ms * 1e-3), "ms_per_step": single_ms, "correct": single_ok},
        "per_level_fused": {"value": total / (levels_ms * 1e-3), "ms_per_step": levels_ms, "launches_per_step": 3,
                            "correct": levels_ok},
        "plain_per_stage": {"value": plain_value, "unit": UNIT, "ms_per_step": staged_ms,
                            "launches_per_step": 9, "correct": staged_ok},
        "batched_over_per_stage": value / plain_value,
        "roofline": roofline,
        "gpu_launches": steps * (1 if info["form"] == "mixed-single-kernel" else 3),
        "clocks": clocks,
    }
    if full:
        line["e2e"] = e2e_mixed(ctx, count, arena, items_d, keys3, m_out, m_expect, stream)
        line["correct"] = line["correct"] and line["e2e"].pop("correct")
    if full and dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        rates = {}
        for lvl, cnt in MIXED_SPLIT:
            rates[lvl] = oracle_rate(lvl, 16, args.cpu_seconds / 3, cores)
        t_total = sum(cnt / rates[l][0] for l, cnt in MIXED_SPLIT)
        line["cpu_baseline"] = {"value": count / t_total, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "per level %s ciphertexts timed separately, combined in the 40/35/25 mix"
                                          % {l: rates[l][1] for l, _ in MIXED_SPLIT}}
    plan.destroy()
    for l in (1, 3, 5):
        per[l][1].free()
    return line


def e2e_mixed(ctx, count, arena, items_d, keys3, m_out, m_expect, stream):
    """The arena and item list from pinned host memory, m back."""
    import torch
    hqc, dist, args, device = ctx.hqc, ctx.dist, ctx.args, ctx.device
    m_bytes = m_out.numel()
    arena_h = arena.cpu().pin_memory()
    items_h = items_d.cpu().pin_memory()
    m_h = torch.empty(m_bytes, dtype=torch.uint8).pin_memory()
    arena_e, items_e, m_e = torch.empty_like(arena), torch.empty_like(items_d), torch.zeros_like(m_out)
    ws_e = torch.zeros(hqc.hqc_mixed_workspace_bytes(), dtype=torch.uint8, device=device)

    def arm(fn, n):
        warm(fn, 3, stream)
        ms, _, _ = timed_steps(fn, n, stream, dist)
        return dist.max(ms) / n

    def serial_step():
        arena_e.copy_(arena_h, non_blocking=True)
        items_e.copy_(items_h, non_blocking=True)
        hqc.hqc_decrypt_mixed(items_e, arena_e, keys3, m_e, workspace=ws_e, stream=stream)
        m_h.copy_(m_e, non_blocking=True)

    e2e_steps = max(5, min(args.steps, 50))
    serial_ms = arm(serial_step, e2e_steps)
    m_cpu = m_expect.cpu()
    ok = bool((m_h == m_cpu).all().item())
    # pipelined: chunks of records and arena ranges uploaded while the
    # previous chunk decrypts; a few chunk counts tried, the best kept
    tried = {}
    for nch in (2, 4, 8):
        c = (count + nch - 1) // nch
        ws_p = torch.empty(hqc.hqc_mixed_host_workspace_bytes(items_h, c), dtype=torch.uint8, device=device)
        fn = (lambda c=c, ws_p=ws_p: hqc.hqc_decrypt_mixed_host(items_h, arena_h, keys3, m_h, chunk=c,
                                                                  workspace=ws_p, stream=stream))
        tried[c] = (arm(fn, 3), fn)
    best = min(tried, key=lambda c: tried[c][0])
    m_h.zero_()
    e2e_ms = arm(tried[best][1], e2e_steps)
    ok = ok and bool((m_h == m_cpu).all().item())
    total = dist.sum(float(count))
    return {"value": total / (e2e_ms * 1e-3), "unit": UNIT,
            "h2d_bytes_per_step": int(arena_h.numel() * 8 + items_h.numel()), "d2h_bytes_per_step": m_bytes,
            "api": "hqc_decrypt_mixed_host: pinned host arena and item list in, m out, chunked uploads "
                   "overlapped with per-level kernels",
            "chunk": best, "chunks_tried_ms": {str(c): v[0] for c, v in tried.items()},
            "serial": {"value": total / (serial_ms * 1e-3),
                       "api": "copy in, hqc_decrypt_mixed (one mixed kernel), copy out"},
            "correct": ok}


def bench_serving(ctx, full):
    """Continuous-batching service loop at several offered loads."""
    import torch
    import synth
    hqc, dist, args, device = ctx.hqc, ctx.dist, ctx.args, ctx.device
    period = 65536
    levels = synth.level_mix(period, ((1, 0.40), (3, 0.35), (5, 0.25)), tag=201)
    per, rows_by_level = {}, {}
    for l in (1, 3, 5):
        cnt = int((levels == l).sum())
        per[l] = make_workload(hqc, l, cnt, 128, dist.rank, device)
        P, keys, u_d, v_d, k_d, m_d, y, kidx = per[l]
        rows_by_level[l] = (u_d.cpu().numpy(), v_d.cpu().numpy(), kidx, m_d.cpu().numpy(), P)
    used = {1: 0, 3: 0, 5: 0}
    parts, key, woff, moff, want = [], np.zeros(period, np.int32), [0], [0], []
    for idx, l in enumerate(levels):
        u, v, kidx, m, P = rows_by_level[int(l)]
        i = used[int(l)]
        used[int(l)] += 1
        parts += [u[i], v[i]]
        key[idx] = kidx[i]
        woff.append(woff[-1] + P.W_u_pitch + P.W_v)
        moff.append(moff[-1] + P.k)
        want.append(m[i])
    words = torch.from_numpy(np.concatenate(parts)).pin_memory()
    woff = np.array(woff, np.int64)
    moff = np.array(moff, np.int64)
    want = np.concatenate(want)
    keys3 = [per[l][1] for l in (1, 3, 5)]
    serve_kw = dict(streams=4, max_batch=16384, budget_bytes=256 << 20, max_queue=1 << 22)
    points = []
    # the default bench line runs 2 s per offered load so that every
    # configuration fits its minute; `--workload serving --serve-seconds 30`
    # runs the full 30 s points (3e8 requests at 1e7 req/s: about 6 GB of
    # host-side arrival, status and latency arrays)
    duration = max(0.2, min(30.0 if full else 2.0, args.serve_seconds))
    warm_s = 0.25
    for load in SERVE_LOADS:
        arr = synth.burst_trace(load, duration, tag=301 + int(np.log10(load)))
        # clocks are read just before and just after each point: an NVML
        # query while the loop runs holds the driver long enough to show in
        # the tail latencies, so the read comes before the point's warm-up
        clk_before = clocks_now(dist.local)
        # warm-up at the point's own load (its own trace), not measured
        hqc.hqc_serve_run(keys3, levels, key, woff, words, moff,
                          synth.burst_trace(load, warm_s, tag=300 + int(np.log10(load))), **serve_kw)
        st, lat, m_out, stats = hqc.hqc_serve_run(keys3, levels, key, woff, words, moff, arr, **serve_kw)
        clk_after = clocks_now(dist.local)
        ok = st == 0
        good = True
        idx = np.nonzero(ok)[0]
        # every completed ring entry must hold its message (later writers repeat it)
        done_entries = np.nonzero(np.bincount(idx % period, minlength=period))[0]
        for j in done_entries[:: max(1, len(done_entries) // 2000)]:
            good &= bool((m_out[moff[j]:moff[j + 1]] == want[moff[j]:moff[j + 1]]).all())
        l_us = lat[ok] / 1e3
        pct = [float(x) for x in np.percentile(l_us, [50, 99, 99.9])] if l_us.size else [None] * 3
        points.append({
            "offered_req_per_s": load, "requests": int(len(arr)), "completed": int(stats["completed"]),
            "rejected": int(stats["rejected_queue"] + stats["rejected_size"] + stats["rejected_invalid"]),
            "sustained_dec_per_s": stats["completed"] / (stats["wall_ns"] * 1e-9) if stats["wall_ns"] else None,
            "p50_us": pct[0], "p99_us": pct[1], "p999_us": pct[2],
            "batches": int(stats["batches"]), "mean_batch": stats["mean_batch"], "correct": good,
            "transfer": "in place (kernels read the pinned host ring)" if stats["in_place"] else "copy engines",
            "clocks": {"before": clk_before, "after": clk_after}})
    top = points[-1]
    line = {
        "metric": METRIC, "value": top["sustained_dec_per_s"], "unit": UNIT, "n_gpus": dist.world,
        "steps": len(points), "warmup": len(points), "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOADS["serving"][3], "duration_s_per_point": duration,
                   "warmup_s_per_point": warm_s, "ring_requests": period,
                   "streams": 4, "max_batch": 16384, "budget_bytes": 256 << 20},
        "latency_us": {"p50": top["p50_us"], "p99": top["p99_us"], "p99.9": top["p999_us"]},
        "points": points,
        "correct": all(p["correct"] for p in points),
        "e2e": {"value": top["sustained_dec_per_s"], "unit": UNIT,
                "h2d_bytes_per_step": int(woff[-1] * 8), "d2h_bytes_per_step": int(moff[-1]),
                "api": "hqc_serve_run: " + top["transfer"] + "; m returned to host memory per batch"},
        "gpu_launches": int(sum(p["batches"] for p in points)),
        "clocks": top["clocks"]["after"],
    }
    for l in (1, 3, 5):
        per[l][1].free()
    return line


def clocks_now(gpu_index):
    """One nvidia-smi sample of the SM clock and throttle reasons."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + Clocks.QUERY,
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10).stdout
        r = out.strip().split(",")
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        return {"sm_mhz": float(r[1]), "sm_max_mhz": float(r[2]),
                "reasons": sorted(n for n, v in zip(names, r[5:9]) if v.strip().lower() == "active")}
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}


def keccak_perms(n_bytes):
    """Keccak-f[1600] calls to absorb n_bytes with SHAKE256 (rate 136)."""
    return n_bytes // 136 + 1


KECCAK_OPS = 180 * 24  # 32-bit funnel / 3-input logic ops per permutation (theta, rho-pi, chi, iota)


def per_decaps_work(P):
    """Algorithmic 32-bit ALU ops of one decapsulation, by kernel."""
    _, _, dec_ops = per_decryption_work(P)
    N32 = (P.n + 31) // 32
    W_v32 = P.n1 * P.n2 // 32
    enc_ops = 2 * P.wr * N32 + 2 * P.wr * W_v32 + P.n1 * 4 * P.mult + (P.k * (2 * P.delta)) * 4 + N32 + W_v32
    words = 2 * P.wr + P.we
    derive_perms = keccak_perms(P.k + 17) + 1 + (words - 1) // 34
    derive_ops = derive_perms * KECCAK_OPS + 2 * (2 * P.wr * P.wr // 2 + P.we * P.we // 2)
    k_len = P.k + (P.n + 7) // 8 + P.n1 * P.n2 // 8 + 17
    K_ops = keccak_perms(k_len) * KECCAK_OPS
    return {"decrypt": dec_ops, "derive": derive_ops, "encrypt_compare": enc_ops, "K": K_ops}


def bench_kem(ctx, wl_name, full):
    """Batched KEM decapsulation (and encapsulation) on seeded key pairs."""
    import torch
    import synth
    hqc, dist, args, device = ctx.hqc, ctx.dist, ctx.args, ctx.device
    level, count, nkeys, desc = WORKLOADS[wl_name]
    P = hqc.hqc_get_params(level)
    tag = 7000 + 100 * level + 10 * dist.rank
    steps, warmup = (args.steps, args.warmup) if full else sub_steps(args)

    def rows(cnt, width, t):
        nw = (cnt * width + 7) // 8 + 1
        a = synth.words(nw, tag=t).view(np.uint8)[:cnt * width].reshape(cnt, width)
        return torch.from_numpy(a.copy()).to(device)

    seed_sk, seed_pk = rows(nkeys, 32, tag), rows(nkeys, 32, tag + 1)
    sigma = rows(nkeys, P.k, tag + 2)
    kidx = torch.from_numpy(synth.key_assignment(count, nkeys, tag=tag + 3)).to(device)
    m = rows(count, P.k, tag + 4)
    salt = rows(count, 16, tag + 5)
    h, x, y, s = hqc.hqc_kem_keygen(level, seed_sk, seed_pk)
    torch.cuda.synchronize()
    keys = hqc.Keyset(level, y.cpu().numpy().view(np.uint32))
    ws = torch.empty(hqc.hqc_kem_workspace_bytes(level, count), dtype=torch.uint8, device=device)
    stream = torch.cuda.Stream(device=device)
    u = torch.empty((count, P.W_u_pitch), dtype=torch.int64, device=device)
    v = torch.empty((count, P.W_v), dtype=torch.int64, device=device)
    K_enc = torch.empty((count, 32), dtype=torch.uint8, device=device)
    K_dec = torch.empty_like(K_enc)
    ok = torch.empty((count,), dtype=torch.int32, device=device)
    m_dec = torch.empty((count, P.k), dtype=torch.uint8, device=device)

    def encaps():
        hqc.hqc_kem_encaps(level, h, s, kidx, m, salt, u, v, K_enc, workspace=ws, stream=stream)

    def decaps():
        hqc.hqc_kem_decaps(level, keys, h, s, sigma, kidx, u, v, salt, K_dec, ok, workspace=ws, stream=stream)

    def decrypt_only():
        hqc.hqc_decrypt_batch_keyed(level, u, v, keys, kidx, m_dec, stream=stream)

    with torch.cuda.stream(stream):
        encaps()
    warm(decaps, warmup, stream)
    total_ms, per, clocks = timed_steps(decaps, steps, stream, dist, clocks_idx=dist.local if full else None)
    max_ms = dist.max(total_ms)
    correct = bool(ok.all().item()) and bool((K_dec == K_enc).all().item())
    sub = max(5, min(steps, 50))
    warm(encaps, 3, stream)
    enc_ms, _, _ = timed_steps(encaps, sub, stream, dist)
    enc_ms = dist.max(enc_ms)
    warm(decrypt_only, 3, stream)
    dec_ms, _, _ = timed_steps(decrypt_only, sub, stream, dist)
    dec_ms = dist.max(dec_ms)
    correct = correct and bool((m_dec == m).all().item())
    # implicit rejection on a tampered copy: every item rejected, K = K(sigma, c)
    v_bad = v.clone()
    v_bad[:, 1] ^= 1 << 20
    K_bad = torch.empty_like(K_enc)
    ok_bad = torch.empty_like(ok)
    hqc.hqc_kem_decaps(level, keys, h, s, sigma, kidx, u, v_bad, salt, K_bad, ok_bad, workspace=ws, stream=stream)
    torch.cuda.synchronize()
    rejected_ok = not bool(ok_bad.any().item())

    work = per_decaps_work(P)
    ops = sum(work.values())
    step_s = (total_ms / steps) * 1e-3
    alu_peak = ctx.peaks["alu_ops_per_s"] / 1e9
    issue_peak = ctx.peaks["issue_ops_per_s"] / 1e9
    int_ach = ops * count / step_s / 1e9
    hbm_b = 3 * (P.W_u_pitch + P.W_v) * 8 + P.k * 2 + 16 * 2 + 32 + 8 + 4 * (2 * P.wr + P.we) * 2
    roofline = {"bound": "alu", "achieved": int_ach, "peak": alu_peak, "unit": "Gop/s",
                "frac": int_ach / alu_peak if alu_peak else None, "traffic": None,
                "kernel": "whole decapsulation step (4 kernels)",
                "ops_per_item": work,
                "peak_source": "measured in this run: 32-bit funnel-shift + XOR issue rate, all SMs",
                "issue": {"peak": issue_peak, "frac": int_ach / issue_peak if issue_peak else None},
                "others": {"hbm": {"bound": "hbm", "achieved": hbm_b * count / step_s / 1e9,
                                   "peak": ctx.hbm_peak, "unit": "GB/s"}}}
    total = dist.sum(float(count))
    value = total * steps / (max_ms * 1e-3)
    line = {
        "metric": "HQC KEM decapsulations/sec per GB300", "value": value, "unit": KEM_UNIT, "n_gpus": dist.world,
        "steps": steps, "warmup": warmup, "ms_per_step": max_ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": desc, "level": level, "count_per_gpu": count, "nkeys": nkeys,
                   "l2": "inputs (%d MB) larger than L2 (129 MB); no flush" % ((u.numel() + v.numel()) * 8 // 2 ** 20),
                   "parallelism": "replicas" if dist.world > 1 else "single GPU"},
        "correct": correct, "implicit_rejection_ok": rejected_ok,
        "latency_ms": {"p50": pct(per, 50), "p99": pct(per, 99), "max": max(per)},
        "encaps": {"value": total * sub / (enc_ms * 1e-3), "unit": "encapsulations/s", "ms_per_step": enc_ms / sub},
        "decrypt_only": {"value": total * sub / (dec_ms * 1e-3), "unit": UNIT, "ms_per_step": dec_ms / sub},
        "roofline": roofline,
        "gpu_launches": 4 * steps,
        "clocks": clocks,
    }
    if full:
        line["e2e"] = e2e_kem(ctx, level, count, keys, h, s, sigma, kidx, u, v, salt, K_enc, stream)
        line["correct"] = line["correct"] and line["e2e"].pop("correct")
    if full and dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        import oracle
        cores = os.cpu_count() or 1
        n = max(4 * cores, 32)
        hh, ss, yy = (t.cpu().numpy().view(np.uint64 if t.dtype == torch.int64 else np.uint32) for t in (h, s, y))
        t0 = time.perf_counter()
        Ko, oko = oracle.kem_decaps(level, hh, ss, yy, sigma.cpu().numpy(), kidx[:n].cpu().numpy(),
                                    u[:n].cpu().numpy().view(np.uint64), v[:n].cpu().numpy().view(np.uint64),
                                    salt[:n].cpu().numpy(), nthreads=cores)
        dt = time.perf_counter() - t0
        line["correct"] = line["correct"] and bool(oko.all()) and bool((Ko == K_enc[:n].cpu().numpy()).all())
        line["cpu_baseline"] = {"value": n / dt, "unit": KEM_UNIT, "cores": cores, "kind": "oracle",
                                "sample": "%d decapsulations of the same workload, %.1f s" % (n, dt)}
    keys.free()
    return line


def e2e_kem(ctx, level, count, keys, h, s, sigma, kidx, u, v, salt, K_enc, stream):
    """Pinned host ciphertexts and salts in, K out, chunked so the uploads
    overlap the kernels."""
    import torch
    hqc, dist, args, device = ctx.hqc, ctx.dist, ctx.args, ctx.device
    u_h, v_h, s_h, k_h = (t.cpu().pin_memory() for t in (u, v, salt, kidx))
    K_h = torch.empty((count, 32), dtype=torch.uint8).pin_memory()
    ok_h = torch.empty((count,), dtype=torch.int32).pin_memory()
    ws_host = torch.empty(hqc.hqc_kem_host_workspace_bytes(level, count), dtype=torch.uint8, device=device)
    chunk_sel = {"chunk": 0}

    def e2e_step():
        hqc.hqc_kem_decaps_host(level, keys, h, s, sigma, k_h, u_h, v_h, s_h, K_h, ok_h, chunk=chunk_sel["chunk"],
                                workspace=ws_host, stream=stream)

    # the chunk count trades copy overlap against kernel occupancy: try a few
    tried = {}
    for c in (count, (count + 1) // 2, (count + 3) // 4):
        chunk_sel["chunk"] = c
        warm(e2e_step, 1, stream)
        tried[c], _, _ = timed_steps(e2e_step, 3, stream, dist)
    chunk_sel["chunk"] = min(tried, key=tried.get)
    sub = max(5, min(args.steps, 50))
    warm(e2e_step, 3, stream)
    e2e_ms, _, _ = timed_steps(e2e_step, sub, stream, dist)
    e2e_ms = dist.max(e2e_ms)
    ok = bool((K_h == K_enc.cpu()).all().item()) and bool(ok_h.all().item())
    h2d = sum(t.numel() * t.element_size() for t in (u_h, v_h, s_h, k_h))
    return {"value": dist.sum(float(count)) * sub / (e2e_ms * 1e-3), "unit": KEM_UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": K_h.numel() + 4 * ok_h.numel(), "steps": sub,
            "api": "hqc_kem_decaps_host: pinned host u, v, salt, key_idx in, K and ok out, chunked "
                   "copies overlapped with the kernels",
            "chunk": chunk_sel["chunk"], "chunks_tried_ms": {str(k): v / 3 for k, v in tried.items()},
            "correct": ok}


# The sub-configurations the default run adds beside its headline: every
# configuration of the benchmark recipe, each with its own correctness
# check, its per-stage comparison where one exists, and its roofline.
SUB_CONFIGS = (
    ("C1_hqc1_plain", "single", "hqc1-plain"),
    ("C3_hqc3", "single", "hqc3"),
    ("C3_hqc5", "single", "hqc5"),
    ("C4_mixed", "mixed", "mixed"),
    ("C5_serving", "serving", "serving"),
    ("KEM_hqc1_decaps", "kem", "kem1-decaps"),
)


def compact(line):
    """A sub-configuration's result without the keys of the headline
    contract that only the top-level line carries."""
    drop = ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "dtype", "data")
    return {k: v for k, v in line.items() if k not in drop}


def run_sub_configs(ctx):
    import torch
    out = {}
    for name, kind, wl in SUB_CONFIGS:
        t0 = time.perf_counter()
        try:
            if kind == "single":
                line = bench_single(ctx, wl, full=False)
            elif kind == "mixed":
                line = bench_mixed(ctx, full=False)
            elif kind == "serving":
                line = bench_serving(ctx, full=False)
            else:
                line = bench_kem(ctx, wl, full=False)
            res = compact(line)
        except Exception as exc:  # a failing sub-configuration is reported, not hidden
            res = {"error": "%s: %s" % (type(exc).__name__, exc), "correct": False}
        res["wall_s"] = time.perf_counter() - t0
        out[name] = res
        torch.cuda.empty_cache()
    return out


def run_ours(args):
    ctx = Ctx(args)
    if args.workload == "mixed":
        line = bench_mixed(ctx, full=True)
    elif args.workload == "serving":
        line = bench_serving(ctx, full=True)
    elif args.workload in KEM_WORKLOADS:
        line = bench_kem(ctx, args.workload, full=True)
    else:
        line = bench_single(ctx, args.workload, full=True)
    want_configs = args.configs == "all" or (args.configs == "auto" and args.workload == "hqc1-bulk"
                                              and ctx.dist.world == 1)
    line["profiles"] = profile_freshness()
    if want_configs:
        line["configs"] = run_sub_configs(ctx)
        line["configs_all_correct"] = all(c.get("correct") is True for c in line["configs"].values())
    if ctx.dist.rank == 0:
        print(json.dumps(line), flush=True)
    ctx.dist.close()
    return 0


def profile_freshness():
    """For each committed ncu summary that records the kernel-source digest
    it was captured at: whether that digest is today's (its counters still
    describe the kernels), else 'stale'."""
    import glob
    import re
    from paper_2512_12904_gb300 import _build
    now = _build.kernel_digest()
    out = {}
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        m = re.search(r"digest at capture: `([0-9a-f]+)`", open(f).read())
        if m:
            out[os.path.basename(f)] = "current" if m.group(1) == now else "stale"
    return out


def traffic_from_profile(level):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary, if current."""
    path = os.path.join(ROOT, "profiles", "dram_traffic_per_launch.txt")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    from paper_2512_12904_gb300 import _build
    ent = rec.get("hqc%d" % level)
    if not ent or ent.get("kernel_digest") != _build.kernel_digest():
        return None
    return ent.get("dram_bytes_per_launch")


def main():
    global KEY_OFFSET
    args = parse_args()
    KEY_OFFSET = args.key_offset
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
