#!/usr/bin/env python3
"""Benchmark: batched SPHINCS+-SHA2-128f-simple signing on one GB300.

Workload (one "step"): one hs_sign_batch call over 16384 random 32-byte
messages signed by 16 seeded keys (key i mod 16), i.e. the whole hot path --
message stage, FORS_Sign, TREE_Sign, WOTS+_Sign -- for one batch.  Inputs
are device-resident when the timed region starts; the 280 MB of signatures
written per step exceed L2, and L2 is additionally flushed (256 MB write)
between timed steps, outside the timed events.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores instead (the reference arm for this workload).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "signatures/s at 128f/192f/256f on 1 GB300; % integer-pipe peak; p99 sign latency"
WORKLOAD = "SPHINCS+-SHA2-128f-simple, 16 keys, 16384 x 32 B messages, one batched call per step"

# Algorithmic SHA-2 compressions per signature of each stage (after the
# per-key PK.seed midstate), from the scheme's structure:
#   TREE: d 2^h' leaves x len chains x 16 (PRF + 15 F), + T_len blocks per leaf, + H per tree
#   FORS: k 2^a x 2 (PRF + F) + k (2^a - 1) H + T_k blocks
#   WOTS: d len PRF + expected digit sum (7.5 per chain) F
# and the idealised integer instructions per compression (rounds 14 ops,
# schedule 10 ops per word, feed-forward 8): 1384 per SHA-256 block; a
# SHA-512 block on 32-bit lanes ~4000.
OPS_C256 = 1384
OPS_C512 = 4000
# Of those, the work that only the ALU pipe (LOP3 / SHF / PRMT) can execute:
# rotations, shifts and 3-input logic -- per SHA-256 round Sigma0, Sigma1 (3
# rotations + 1 LOP3 each), Ch, Maj (1 LOP3 each) = 10, per schedule word
# sigma0, sigma1 = 8 -> 64 x 10 + 48 x 8 = 1024; per SHA-512 compression on
# 32-bit lanes (every 64-bit rotation or XOR is two 32-bit ops) 80 x 20 +
# 64 x 16 = 2624.  Additions can run on the FMA pipe and are not counted.
ALU_C256 = 1024
ALU_C512 = 2624
STAGE_WORK = {
    # set: {stage: (c256, c512)}
    "128f": {"tree": (22 * 8 * 35 * 16 + 22 * 8 * 10 + 22 * 7, 0),
             "fors": (33 * 64 * 2 + 33 * 63 + 9, 0),
             "wots": (22 * 35 * (1 + 7.5), 0)},
    "192f": {"tree": (22 * 8 * 51 * 16, 22 * 8 * 10 + 22 * 7),
             "fors": (33 * 256 * 2, 33 * 255 + 7),
             "wots": (22 * 51 * (1 + 7.5), 0)},
    "256f": {"tree": (17 * 16 * 67 * 16, 17 * 16 * 18 + 17 * 15),
             "fors": (35 * 512 * 2, 35 * 511 + 10),
             "wots": (17 * 67 * (1 + 7.5), 0)},
    # the small-signature sets (2^h' = 512 / 512 / 256 leaves, FORS height 12 / 14 / 14)
    "128s": {"tree": (7 * 512 * 35 * 16 + 7 * 512 * 10 + 7 * 511, 0),
             "fors": (14 * 4096 * 2 + 14 * 4095 + 4, 0),
             "wots": (7 * 35 * (1 + 7.5), 0)},
    "192s": {"tree": (7 * 512 * 51 * 16, 7 * 512 * 10 + 7 * 511),
             "fors": (17 * 16384 * 2, 17 * 16383 + 4),
             "wots": (7 * 51 * (1 + 7.5), 0)},
    "256s": {"tree": (8 * 256 * 67 * 16, 8 * 256 * 18 + 8 * 255),
             "fors": (22 * 16384 * 2, 22 * 16383 + 6),
             "wots": (8 * 67 * (1 + 7.5), 0)},
}


# The SHAKE instantiation: every hash is Keccak-f[1600] permutations.  ALU
# work of one permutation on 32-bit lane halves, per round: column parities
# 20 (2 LOP3 per half), D 20 (rotate-by-1 and XOR), theta's XOR into the
# 25 lanes 50, rho 48 funnel shifts (lanes rotated by 0 or 32 cost nothing),
# chi 50 LOP3, iota 2 -> 190 x 24 = 4560.
ALU_KECCAK = 4560


def _keccak_work(n, d, hp, a, k, length):
    """Permutations per signature of each stage (T_l absorbs n + 32 + l n
    bytes plus a pad byte at 136 bytes per permutation)."""
    t_len = -(-(n + 32 + length * n + 1) // 136)
    t_k = -(-(n + 32 + k * n + 1) // 136)
    return {"tree": d * (2 ** hp) * (length * 16 + t_len) + d * (2 ** hp - 1),
            "fors": k * (2 ** a) * 2 + k * (2 ** a - 1) + t_k,
            "wots": d * length * (1 + 7.5)}


KECCAK_WORK = {"shake-128f": _keccak_work(16, 22, 3, 6, 33, 35), "shake-192f": _keccak_work(24, 22, 3, 8, 33, 51),
               "shake-256f": _keccak_work(32, 17, 4, 9, 35, 67), "shake-128s": _keccak_work(16, 7, 9, 12, 14, 35),
               "shake-192s": _keccak_work(24, 7, 9, 14, 17, 51), "shake-256s": _keccak_work(32, 8, 8, 14, 22, 67)}


# The same ALU work as the kernels execute it.  The basis above prices
# every compression in full; the signing kernels skip part of it, bit for
# bit the same result:
#  * a WOTS+ chain step (and a FORS leaf PRF / F where k 2^a <= 2^16) takes
#    its state after rounds 0..4, round 5 up to its message word, and sigma0
#    of message words 1..4 from a context computed once per chain (per hash
#    type), and runs rounds 6..63;
#  * its message words 6 + n/4 .. 14 are zero and word 15 is a constant, so
#    their sigma0 / sigma1 terms fold away in the unrolled schedule.
# So one such step costs 58 x 10 + 4 x (46 sigma1 + 34 + n/4 sigma0) ALU
# ops (at n = 16 two sigma1 fewer: words 17 and 19 depend on the address
# alone and come from the context too), and a chain 2 contexts (6 x 10 +
# 4 x 4 each, + 8 at n = 16) plus 16 steps.  T_l, H and T_k run the rolled
# compression in full (1024 / 2624 per block).
SET_SHAPE = {  # n, d, h', a, k, len
    "128f": (16, 22, 3, 6, 33, 35), "192f": (24, 22, 3, 8, 33, 51), "256f": (32, 17, 4, 9, 35, 67),
    "128s": (16, 7, 9, 12, 14, 35), "192s": (24, 7, 9, 14, 17, 51), "256s": (32, 8, 8, 14, 22, 67)}


def _step_alu(nw, ctx=True):
    """ALU ops of one one-block F / PRF compression over nw payload words
    (at n = 16 the context also holds sigma1 of message words 17 and 19,
    which depend on the address alone when words 10..14 are zero)."""
    s1 = 48 - 2 - (2 if ctx and nw == 4 else 0)
    s0 = 48 - (9 - nw) - 1 - (4 if ctx else 0)
    return (58 if ctx else 64) * 10 + 4 * (s1 + s0)


def _ctx_alu(nw):
    """ALU ops of one chain context: rounds 0..5 (round 5 up to its message
    word), sigma0 of message words 1..4, and at n = 16 sigma1 of words 17
    and 19."""
    return 6 * 10 + 4 * 4 + (8 if nw == 4 else 0)


def exec_alu_per_sig(ps, stage):
    """ALU-pipe ops per signature of a stage as the kernels execute them
    (the roofline's work basis); the SHAKE sets execute the full basis."""
    if ps in KECCAK_WORK:
        return alu_ops_per_sig(ps, stage)
    n, d, hp, a, k, length = SET_SHAPE[ps]
    nw, big = n // 4, n > 16
    c_blk = ALU_C512 if big else ALU_C256
    if stage == "tree":
        chain = 2 * _ctx_alu(nw) + 16 * _step_alu(nw)
        tl_blocks = -(-(22 + length * n + (17 if big else 9)) // (128 if big else 64))
        leaves = d * (1 << hp)
        return leaves * (length * chain + tl_blocks * c_blk) + d * ((1 << hp) - 1) * c_blk
    if stage == "fors":
        ctx = (k << a) <= 65536
        tk_blocks = -(-(22 + k * n + (17 if big else 9)) // (128 if big else 64))
        return k * (1 << a) * 2 * _step_alu(nw, ctx) + (k * ((1 << a) - 1) + tk_blocks) * c_blk
    return alu_ops_per_sig(ps, stage)


def exec_split_per_sig(ps, stage):
    """(SHA-256 ALU ops, SHA-512 blocks) per signature of a stage as the
    kernels execute them: the SHA-256 part on the executed basis above, the
    SHA-512 blocks (T_l, H, T_k at n = 24 / 32) whole."""
    n, d, hp, a, k, length = SET_SHAPE[ps]
    big = n > 16
    total = exec_alu_per_sig(ps, stage)
    if not big:
        return total, 0
    c512 = STAGE_WORK[ps][stage][1]
    return total - c512 * ALU_C512, c512


def ops_per_sig(ps, stage):
    if ps in KECCAK_WORK:          # Keccak is all ALU work: the two bases coincide
        return KECCAK_WORK[ps][stage] * ALU_KECCAK
    c256, c512 = STAGE_WORK[ps][stage]
    return c256 * OPS_C256 + c512 * OPS_C512


def alu_ops_per_sig(ps, stage):
    if ps in KECCAK_WORK:
        return KECCAK_WORK[ps][stage] * ALU_KECCAK
    c256, c512 = STAGE_WORK[ps][stage]
    return c256 * ALU_C256 + c512 * ALU_C512


def int_peak_tops(sm_count, sm_mhz):
    """Integer issue peak: every SM issues one warp instruction per cycle on
    each of its 4 sub-partitions, 32 lanes wide -> SMs x 128 lane-ops/clk."""
    return sm_count * 4 * 32 * sm_mhz * 1e6 / 1e12


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
def oracle_rate(ps, sks, wl, seconds, idx_start=0):
    """Sign messages of the workload with the CPU oracle on every host core
    (ctypes releases the GIL) until 'seconds' have passed; return
    (sig/s, signatures done, cores)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle as O
    cores = len(os.sched_getaffinity(0))
    done = [0]
    stop = time.perf_counter() + seconds
    lock = threading.Lock()

    def worker(tid):
        i = idx_start + tid
        n = 0
        while time.perf_counter() < stop:
            m = i % wl.count
            O.sign(ps, sks[int(wl.key_idx[m])], wl.message(m))
            n += 1
            i += cores
        with lock:
            done[0] += n

    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(worker, range(cores)))
    dt = time.perf_counter() - t0
    return done[0] / dt, done[0], cores


def oracle_keys(ps, seeds):
    from oracle import oracle as O
    return [O.keygen(ps, bytes(s))[1] for s in seeds]


# ------------------------------------------------------------------ arms
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """CPU oracle arm: bounded oracle signing per step on the host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2512_23969_gb300 import inputs
    wl = inputs.config(1)
    sks = oracle_keys("128f", wl.seeds)
    # each step is a bounded sample; the whole run stays near a minute
    per_step = max(1.0, min(args.ref_step_seconds, 60.0 / max(1, args.steps)))
    for _ in range(args.warmup):
        oracle_rate("128f", sks, wl, 0.5)
    rates, total = [], 0
    for k in range(args.steps):
        r, n, cores = oracle_rate("128f", sks, wl, per_step, idx_start=k * 977)
        rates.append(r)
        total += n
    value = sum(rates) / len(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "signatures/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(per_step * 1e3, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "params": "128f", "global_batch": 16384, "msg_bytes": 32,
                   "keys": 16, "parallelism": "none (CPU oracle)"},
        "cpu_baseline": {"value": round(value, 3), "unit": "signatures/s", "cores": cores, "kind": "oracle",
                         "sample": "%d signatures of the workload (messages i mod 16384, keys i mod 16), "
                                   "%.0f s per step on all host cores" % (total, per_step)},
        "e2e": {"value": round(value, 3), "unit": "signatures/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def log(msg):
    """Progress line on stderr (the JSON line alone goes to stdout)."""
    print("[bench %.1fs] %s" % (time.perf_counter() - T_START, msg), file=sys.stderr, flush=True)


T_START = time.perf_counter()


def _time_steps(fn, stream, flush, steps, warmup):
    """CUDA-event time of fn() per step (L2 flushed between steps, outside)."""
    import torch
    for i in range(warmup):
        flush.fill_(i & 0xFF)
        fn()
    torch.cuda.synchronize()
    ms = []
    for k in range(steps):
        flush.fill_((k + 3) & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return ms


def sha_mix_time_ms(ps, stage, count, mix, sm_count, mhz):
    """Time a stage's executed SHA-2 work would take at the SHA-mix peak
    (ms): its SHA-256 ALU ops in compression equivalents (1024 each) at the
    probe's SHA-256 rate, its SHA-512 blocks at the probe's SHA-512 rate."""
    per_s = lambda rate: rate * sm_count * mhz * 1e6
    alu256, c512 = exec_split_per_sig(ps, stage)
    return 1e3 * count * (alu256 / ALU_C256 / per_s(mix["sha256_per_clk_sm"]) +
                          (c512 / per_s(mix["sha512_per_clk_sm"]) if c512 else 0.0))


def sha_mix_roofline(mix, sm_count, mhz, ps, count, ms, alu_rate):
    """TREE_Sign against the SHA-mix peak: the time its executed SHA-2 work
    takes at the rates the signer's own compression code reaches alone
    (hs_probe_sha_mix), over the launch's measured time."""
    out = {"probe": mix, "sm_mhz": mhz,
           "c256_peak_per_s": round(mix["sha256_per_clk_sm"] * sm_count * mhz * 1e6, 1),
           "c512_peak_per_s": round(mix["sha512_per_clk_sm"] * sm_count * mhz * 1e6, 1),
           "alu_efficiency_of_mix": {
               "sha256": round(mix["sha256_per_clk_sm"] * ALU_C256 / alu_rate, 4),
               "sha512": round(mix["sha512_per_clk_sm"] * ALU_C512 / alu_rate, 4),
               "sha256_plain": round(mix.get("sha256_plain_per_clk_sm", 0.0) * ALU_C256 / alu_rate, 4)},
           "basis": "hs_probe_sha_mix: the signer's SHA-256 round code (64 rounds unrolled, additions on "
                    "IMAD) and SHA-512 compression (16 rounds x 5) back to back per thread, one "
                    "full-occupancy wave, SM cycle counters; the kernel's executed work priced at those "
                    "rates (chain steps as 908-932 / 1024 of a compression)"}
    if ps in SET_SHAPE and ms > 0:
        out["tree_frac"] = round(sha_mix_time_ms(ps, "tree", count, mix, sm_count, mhz) / ms, 4)
    return out


def measure_other_configs(hs, inputs, args, stream, flush, alu_peak, mix=None, sm_count=0, mhz=0.0):
    import torch
    res = {}
    dev = lambda x: torch.from_numpy(x).cuda()
    steps, warmup = max(2, args.steps // 2), 3
    # the SHAKE sets on fewer messages (a permutation costs ~4.5 SHA-256 compressions)
    shake_counts = {"shake-128f": 4096, "shake-192f": 2048, "shake-256f": 2048, "shake-128s": 256,
                    "shake-192s": 256, "shake-256s": 256,
                    # the robust SHA2 instantiation: every F, H and T_l also computes its mask
                    "robust-128f": 8192, "robust-192f": 4096, "robust-256f": 4096}
    for ps in ("192f", "256f", "128s", "192s", "256s") + tuple(shake_counts):
        log("config %s" % ps)
        if ps in ("192f", "256f"):
            wl = inputs.config(2, ps)
        else:       # the same shape of workload for the other sets
            cnt = shake_counts.get(ps, 1024)
            wl = inputs.make(ps, cnt, 16, ("uniform", 32, 1024), inputs.BASE_SEED + 3,
                             "%s-16keys-%dxU[32,1024]B" % (ps, cnt))
        pk, sk = hs.hs_keygen(ps, dev(wl.seeds))
        m, l, k = dev(wl.msgs), dev(wl.lens), dev(wl.key_idx)
        sig = torch.empty(wl.count * hs.sig_bytes(ps), dtype=torch.uint8, device="cuda")
        hs.hs_profile_enable(True)
        ms = _time_steps(lambda: hs.hs_sign_batch(ps, sk, m, l, key_idx=k, sigs=sig, num_keys=wl.num_keys,
                                                   stream=stream), stream, flush, steps, warmup)
        prof = hs.hs_profile_read()
        hs.hs_profile_enable(False)
        ok = hs.hs_verify_batch(ps, pk, m, l, sig.view(wl.count, -1), key_idx=k, num_keys=wl.num_keys)
        res[ps] = {"workload": wl.name, "value": round(wl.count * len(ms) / (sum(ms) / 1e3), 1),
                   "unit": "signatures/s", "ms_per_step": round(sum(ms) / len(ms), 3),
                   "stage_ms": {a: round(b, 3) for a, b in prof.items()},
                   "alu_frac": ({st: round(exec_alu_per_sig(ps, st) * wl.count / (prof[st] / 1e3) / 1e12 / alu_peak, 4)
                                 for st in ("tree", "fors") if prof.get(st, 0) > 0}
                                if not ps.startswith("robust-") else None),
                   "alu_frac_full_compression": ({
                       st: round(alu_ops_per_sig(ps, st) * wl.count / (prof[st] / 1e3) / 1e12 / alu_peak, 4)
                       for st in ("tree", "fors") if prof.get(st, 0) > 0} if not ps.startswith("robust-") else None),
                   "verified": int(ok.sum().item()) == wl.count}
        if mix and ps in SET_SHAPE:
            res[ps]["sha_mix_frac"] = {
                st: round(sha_mix_time_ms(ps, st, wl.count, mix, sm_count, mhz) / prof[st], 4)
                for st in ("tree", "fors") if prof.get(st, 0) > 0}
    # the bench workload again with tree sharing on (same signatures, less work)
    log("128f with tree sharing")
    wl = inputs.config(1)
    pk, sk = hs.hs_keygen("128f", dev(wl.seeds))
    m, l, k = dev(wl.msgs), dev(wl.lens), dev(wl.key_idx)
    sig = torch.empty(wl.count * hs.sig_bytes("128f"), dtype=torch.uint8, device="cuda")
    ref = hs.hs_sign_batch("128f", sk, m, l, key_idx=k, num_keys=wl.num_keys).view(-1).clone()
    hs.hs_set_tree_sharing(True)
    try:
        hs.hs_profile_enable(True)
        ms = _time_steps(lambda: hs.hs_sign_batch("128f", sk, m, l, key_idx=k, sigs=sig, num_keys=wl.num_keys,
                                                   stream=stream), stream, flush, steps, warmup)
        prof = hs.hs_profile_read()
        hs.hs_profile_enable(False)
    finally:
        hs.hs_set_tree_sharing(False)
    res["128f_tree_sharing"] = {"workload": wl.name + ", repeated upper-layer trees built once per batch",
                                "value": round(wl.count * len(ms) / (sum(ms) / 1e3), 1), "unit": "signatures/s",
                                "ms_per_step": round(sum(ms) / len(ms), 3),
                                "stage_ms": {a: round(b, 3) for a, b in prof.items()},
                                "identical_to_full_work": bool(torch.equal(sig, ref))}
    # batched GPU verification of the bench workload's signatures
    log("128f verify")
    ms = _time_steps(lambda: hs.hs_verify_batch("128f", pk, m, l, sig.view(wl.count, -1), key_idx=k,
                                                num_keys=wl.num_keys, stream=stream), stream, flush, steps, warmup)
    ok = hs.hs_verify_batch("128f", pk, m, l, sig.view(wl.count, -1), key_idx=k, num_keys=wl.num_keys)
    res["128f_verify"] = {"workload": wl.name + ", hs_verify_batch of the batch's signatures",
                          "value": round(wl.count * len(ms) / (sum(ms) / 1e3), 1), "unit": "verifications/s",
                          "ms_per_step": round(sum(ms) / len(ms), 3), "accepted": int(ok.sum().item())}
    # the bench workload signed from a keyset with the top 4 layers of each key prebuilt
    log("128f from a keyset with cached top layers")
    sig.zero_()
    t0 = time.perf_counter()
    ks = hs.KeySet("128f", sk, cache_layers=4, stream=stream)
    build_s = time.perf_counter() - t0
    try:
        hs.hs_profile_enable(True)
        ms = _time_steps(lambda: ks.sign(m, l, key_idx=k, sigs=sig, stream=stream), stream, flush, steps, warmup)
        prof = hs.hs_profile_read()
        hs.hs_profile_enable(False)
        res["128f_keyset_cache4"] = {
            "workload": wl.name + ", keys resident with layers 18-21 of every key prebuilt (585 trees per key)",
            "value": round(wl.count * len(ms) / (sum(ms) / 1e3), 1), "unit": "signatures/s",
            "ms_per_step": round(sum(ms) / len(ms), 3), "stage_ms": {a: round(b, 3) for a, b in prof.items()},
            "cache_build_s": round(build_s, 3), "keyset_bytes": ks.nbytes,
            "identical_to_full_work": bool(torch.equal(sig, ref))}
    finally:
        ks.close()
    # mixed-parameter batch (32768 messages 50/30/20, log-uniform 16 B - 64 KB, 64 keys)
    wls = inputs.mixed()
    jobs = []
    for wl in wls:
        pk, sk = hs.hs_keygen(wl.params, dev(wl.seeds))
        jobs.append({"params": wl.params, "sk": sk, "pk": pk, "msgs": dev(wl.msgs), "lens": dev(wl.lens),
                     "key_idx": dev(wl.key_idx), "num_keys": wl.num_keys,
                     "sigs": torch.empty(wl.count * hs.sig_bytes(wl.params), dtype=torch.uint8, device="cuda")})
    total = sum(wl.count for wl in wls)

    def plain():
        for j in jobs:
            hs.hs_sign_batch(j["params"], j["sk"], j["msgs"], j["lens"], key_idx=j["key_idx"], sigs=j["sigs"],
                             num_keys=j["num_keys"], stream=stream)

    out = {"workload": "mixed 32768 msgs 50/30/20 128f/192f/256f, log-U[16 B, 64 KB], 64 keys (32/19/13)",
           "messages": total, "msg_bytes": int(sum(int(wl.lens.sum()) for wl in wls))}
    for name, fn in (("plain_per_set_calls", plain),
                     ("one_graph_launch", lambda: hs.hs_sign_mixed(jobs, use_graph=True, stream=stream)),
                     ("streams_no_graph", lambda: hs.hs_sign_mixed(jobs, use_graph=False, stream=stream))):
        ms = _time_steps(fn, stream, flush, steps, warmup)
        out[name] = {"value": round(total * len(ms) / (sum(ms) / 1e3), 1), "unit": "signatures/s",
                     "ms_per_step": round(sum(ms) / len(ms), 3), "max_ms": round(max(ms), 3)}
    n_ok = 0
    for j, wl in zip(jobs, wls):
        ok = hs.hs_verify_batch(wl.params, j["pk"], j["msgs"], j["lens"], j["sigs"].view(wl.count, -1),
                                key_idx=j["key_idx"], num_keys=wl.num_keys)
        n_ok += int(ok.sum().item())
    out["verified"] = "%d/%d" % (n_ok, total)
    res["mixed"] = out
    # a small mixed batch, where per-launch overheads weigh most
    swls = inputs.mixed(count=96, seed=inputs.BASE_SEED + 61, name="mixed-small")
    sjobs = []
    for wl in swls:
        pk, sk = hs.hs_keygen(wl.params, dev(wl.seeds))
        sjobs.append({"params": wl.params, "sk": sk, "msgs": dev(wl.msgs), "lens": dev(wl.lens),
                      "key_idx": dev(wl.key_idx), "num_keys": wl.num_keys, "max_len": int(wl.lens.max()),
                      "sigs": torch.empty(wl.count * hs.sig_bytes(wl.params), dtype=torch.uint8, device="cuda")})
    stotal = sum(wl.count for wl in swls)

    def splain():
        for j in sjobs:
            hs.hs_sign_batch(j["params"], j["sk"], j["msgs"], j["lens"], key_idx=j["key_idx"], sigs=j["sigs"],
                             num_keys=j["num_keys"], stream=stream)

    sout = {"workload": "mixed 96 msgs 50/30/20 128f/192f/256f, log-U[16 B, 64 KB], 64 keys (32/19/13)",
            "messages": stotal}
    for name, fn in (("plain_per_set_calls", splain),
                     ("one_graph_launch", lambda: hs.hs_sign_mixed(sjobs, use_graph=True, stream=stream)),
                     ("streams_no_graph", lambda: hs.hs_sign_mixed(sjobs, use_graph=False, stream=stream))):
        ms = sorted(_time_steps(fn, stream, flush, 20, warmup))     # short steps: 20, median reported too
        sout[name] = {"value": round(stotal * len(ms) / (sum(ms) / 1e3), 1), "unit": "signatures/s",
                      "ms_per_step": round(sum(ms) / len(ms), 3), "median_ms": round(ms[len(ms) // 2], 3),
                      "min_ms": round(ms[0], 3)}
    try:
        sout["stage_ms_per_set"] = stage_breakdown(hs, sjobs, stream, flush)
    except Exception as exc:
        sout["stage_ms_per_set"] = {"error": repr(exc)[:200]}
    res["mixed_small"] = sout
    # a batch of the serving run's mean size (~78 requests of one set, log-U[16 B, 4 KB])
    bjobs = []
    for i, ps in enumerate(("128f", "192f", "256f")):
        wl = inputs.make(ps, 78, 16, ("loguniform", 16, 4096), inputs.BASE_SEED + 70 + i, "%s-78-serving" % ps)
        _, sk = hs.hs_keygen(ps, dev(wl.seeds))
        bjobs.append({"params": ps, "sk": sk, "msgs": dev(wl.msgs), "lens": dev(wl.lens),
                      "key_idx": dev(wl.key_idx), "num_keys": wl.num_keys, "max_len": int(wl.lens.max()),
                      "sigs": torch.empty(wl.count * hs.sig_bytes(ps), dtype=torch.uint8, device="cuda")})
    try:
        bd = stage_breakdown(hs, bjobs, stream, flush)
    except Exception as exc:
        bd = {"error": repr(exc)[:200]}
    res["serving_batch"] = {"workload": "78 requests of one set, log-U[16 B, 4 KB], 16 keys (the serving run's "
                                        "mean batch)", "stage_ms_per_set": bd}
    return res


def stage_breakdown(hs, jobs, stream, flush, reps=5):
    """Per-stage CUDA-event times (median of reps) of each job signed alone."""
    out = {}
    for j in jobs:
        runs = []
        for r in range(reps + 1):
            flush.fill_(r & 0xFF)
            hs.hs_profile_enable(True)
            hs.hs_sign_batch(j["params"], j["sk"], j["msgs"], j["lens"], key_idx=j["key_idx"], sigs=j["sigs"],
                             num_keys=j["num_keys"], stream=stream)
            prof = hs.hs_profile_read()
            hs.hs_profile_enable(False)
            if r:                          # the first is a warm-up
                runs.append(prof)
        med = {k: round(sorted(p[k] for p in runs)[len(runs) // 2], 3) for k in runs[0]}
        med["total"] = round(sum(v for k, v in med.items()), 3)
        med["messages"] = int(j["lens"].numel())
        med["max_msg_bytes"] = int(j["max_len"])
        out[j["params"]] = med
    return out


def _replay_point(srv, inputs, np, rate, seconds, seed):
    """Poisson arrivals at 'rate' for 'seconds'; achieved rate and latency."""
    tr = inputs.serving_trace(rate=rate, seconds=seconds, seed=seed)
    n = len(tr["params"])
    st0 = srv.stats()
    lat, _ = srv.replay(tr["params"], tr["keys"], tr["pool_idx"], tr["pool_msgs"], tr["pool_lens"],
                        tr["arrival_ns"], timeout_ms=int(seconds * 1000) + 120000)
    st1 = srv.stats()
    finish = (tr["arrival_ns"].astype(np.float64) + lat.astype(np.float64)).max() / 1e9
    nb = st1["batches"] - st0["batches"]
    return {"offered": round(rate, 1), "seconds": seconds, "requests": n, "value": round(n / finish, 1),
            "unit": "signatures/s", "p50_ms": round(float(np.percentile(lat, 50)) / 1e6, 3),
            "p99_ms": round(float(np.percentile(lat, 99)) / 1e6, 3), "max_ms": round(float(lat.max()) / 1e6, 3),
            "batches": nb, "mean_batch": round((st1["batched_requests"] - st0["batched_requests"]) / max(1, nb), 1)}


def measure_serving(hs, inputs, seconds, rhos, search_steps, p99_bound_ms, burst=60000):
    """Serving run: 1024 resident keys (614/256/154), mix 60/25/15 of
    128f/192f/256f, log-uniform 16 B - 4 KB messages, an 8 GiB device-memory
    admission budget.  A saturating burst (all requests at t = 0) measures
    the peak rate of this mix; then Poisson arrivals at rho x peak for
    'seconds' each, reporting achieved rate and p50/p99 latency from arrival
    to host-observed completion; then the sustained capacity: the highest
    offered rate whose p99 stays within p99_bound_ms over 'seconds', found by
    bisection ('search_steps' runs) between the highest rho that held and
    1.05 x the burst peak."""
    import numpy as np
    import torch
    budget, max_batch, inflight = 8 << 30, 2048, 4
    base = inputs.serving_trace(rate=1.0, seconds=1.0)          # keys and pool only
    keys = {}
    for ps in ("128f", "192f", "256f"):
        keys[ps] = hs.hs_keygen(ps, torch.from_numpy(base["seeds"][ps]).cuda())[1]
    out = {"workload": "serving: 1024 keys (614/256/154), mix 60/25/15 128f/192f/256f, log-U[16 B, 4 KB]",
           "mem_budget_bytes": budget, "max_batch": max_batch, "max_inflight": inflight,
           "p99_bound_ms": p99_bound_ms}
    with hs.Server(keys, max_inflight=inflight, max_batch=max_batch, mem_budget=budget) as srv:
        tr = inputs.serving_trace(rate=1e6, seconds=burst / 1e6, seed=inputs.BASE_SEED + 40)
        tr["arrival_ns"][:] = 0
        n = len(tr["params"])
        log("serving: burst of %d requests" % n)
        t0 = time.perf_counter()
        try:
            lat, _ = srv.replay(tr["params"], tr["keys"], tr["pool_idx"], tr["pool_msgs"], tr["pool_lens"],
                                tr["arrival_ns"], timeout_ms=120000)
        except hs.HSError:
            log("serving: burst timed out; server stats %s" % srv.stats())
            raise
        wall = time.perf_counter() - t0
        peak = n / wall
        out["burst"] = {"requests": n, "value": round(peak, 1), "unit": "signatures/s",
                        "p50_ms": round(float(np.percentile(lat, 50)) / 1e6, 3),
                        "p99_ms": round(float(np.percentile(lat, 99)) / 1e6, 3)}
        held = 0.0
        for rho in rhos:
            log("serving: rho %.2f for %.0f s" % (rho, seconds))
            pt = _replay_point(srv, inputs, np, rho * peak, seconds, inputs.BASE_SEED + 41 + int(rho * 100))
            out["rho_%.2f" % rho] = pt
            if pt["p99_ms"] <= p99_bound_ms:
                held = max(held, rho)
        # sustained capacity: bisection on rho for p99 <= bound
        lo, hi, best = held, 1.05, None
        if held > 0:
            best = dict(out["rho_%.2f" % held], rho=held)
        search = []
        for k in range(search_steps):
            mid = round((lo + hi) / 2, 4)
            log("serving: capacity search rho %.4f for %.0f s" % (mid, seconds))
            pt = _replay_point(srv, inputs, np, mid * peak, seconds, inputs.BASE_SEED + 300 + k)
            pt["rho"] = mid
            search.append(pt)
            if pt["p99_ms"] <= p99_bound_ms:
                lo, best = mid, pt
            else:
                hi = mid
        out["capacity_search"] = search
        out["sustained"] = best
        st = srv.stats()
        out["batches"] = st["batches"]
        out["mean_batch"] = round(st["batched_requests"] / max(1, st["batches"]), 1)
        out["max_inflight_batches"] = st["max_inflight_batches"]
        out["max_device_bytes_in_use"] = st["max_device_bytes_in_use"]
    # the same keys as keysets with their top 2 layers prebuilt: the same
    # saturating burst, and the load of the uncached sustained capacity
    with hs.Server(keys, max_inflight=inflight, max_batch=max_batch, mem_budget=budget, cache_layers=2) as srv:
        cached = {"cache_layers": 2}
        tr = inputs.serving_trace(rate=1e6, seconds=burst / 1e6, seed=inputs.BASE_SEED + 40)
        tr["arrival_ns"][:] = 0
        n = len(tr["params"])
        log("serving with cached top layers: burst of %d" % n)
        t0 = time.perf_counter()
        lat, _ = srv.replay(tr["params"], tr["keys"], tr["pool_idx"], tr["pool_msgs"], tr["pool_lens"],
                            tr["arrival_ns"], timeout_ms=120000)
        cached["burst"] = {"requests": n, "value": round(n / (time.perf_counter() - t0), 1),
                           "unit": "signatures/s", "p50_ms": round(float(np.percentile(lat, 50)) / 1e6, 3),
                           "p99_ms": round(float(np.percentile(lat, 99)) / 1e6, 3)}
        if best is not None:
            log("serving with cached top layers: at the uncached sustained rate for %.0f s" % seconds)
            cached["at_uncached_sustained"] = _replay_point(srv, inputs, np, best["offered"], seconds,
                                                            inputs.BASE_SEED + 141)
        out["cached_top_layers"] = cached
    return out


def summarize(line):
    """The figures a reader looks for first, as a short object at the end of
    the JSON line."""
    r = line.get("roofline") or {}
    sm = {"sig_per_s": line.get("value"), "e2e_sig_per_s": (line.get("e2e") or {}).get("value"),
          "alu_frac_executed": r.get("frac"), "alu_frac_full_compression": r.get("frac_full_compression"),
          "issue_frac": r.get("issue_frac"), "sha_mix_frac": (r.get("sha_mix") or {}).get("tree_frac")}
    p = line.get("plain_per_stage") or {}
    sm["plain_per_stage_sig_per_s"] = p.get("value")
    sv = line.get("serving") or {}
    for key in ("rho_0.50", "rho_0.75"):
        if isinstance(sv.get(key), dict):
            sm["serving_" + key] = {k: sv[key].get(k) for k in ("seconds", "value", "p50_ms", "p99_ms")}
    if isinstance(sv.get("sustained"), dict):
        b = sv["sustained"]
        sm["serving_sustained"] = {"rho": b.get("rho"), "offered": b.get("offered"), "value": b.get("value"),
                                   "p50_ms": b.get("p50_ms"), "p99_ms": b.get("p99_ms"),
                                   "p99_bound_ms": sv.get("p99_bound_ms"), "seconds": b.get("seconds")}
    if isinstance(sv.get("burst"), dict):
        sm["serving_burst_sig_per_s"] = sv["burst"].get("value")
    oc = line.get("other_configs") or {}
    for key in ("mixed_small", "mixed"):
        if isinstance(oc.get(key), dict):
            sm[key + "_ms"] = {k: v.get("ms_per_step") for k, v in oc[key].items() if isinstance(v, dict)
                               and "ms_per_step" in v}
    for ps in ("192f", "256f"):
        if isinstance(oc.get(ps), dict):
            sm[ps + "_sig_per_s"] = oc[ps].get("value")
            if oc[ps].get("sha_mix_frac"):
                sm[ps + "_sha_mix_frac"] = oc[ps]["sha_mix_frac"]
    return sm


def run_probe_only():
    """The roofline's peak probes alone (hs_probe_int_pipes, hs_probe_sha_mix):
    one JSON line of per-clock-per-SM rates."""
    from paper_2512_23969_gb300 import build as hs_build
    hs_build.build()
    from paper_2512_23969_gb300 import hs
    hs.load()
    print(json.dumps({"int_pipes_lane_ops_per_clk_sm": hs.hs_probe_int_pipes(), "sha_mix": hs.hs_probe_sha_mix()}))
    return 0


def run_verify_only(args):
    """Verification of the bench batch: 1 signing call, then 3 timed
    hs_verify_batch calls (CUDA events); prints one JSON line."""
    import torch
    from paper_2512_23969_gb300 import build as hs_build
    hs_build.build()
    from paper_2512_23969_gb300 import hs, inputs
    hs.load()
    ps = args.params
    wl = inputs.config(1) if ps == "128f" and args.count == 16384 else \
        inputs.make(ps, args.count, 16, 32, inputs.BASE_SEED + 1, "%s-16keys-%dx32B" % (ps, args.count))
    pk, sk = hs.hs_keygen(ps, torch.from_numpy(wl.seeds).cuda())
    m, l, k = (torch.from_numpy(x).cuda() for x in (wl.msgs, wl.lens, wl.key_idx))
    sig = hs.hs_sign_batch(ps, sk, m, l, key_idx=k, num_keys=wl.num_keys)
    ms = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ok = hs.hs_verify_batch(ps, pk, m, l, sig, key_idx=k, num_keys=wl.num_keys)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(json.dumps({"metric": "verifications/s", "value": round(wl.count / (min(ms) / 1e3), 1),
                      "ms": [round(x, 3) for x in ms], "accepted": int(ok.sum().item()), "count": wl.count,
                      "params": ps}))
    return 0


def run_own(args):
    import numpy as np
    import torch
    from paper_2512_23969_gb300 import replicas
    ws, rank, local = replicas.init_from_env()
    torch.cuda.set_device(local)
    from paper_2512_23969_gb300 import build as hs_build
    hs_build.build()
    from paper_2512_23969_gb300 import autotune, hs, inputs
    hs.load()
    tuned = autotune.apply()
    props = torch.cuda.get_device_properties(local)
    sm_count = props.multi_processor_count

    ps = args.params
    if ps == "128f" and args.count == 16384:
        wl = inputs.config(1)
    else:
        wl = inputs.make(ps, args.count, 16, 32, inputs.BASE_SEED + 1, "%s-16keys-%dx32B" % (ps, args.count))
    count = wl.count
    S = hs.sig_bytes(ps)
    stream = torch.cuda.current_stream()
    seeds = torch.from_numpy(wl.seeds).cuda()
    pk, sk = hs.hs_keygen(ps, seeds)
    msgs = torch.from_numpy(wl.msgs).cuda()
    lens = torch.from_numpy(wl.lens).cuda()
    kidx = torch.from_numpy(wl.key_idx).cuda()
    sigs = torch.empty(count * S, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        hs.hs_sign_batch(ps, sk, msgs, lens, key_idx=kidx, sigs=sigs, num_keys=wl.num_keys, stream=stream)

    log("main workload: %d x %s" % (count, ps))
    hs.hs_profile_enable(True)
    for i in range(args.warmup):
        flush.fill_(i & 0xFF)
        step()
    torch.cuda.synchronize()
    replicas.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, stage_ms = [], {}
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_((k + 7) & 0xFF)          # L2 flush, outside the timed events
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
        evs[k][1].synchronize()
        for name, v in hs.hs_profile_read().items():
            stage_ms.setdefault(name, []).append(v)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    for a, b in evs:
        step_ms.append(a.elapsed_time(b))
    hs.hs_profile_enable(False)
    torch.cuda.synchronize()
    replicas.barrier()
    total_ms = replicas.max_over_ranks(sum(step_ms))
    value = replicas.job_rate(ws, count, args.steps, total_ms)

    # correctness guard on the timed output: GPU verify of every signature
    ok = hs.hs_verify_batch(ps, pk, msgs, lens, sigs.view(count, S), key_idx=kidx, num_keys=wl.num_keys)
    n_ok = int(ok.sum().item())

    # end to end through the C ABI with pinned host buffers (copies inside the call)
    e2e = None
    if args.e2e_steps > 0 and rank == 0:
        sk_h = sk.cpu().pin_memory()
        msgs_h = torch.from_numpy(wl.msgs).pin_memory()
        lens_h = torch.from_numpy(wl.lens).pin_memory()
        kidx_h = torch.from_numpy(wl.key_idx).pin_memory()
        sigs_h = torch.empty(count * S, dtype=torch.uint8).pin_memory()
        hs.hs_sign_batch(ps, sk_h, msgs_h, lens_h, key_idx=kidx_h, sigs=sigs_h, num_keys=wl.num_keys)
        e2e_t = []
        for k in range(args.e2e_steps):
            flush.fill_(k & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hs.hs_sign_batch(ps, sk_h, msgs_h, lens_h, key_idx=kidx_h, sigs=sigs_h, num_keys=wl.num_keys)
            e2e_t.append(time.perf_counter() - t0)
        h2d = sk_h.numel() + msgs_h.numel() + lens_h.numel() * 8 + kidx_h.numel() * 4
        # the same calls with the signatures staged in device memory and copied back
        hs.hs_set_host_direct(False)
        staged_t = []
        try:
            for k in range(args.e2e_steps):
                flush.fill_(k & 0xFF)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                hs.hs_sign_batch(ps, sk_h, msgs_h, lens_h, key_idx=kidx_h, sigs=sigs_h, num_keys=wl.num_keys)
                staged_t.append(time.perf_counter() - t0)
        finally:
            hs.hs_set_host_direct(True)
        srt = sorted(e2e_t)
        e2e = {"value": round(count / (sum(e2e_t) / len(e2e_t)), 1), "unit": "signatures/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(sigs_h.numel()),
               "steps": len(e2e_t), "ms_median": round(srt[len(srt) // 2] * 1e3, 3),
               "ms_max": round(srt[-1] * 1e3, 3),
               "path": "hs_sign_batch with pinned host buffers: inputs staged H2D, signatures written by the "
                       "kernels straight into the mapped host buffer (NVLink-C2C), stream sync",
               "staged_d2h_value": round(count / (sum(staged_t) / len(staged_t)), 1) if staged_t else None}
        if not torch.equal(sigs_h, sigs.cpu()):
            e2e["mismatch"] = True

    # roofline of the dominant kernel (TREE_Sign), from its CUDA-event durations.
    # Bound: the ALU pipe.  Peak = measured ALU-pipe lane-ops/clk/SM (LOP3 and
    # SHF probes) x SMs x max SM clock; work = ALU-only ops of the algorithm.
    pipes = hs.hs_probe_int_pipes()
    alu_rate = min(pipes["lop3"], pipes["shf"])
    tree_ms = sum(stage_ms.get("tree", [0])) / max(1, len(stage_ms.get("tree", [1])))
    stage_avg = {k: round(sum(v) / len(v), 3) for k, v in stage_ms.items()}
    sm_mhz_peak = 2070.0
    alu_peak = sm_count * alu_rate * sm_mhz_peak * 1e6 / 1e12
    alu_work = exec_alu_per_sig(ps, "tree") * count
    alu_work_full = alu_ops_per_sig(ps, "tree") * count
    achieved = alu_work / (tree_ms / 1e3) / 1e12 if tree_ms > 0 else None
    achieved_full = alu_work_full / (tree_ms / 1e3) / 1e12 if tree_ms > 0 else None
    issue_peak = int_peak_tops(sm_count, sm_mhz_peak)
    issue_achieved = ops_per_sig(ps, "tree") * count / (tree_ms / 1e3) / 1e12 if tree_ms > 0 else None
    traffic = None
    prof_file = os.path.join(ROOT, "profiles", "tree_%s_traffic.json" % ps)
    if os.path.exists(prof_file):
        try:
            traffic = json.load(open(prof_file)).get("bytes_per_launch_scaled")
        except (OSError, ValueError):
            traffic = None
    tree_c = STAGE_WORK[ps]["tree"] if ps in STAGE_WORK else None
    roofline = {"bound": "alu", "kernel": "tree_kernel<%s> (TREE_Sign)" % ps,
                "compressions_per_s": ({"sha256": round(tree_c[0] * count / (tree_ms / 1e3), 1),
                                        "sha512": round(tree_c[1] * count / (tree_ms / 1e3), 1)}
                                       if tree_c and tree_ms > 0 else None),
                "achieved": round(achieved, 3) if achieved else None, "peak": round(alu_peak, 3),
                "unit": "Tops/s", "frac": round(achieved / alu_peak, 4) if achieved else None, "traffic": traffic,
                "frac_full_compression": round(achieved_full / alu_peak, 4) if achieved_full else None,
                "issue_frac": round(issue_achieved / issue_peak, 4) if issue_achieved else None,
                "peak_basis": "ALU pipe %.1f lane-ops/clk/SM (measured LOP3/SHF rate) x %d SMs x %.0f MHz"
                              % (alu_rate, sm_count, sm_mhz_peak),
                "work_basis": "ALU-pipe ops as executed: chain steps run rounds 6..63 with sigma terms of "
                              "constant words folded (%d per 128f step), T_len / H in full (%d per SHA-256 "
                              "block, %d per SHA-512); %.4g per launch; frac_full_compression prices every "
                              "compression in full (%.4g per launch)"
                              % (_step_alu(4), ALU_C256, ALU_C512, alu_work, alu_work_full),
                "issue": {"achieved": round(issue_achieved, 3) if issue_achieved else None,
                          "peak": round(issue_peak, 3),
                          "frac": round(issue_achieved / issue_peak, 4) if issue_achieved else None,
                          "basis": "%d int ops per SHA-256 compression vs %d SMs x 128 lanes/clk x %.0f MHz"
                                   % (OPS_C256, sm_count, sm_mhz_peak)},
                "measured_pipes_lane_ops_per_clk_per_sm": pipes}
    if clk.get("sm_mhz") and achieved:
        roofline["frac_at_sampled_clock"] = round(achieved / (sm_count * alu_rate * clk["sm_mhz"] * 1e6 / 1e12), 4)
    # the SHA-mix peak: compressions/s the signer's own SHA-2 code reaches on
    # its own (hs_probe_sha_mix), at the SM clock sampled during the run
    mix = hs.hs_probe_sha_mix()
    mix_mhz = clk.get("sm_mhz") or sm_mhz_peak
    roofline["sha_mix"] = sha_mix_roofline(mix, sm_count, mix_mhz, ps, count, tree_ms, alu_rate)

    # the same workload through the plain per-stage kernels: no chain
    # checkpoints, so WOTS+_Sign recomputes every chain from its secret
    plain = None
    if rank == 0 and args.plain_steps > 0:
        hs.hs_set_chain_checkpoint(0)
        try:
            hs.hs_profile_enable(True)
            pms = _time_steps(step, stream, flush, args.plain_steps, 3)
            pprof = hs.hs_profile_read()
            hs.hs_profile_enable(False)
        finally:
            hs.hs_set_chain_checkpoint(2)
        plain = {"value": round(count * len(pms) / (sum(pms) / 1e3), 1), "unit": "signatures/s",
                 "ms_per_step": round(sum(pms) / len(pms), 3), "checkpoint_stride": 0,
                 "stage_ms": {a: round(b, 3) for a, b in pprof.items()},
                 "what": "the line's workload with WOTS+_Sign recomputing its chains (no TREE_Sign checkpoints)"}

    # the other workloads of the signer's specification, measured with the
    # same events: 192f / 256f batches, and the mixed-parameter batch in one
    # graph launch against one hs_sign_batch call per set
    others = {}
    if args.other_configs and rank == 0:
        try:
            others = measure_other_configs(hs, inputs, args, stream, flush, alu_peak, mix, sm_count, mix_mhz)
        except Exception as exc:      # keep the main line; report what failed
            others = {"error": repr(exc)[:300]}

    serving = None
    if args.serving_seconds > 0 and rank == 0:
        try:
            serving = measure_serving(hs, inputs, args.serving_seconds, (0.5, 0.75), args.serving_search,
                                      args.p99_bound_ms)
        except Exception as exc:
            serving = {"error": repr(exc)[:300]}

    # CPU oracle baseline on a bounded sample
    cpu = None
    if rank == 0 and args.cpu_seconds > 0:
        sks = oracle_keys(ps, wl.seeds)
        r, n, cores = oracle_rate(ps, sks, wl, args.cpu_seconds)
        # and on one host thread, over the first 16 messages
        from oracle import oracle as O
        t0 = time.perf_counter()
        for i in range(16):
            O.sign(ps, sks[int(wl.key_idx[i])], wl.message(i))
        one = 16 / (time.perf_counter() - t0)
        cpu = {"value": round(r, 3), "unit": "signatures/s", "cores": cores, "kind": "oracle",
               "sample": "%d signatures of this workload (messages i mod 16384) in %.0f s on %d host threads"
                         % (n, args.cpu_seconds, cores),
               "single_thread": {"value": round(one, 3), "sample": "messages 0..15 on one host thread"}}

    ms_sorted = sorted(step_ms)
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "signatures/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD if (ps == "128f" and count == 16384) else wl.name, "params": ps,
                   "global_batch": count * ws, "msg_bytes": 32,
                   "keys": 16, "parallelism": "replicas" if ws > 1 else "single GPU",
                   "l2": "flushed between timed steps (256 MB write, outside the events); outputs 280 MB > L2"},
        "e2e": e2e,
        "gpu_launches": hs.hs_sign_kernel_count() * args.steps,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clk,
        "stage_ms": stage_avg,
        "batch_latency_ms": {"p50": round(ms_sorted[len(ms_sorted) // 2], 3), "max": round(ms_sorted[-1], 3)},
        "verified": "%d/%d signatures accepted by GPU verify" % (n_ok, count),
        "other_configs": others,
        "serving": serving,
        "wall_s": round(wall, 3),
        "device": props.name, "sm_count": sm_count,
        "tuning": {k: autotune.get(ps, k) for k in autotune.KNOBS} | {"from_cache": bool(tuned)},
        "plain_per_stage": plain,
    }
    line["summary"] = summarize(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    replicas.barrier()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    import faulthandler
    faulthandler.enable()
    faulthandler.dump_traceback_later(1200, repeat=True)    # stacks on stderr if a stage stalls
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["own", "reference"], default="own")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--plain-steps", type=int, default=10,
                    help="steps of the same workload with WOTS+_Sign recomputing its chains (0 = skip)")
    ap.add_argument("--ref-step-seconds", type=float, default=10.0)
    ap.add_argument("--params", default="128f",
                    choices=["128f", "192f", "256f", "128s", "192s", "256s", "shake-128f", "shake-192f", "shake-256f",
                             "shake-128s", "shake-192s", "shake-256s"],
                    help="parameter set (the default workload is 128f; the others serve small profiling cases)")
    ap.add_argument("--no-other-configs", dest="other_configs", action="store_false",
                    help="skip the 192f / 256f / mixed-parameter measurements")
    ap.add_argument("--serving-seconds", type=float, default=60.0,
                    help="seconds of Poisson load per rate in the serving measurement (0 = skip)")
    ap.add_argument("--serving-search", type=int, default=3,
                    help="bisection steps of the sustained-capacity search (runs of --serving-seconds each)")
    ap.add_argument("--p99-bound-ms", type=float, default=25.0,
                    help="p99 latency bound that defines the sustained serving capacity")
    ap.add_argument("--verify-only", action="store_true",
                    help="sign the batch once, then time hs_verify_batch on it (3 calls) and print one line")
    ap.add_argument("--probe-only", action="store_true",
                    help="run the integer-pipe and SHA-2 mix probes only and print one line (profiler captures)")
    ap.add_argument("--count", type=int, default=16384,
                    help="messages per step (smaller counts are for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "own":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.verify_only:
        return run_verify_only(args)
    if args.probe_only:
        return run_probe_only()
    return run_own(args)


if __name__ == "__main__":
    sys.exit(main())
