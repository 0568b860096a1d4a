"""Measured launch-shape autotuner for the signer's kernels.

The library compiles a few variants per parameter set -- lanes per FORS
tree; TREE_Sign's addition placement (which pipe runs the SHA-256 sums),
chains per thread (threads per tree: one thread per leaf running one chain
at a time, or two interleaved) and minimum resident blocks -- and takes the
batch size below which TREE_Sign runs a thread per chain and the chain
checkpoint stride at run time; ``hs_tune_options`` / ``hs_tune_set``
(include/hs.h) expose them.  This module times each value on a seeded batch
with the library's own per-stage CUDA events (the stages the knob changes:
TREE_Sign and WOTS+_Sign together for the checkpoint stride) and keeps the
fastest, in a JSON cache keyed by the device (name, SM count,
compute capability, driver) so that a later process can apply it without
re-measuring.  Signatures are identical for every setting, so the choice is
purely about speed -- the same idea as the paper's offline tuning followed by
profiling-based selection (Sec. III-B-2, III-C), with measurement on the
target GPU in place of Alg. 1's analytic model.
"""
import ctypes as C
import json
import os

import numpy as np

from . import hs, inputs

KNOBS = {"fors_lanes": 0, "tree_min_blocks": 1, "tree_split_below": 2, "tree_policy": 3, "tree_chains": 4,
         "checkpoint": 5, "tree_step_us": 6, "tree_split_ns": 7, "msg_warp_below": 8}
# knobs whose values are measured quantities rather than compiled variants
FREE_KNOBS = ("tree_split_below", "tree_step_us", "tree_split_ns", "msg_warp_below")
# the stages each knob changes, timed together; in tuning order (TREE_Sign's
# policy and chains per thread before its min blocks: the alternatives of
# each are compiled only with the other two at their defaults)
STAGE_OF_KNOB = {"fors_lanes": ("fors",), "tree_policy": ("tree",), "tree_chains": ("tree",),
                 "tree_min_blocks": ("tree",), "checkpoint": ("tree", "wots")}
DEFAULT_COUNTS = {"128f": 16384, "192f": 8192, "256f": 8192, "toy": 4096, "128s": 512, "192s": 256, "256s": 256,
                  "shake-128f": 4096, "shake-192f": 2048, "shake-256f": 2048, "shake-128s": 256, "shake-192s": 256,
                  "shake-256s": 256, "robust-128f": 8192, "robust-192f": 4096, "robust-256f": 4096}
# batch sizes at which the two TREE_Sign forms are compared, per family
# (down to a few messages: the per-leaf form is latency-bound below one wave
# of threads, so its time hardly falls with the batch while the chain-
# parallel form's does)
SPLIT_COUNTS = {"f": (8, 16, 32, 64, 128, 256, 1024, 2048, 4096, 8192), "s": (8, 16, 32, 64, 128, 256),
                "shake-f": (8, 16, 32, 64, 128, 256, 1024, 2048, 4096, 8192), "shake-s": (4, 8, 16, 32, 64, 128)}


def _family(ps):
    if ps.startswith("robust-"):
        ps = ps[len("robust-"):]
    base = ps[len("shake-"):] if ps.startswith("shake-") else ps
    fam = "s" if base.endswith("s") else "f"
    return ("shake-" + fam) if ps.startswith("shake-") else fam
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def options(params, knob):
    L = hs.load()
    L.hs_tune_options.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int32), C.c_int]
    L.hs_tune_options.restype = C.c_int
    vals = (C.c_int32 * 16)()
    n = L.hs_tune_options(hs.PARAMS[params], KNOBS[knob], vals, 16)
    return [int(v) for v in vals[:max(n, 0)]]


def get(params, knob):
    L = hs.load()
    L.hs_tune_get.argtypes = [C.c_int, C.c_int]
    L.hs_tune_get.restype = C.c_int32
    return int(L.hs_tune_get(hs.PARAMS[params], KNOBS[knob]))


def set(params, knob, value):   # noqa: A001 - mirrors hs_tune_set
    L = hs.load()
    L.hs_tune_set.argtypes = [C.c_int, C.c_int, C.c_int32]
    L.hs_tune_set.restype = C.c_int
    rc = L.hs_tune_set(hs.PARAMS[params], KNOBS[knob], int(value))
    if rc != 0:
        raise hs.HSError(rc, hs.last_error())


def try_set(params, knob, value):
    """set(), returning False where the value (or, for TREE_Sign's knobs,
    the combination with the other two) is not compiled."""
    try:
        set(params, knob, value)
        return True
    except hs.HSError:
        return False


def device_key():
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    drv = C.c_int(0)
    try:
        C.CDLL("libcuda.so.1").cuDriverGetVersion(C.byref(drv))
    except OSError:
        pass
    return "%s|sm%d%d|%dSM|drv%d" % (p.name, p.major, p.minor, p.multi_processor_count, drv.value)


def _batch(params, count, seed=4242):
    import torch
    wl = inputs.make(params, count, 16, 32, seed)
    pk, sk = hs.hs_keygen(params, torch.from_numpy(wl.seeds).cuda())
    dev = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("msgs", "lens", "key_idx")}
    sigs = torch.empty(count * hs.sig_bytes(params), dtype=torch.uint8, device="cuda")
    return wl, sk, dev, sigs


def _stage_ms(params, wl, sk, dev, sigs, stage, reps):
    """Best-of-reps time of a stage, or of the sum of several stages."""
    import torch
    stages = (stage,) if isinstance(stage, str) else tuple(stage)
    hs.hs_profile_enable(True)
    best = float("inf")
    for _ in range(reps + 1):                       # first call warms up
        hs.hs_sign_batch(params, sk, dev["msgs"], dev["lens"], key_idx=dev["key_idx"], sigs=sigs,
                         num_keys=wl.num_keys)
        torch.cuda.synchronize()
        prof = hs.hs_profile_read()
        best = min(best, sum(prof[st] for st in stages))
    hs.hs_profile_enable(False)
    return best


def _shape(ps):
    """(d, 2^h') of a set, for the per-leaf form's warp count."""
    n = {"128f": (22, 8), "192f": (22, 8), "256f": (17, 16), "toy": (2, 4), "128s": (7, 512), "192s": (7, 512),
         "256s": (8, 256)}
    base = ps.split("-")[-1]
    return n[base]


def tune_tree_costs(ps, reps=3, verbose=True):
    """The per-leaf TREE_Sign time of one step (a warp per SM sub-partition:
    the per-leaf time grows in whole steps) and the chain-parallel time per
    message, measured at one and at four steps' worth of messages."""
    import torch
    d, leaves = _shape(ps)
    smsp = 4 * torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    one = max(1, (smsp * 32) // (d * leaves))
    saved = get(ps, "tree_split_below")
    set(ps, "tree_step_us", 0)
    set(ps, "tree_split_ns", 0)
    try:
        wl, sk, dev, sigs = _batch(ps, one)
        set(ps, "tree_split_below", 0)
        leaf_ms = _stage_ms(ps, wl, sk, dev, sigs, "tree", reps)
        wl, sk, dev, sigs = _batch(ps, 4 * one)
        set(ps, "tree_split_below", 1 << 30)
        split_ms = _stage_ms(ps, wl, sk, dev, sigs, "tree", reps)
    finally:
        set(ps, "tree_split_below", saved)
    step_us, split_ns = int(round(leaf_ms * 1e3)), int(round(split_ms * 1e6 / (4 * one)))
    set(ps, "tree_step_us", step_us)
    set(ps, "tree_split_ns", split_ns)
    if verbose:
        print("tune %s tree costs: per-leaf step %d us (%d msgs), chain-parallel %d ns per message"
              % (ps, step_us, one, split_ns), flush=True)
    return {"tree_step_us": {"best": step_us, "messages": one},
            "tree_split_ns": {"best": split_ns, "messages": 4 * one}}


def tune_split(ps, counts=None, reps=3, verbose=True):
    """Batch size below which the chain-parallel TREE_Sign is faster: time
    the TREE stage in both forms at growing batch sizes."""
    counts = counts or SPLIT_COUNTS[_family(ps)]
    rows = {}
    below = 0
    set(ps, "tree_step_us", 0)                 # forms forced by the threshold alone while timing
    set(ps, "tree_split_ns", 0)
    for count in counts:
        wl, sk, dev, sigs = _batch(ps, count)
        ms = {}
        for form, thr in (("split", 1 << 30), ("leaf", 0)):
            set(ps, "tree_split_below", thr)
            ms[form] = _stage_ms(ps, wl, sk, dev, sigs, "tree", reps)
        rows[str(count)] = {k: round(v, 4) for k, v in ms.items()}
        if verbose:
            print("tune %s tree form at %d: split %.3f ms, per-leaf %.3f ms" % (ps, count, ms["split"], ms["leaf"]),
                  flush=True)
        if ms["split"] < ms["leaf"]:
            below = count * 2 if count == counts[-1] else counts[counts.index(count) + 1]
    set(ps, "tree_split_below", below)
    return {"best": below, "ms": rows}


MSG_COUNTS = (64, 128, 256, 512, 1024, 2048, 4096)


def tune_msg_warp(ps, counts=MSG_COUNTS, reps=3, verbose=True):
    """Batch size below which the message stage runs a warp per message:
    time the stage in both forms at growing batch sizes, with the serving
    workload's lengths (log-uniform 16 B - 4 KB).  The SHAKE sets have only
    the thread form (0)."""
    import torch
    if ps.startswith("shake-"):
        set(ps, "msg_warp_below", 0)
        return {"best": 0}
    rows = {}
    below = 0
    for count in counts:
        wl = inputs.make(ps, count, 16, ("loguniform", 16, 4096), 4343 + count)
        pk, sk = hs.hs_keygen(ps, torch.from_numpy(wl.seeds).cuda())
        dev = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("msgs", "lens", "key_idx")}
        sigs = torch.empty(count * hs.sig_bytes(ps), dtype=torch.uint8, device="cuda")
        ms = {}
        for form, thr in (("warp", 1 << 30), ("thread", 0)):
            set(ps, "msg_warp_below", thr)
            ms[form] = _stage_ms(ps, wl, sk, dev, sigs, "message", reps)
        rows[str(count)] = {k: round(v, 4) for k, v in ms.items()}
        if verbose:
            print("tune %s message form at %d: warp %.4f ms, thread %.4f ms" % (ps, count, ms["warp"], ms["thread"]),
                  flush=True)
        if ms["warp"] < ms["thread"]:
            below = count * 2 if count == counts[-1] else counts[counts.index(count) + 1]
    set(ps, "msg_warp_below", below)
    return {"best": below, "ms": rows, "lengths": "log-uniform 16 B - 4 KB, 16 keys"}


def tune(params_list=("128f", "192f", "256f"), counts=None, reps=3, verbose=True):
    """Time every compiled variant of every knob; apply and return the best
    ({params: {knob: {"best": v, "ms": {v: ms}}}})."""
    import torch
    result = {}
    for ps in params_list:
        count = (counts or {}).get(ps, DEFAULT_COUNTS[ps])
        wl, sk, dev, sigs = _batch(ps, count)
        ref = None
        result[ps] = {}
        result[ps]["tree_split_below"] = tune_split(ps, reps=reps, verbose=verbose)
        result[ps].update(tune_tree_costs(ps, reps=reps, verbose=verbose))
        result[ps]["msg_warp_below"] = tune_msg_warp(ps, reps=reps, verbose=verbose)
        for knob in ("tree_min_blocks", "tree_chains"):   # 0 min blocks, 1 chain: every policy is compiled there
            try_set(ps, knob, options(ps, knob)[0])
        for knob, stage in STAGE_OF_KNOB.items():
            timings = {}
            for v in options(ps, knob):
                if not try_set(ps, knob, v):            # not compiled with the other knobs' choice
                    continue
                timings[v] = _stage_ms(ps, wl, sk, dev, sigs, stage, reps)
                cur = sigs.clone()
                if ref is None:
                    ref = cur
                elif not torch.equal(ref, cur):
                    raise RuntimeError("tuning %s=%d changed the signatures of %s" % (knob, v, ps))
                if verbose:
                    print("tune %s %s=%d: %s %.3f ms" % (ps, knob, v, "+".join(stage), timings[v]), flush=True)
            best = min(timings, key=timings.get)
            set(ps, knob, best)
            result[ps][knob] = {"best": best, "ms": {str(k): round(t, 4) for k, t in timings.items()},
                                "count": count, "stages": list(stage)}
    return result


def save(result, path=CACHE):
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    entry = data.setdefault(device_key(), {})
    for ps, knobs in result.items():                     # keep the sets and knobs not tuned this time
        entry.setdefault(ps, {}).update(knobs)
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


def apply(path=CACHE):
    """Apply the cached choices for this device; return them (or {} if none)."""
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        data = json.load(f)
    entry = data.get(device_key(), {})
    order = ("tree_split_below", "tree_step_us", "tree_split_ns", "fors_lanes", "tree_min_blocks", "tree_policy",
             "tree_chains", "checkpoint", "msg_warp_below")
    for ps, knobs in entry.items():
        if ps not in hs.PARAMS:
            continue
        for knob in order:                  # min blocks first: the others' alternatives need its default
            rec = knobs.get(knob)
            if rec is not None and (knob in FREE_KNOBS or rec.get("best") in options(ps, knob)):
                try_set(ps, knob, rec["best"])
    return entry


if __name__ == "__main__":
    import sys
    args = sys.argv[1:]
    if args and args[0] == "--split-only":     # re-measure only the TREE_Sign form choice
        sets = args[1:] or list(DEFAULT_COUNTS)
        res = {ps: dict({"tree_split_below": tune_split(ps)}, **tune_tree_costs(ps)) for ps in sets}
    elif args and args[0] == "--msg-only":     # re-measure only the message stage's form choice
        sets = args[1:] or list(DEFAULT_COUNTS)
        res = {ps: {"msg_warp_below": tune_msg_warp(ps)} for ps in sets}
    else:
        sets = args or list(DEFAULT_COUNTS)
        res = tune(sets)
    save(res)
    print(json.dumps(res, indent=1))
