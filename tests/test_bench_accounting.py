"""The roofline's work accounting in bench.py (compressions or Keccak
permutations per signature and stage) agrees with what the oracle actually
hashes: the blocks of each tweakable-hash call are read off the oracle's
per-thread counters (SHA-2 blocks after the PK.seed block, or Keccak-f
permutations) and assembled into the per-stage totals by the scheme's
structure, then compared with bench.STAGE_WORK / bench.KECCAK_WORK."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

SHA = ("128f", "192f", "256f", "128s", "192s", "256s")
WORDS = [3, 0, 1, 2, 2, 9, 4, 77]


def _blocks(O, ps, which, l=0):
    """(SHA-256 blocks, SHA-512 blocks, permutations) of one call, without
    the PK.seed block of the SHA-2 forms."""
    P = O.params(ps)
    O.counters(reset=True)
    data = bytes((l if l else (2 if which == O.THASH_H else 1)) * P.n)
    O.thash(ps, which, bytes(P.n), WORDS, data if which != O.THASH_PRF else b"", l=l, sk_seed=bytes(P.n))
    c = O.counters(reset=True)
    if ps.startswith("shake-"):
        return 0, 0, c[6]
    return c[0] - (0 if P.big and which in (O.THASH_H, O.THASH_T) else 1), \
        c[1] - (1 if P.big and which in (O.THASH_H, O.THASH_T) else 0), 0


def _stage_work(O, ps):
    P = O.params(ps)
    f = _blocks(O, ps, O.THASH_F)
    prf = _blocks(O, ps, O.THASH_PRF)
    h = _blocks(O, ps, O.THASH_H)
    tl = _blocks(O, ps, O.THASH_T, l=P.len)
    tk = _blocks(O, ps, O.THASH_T, l=P.k)
    leaves, fl = 2 ** P.hp, 2 ** P.a

    def comb(*terms):
        return tuple(sum(n * t[i] for n, t in terms) for i in range(3))

    tree = comb((P.d * leaves * P.len, prf), (P.d * leaves * P.len * 15, f), (P.d * leaves, tl),
                (P.d * (leaves - 1), h))
    fors = comb((P.k * fl, prf), (P.k * fl, f), (P.k * (fl - 1), h), (1, tk))
    return tree, fors


@pytest.mark.parametrize("ps", SHA)
def test_sha2_stage_work_matches_oracle(O, ps):
    tree, fors = _stage_work(O, ps)
    assert bench.STAGE_WORK[ps]["tree"] == tree[:2], (ps, tree)
    assert bench.STAGE_WORK[ps]["fors"] == fors[:2], (ps, fors)
    P = O.params(ps)
    assert bench.STAGE_WORK[ps]["wots"] == (P.d * P.len * (1 + 7.5), 0)   # PRF + expected digit sum


@pytest.mark.parametrize("ps", SHA)
def test_shake_stage_work_matches_oracle(O, ps):
    tree, fors = _stage_work(O, "shake-" + ps)
    assert bench.KECCAK_WORK["shake-" + ps]["tree"] == tree[2], (ps, tree)
    assert bench.KECCAK_WORK["shake-" + ps]["fors"] == fors[2], (ps, fors)


def test_per_call_blocks(O):
    # after the PK.seed block every F / PRF is one SHA-256 block, every H one
    # SHA-x block; SHAKE: one permutation each
    for ps in SHA:
        P = O.params(ps)
        assert _blocks(O, ps, O.THASH_F) == (1, 0, 0)
        assert _blocks(O, ps, O.THASH_PRF) == (1, 0, 0)
        assert _blocks(O, ps, O.THASH_H) == ((0, 1, 0) if P.big else (1, 0, 0))
        assert _blocks(O, "shake-" + ps, O.THASH_F) == (0, 0, 1)
        assert _blocks(O, "shake-" + ps, O.THASH_H) == (0, 0, 1)


def _enumerated_step_alu(nw, ctx):
    """ALU ops of one one-block SHA-256 F / PRF call, enumerated round by
    round and word by word: message words 0..4 are the address (their
    rounds, round 5 but for its message word, and their sigma0 terms come
    from a per-chain context when ctx), words
    5 .. 5 + nw carry data, words 6 + nw .. 14 are zero, word 15 is the
    constant bit length.  Sigma / sigma terms of a known word cost nothing."""
    known = set(range(6 + nw, 15)) | {15}
    hoisted = {1, 2, 3, 4} if ctx else set()
    # W17 = sigma1(W15) + W10 + sigma0(W2) + W1 and W19 = sigma1(W17) + W12 +
    # sigma0(W4) + W3 involve the address and known words only when words
    # 10 and 12 are zero (nw = 4): their sigma1 terms come from the context
    addr_only = {17, 19} if ctx and all(w in known for w in (10, 12)) else set()
    rounds = range(6, 64) if ctx else range(64)
    ops = 10 * len(rounds)                         # Sigma0, Sigma1 (4 each), Ch, Maj
    for t in range(16, 64):
        if (t - 2) not in known and (t - 2) not in addr_only:
            ops += 4                               # sigma1(W[t-2])
        if (t - 15) not in known and (t - 15) not in hoisted:
            ops += 4                               # sigma0(W[t-15])
    return ops


@pytest.mark.parametrize("nw", [4, 6, 8])
def test_executed_alu_model(nw):
    assert bench._step_alu(nw, True) == _enumerated_step_alu(nw, True)
    assert bench._step_alu(nw, False) == _enumerated_step_alu(nw, False)
    assert bench._step_alu(nw, False) <= bench.ALU_C256


def test_executed_alu_never_exceeds_full_basis():
    for ps in SHA:
        for st in ("tree", "fors"):
            e, f = bench.exec_alu_per_sig(ps, st), bench.alu_ops_per_sig(ps, st)
            assert 0.85 * f < e <= f, (ps, st)      # the contexts skip at most 7 rounds' worth
    # 128f TREE: 176 leaves x (35 chains x (2 x 84 + 16 x 908) + 10 x 1024) + 154 x 1024
    assert bench.exec_alu_per_sig("128f", "tree") == 176 * (35 * (2 * 84 + 16 * 908) + 10 * 1024) + 154 * 1024


def test_summary_lists_headline_figures():
    line = {"value": 1.0, "e2e": {"value": 2.0}, "roofline": {"frac": 0.9, "frac_full_compression": 0.95,
                                                               "issue_frac": 0.6},
            "plain_per_stage": {"value": 0.8},
            "serving": {"rho_0.75": {"seconds": 60, "value": 3, "p50_ms": 1, "p99_ms": 2},
                        "sustained": {"rho": 0.9, "offered": 9, "value": 8, "p50_ms": 3, "p99_ms": 20,
                                      "seconds": 60}, "p99_bound_ms": 25, "burst": {"value": 10}},
            "other_configs": {"mixed_small": {"plain_per_set_calls": {"ms_per_step": 1.5}, "messages": 96}}}
    sm = bench.summarize(line)
    assert sm["alu_frac_executed"] == 0.9 and sm["issue_frac"] == 0.6
    assert sm["plain_per_stage_sig_per_s"] == 0.8
    assert sm["serving_rho_0.75"]["p99_ms"] == 2 and sm["serving_sustained"]["rho"] == 0.9
    assert sm["mixed_small_ms"] == {"plain_per_set_calls": 1.5}


def test_sha_mix_pricing():
    """The SHA-2 mix fraction prices a stage's executed SHA-256 ALU work in
    compression equivalents (1024 each) at the probe's SHA-256 rate and its
    SHA-512 blocks at the probe's SHA-512 rate: a kernel running exactly at
    the probe's rates reads 1.0."""
    mix = {"sha256_per_clk_sm": 0.05, "sha512_per_clk_sm": 0.02}
    sms, mhz, count = 152, 2000.0, 1000
    for ps in SHA:
        for st in ("tree", "fors"):
            alu256, c512 = bench.exec_split_per_sig(ps, st)
            assert alu256 + c512 * bench.ALU_C512 == bench.exec_alu_per_sig(ps, st)
            per_s = lambda r: r * sms * mhz * 1e6
            want_ms = 1e3 * count * (alu256 / 1024 / per_s(0.05) + c512 / per_s(0.02))
            assert abs(bench.sha_mix_time_ms(ps, st, count, mix, sms, mhz) - want_ms) < 1e-9 * want_ms
    ms = bench.sha_mix_time_ms("128f", "tree", count, mix, sms, mhz)
    r = bench.sha_mix_roofline(dict(mix, sha256_plain_per_clk_sm=0.04), sms, mhz, "128f", count, ms, 64.0)
    assert abs(r["tree_frac"] - 1.0) < 1e-4
    assert r["alu_efficiency_of_mix"]["sha256"] == round(0.05 * 1024 / 64.0, 4)
    assert r["alu_efficiency_of_mix"]["sha512"] == round(0.02 * 2624 / 64.0, 4)
    # the SHA-512 sets' stages carry SHA-512 blocks, the n = 16 sets none
    assert bench.exec_split_per_sig("128f", "fors")[1] == 0
    assert bench.exec_split_per_sig("256f", "fors")[1] == bench.STAGE_WORK["256f"]["fors"][1]
