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
