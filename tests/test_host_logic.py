"""Host-side logic that needs no GPU: the seeded workload generators (sizes,
distributions, determinism), the binding's parameter tables against the C
header and library, and the tuning cache (merging and applying per device)."""
import json
import os
import re

import numpy as np
import pytest

from paper_2512_23969_gb300 import autotune, hs, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_config_recipes_sizes_and_determinism():
    c0 = inputs.config(0)
    assert (c0.params, c0.count, c0.num_keys) == ("128f", 64, 1) and set(c0.lens.tolist()) == {32}
    c1 = inputs.config(1)
    assert (c1.params, c1.count, c1.num_keys) == ("128f", 16384, 16)
    assert np.array_equal(c1.key_idx, np.arange(16384, dtype=np.uint32) % 16)
    assert set(c1.lens.tolist()) == {32} and c1.msgs.size == 16384 * 32
    assert len(set(c1.subset.tolist())) == 256 and c1.subset.max() < 16384
    again = inputs.config(1)
    assert np.array_equal(again.msgs, c1.msgs) and np.array_equal(again.seeds, c1.seeds)
    for ps in ("192f", "256f"):
        c2 = inputs.config(2, ps)
        assert (c2.params, c2.count, c2.num_keys) == (ps, 8192, 16)
        assert c2.lens.min() >= 32 and c2.lens.max() <= 1024 and c2.seeds.shape[1] == 3 * inputs.N_BYTES[ps]
    assert not np.array_equal(inputs.config(2, "192f").msgs[:64], inputs.config(2, "256f").msgs[:64])


def test_log_uniform_lengths():
    rng = np.random.default_rng(1)
    L = inputs.log_uniform_lengths(rng, 200000, 16, 65536)
    assert L.min() >= 16 and L.max() <= 65536
    # log-uniform: the median sits near the geometric mean of the range
    assert 0.8 < np.median(L) / np.sqrt(16 * 65537) < 1.25
    # a quarter of the mass per quarter of the log range
    q = np.log(L.astype(np.float64) / 16) / np.log(65537 / 16)
    hist = np.histogram(q, bins=4, range=(0, 1))[0] / L.size
    assert np.all(np.abs(hist - 0.25) < 0.02)


def test_mixed_recipe():
    wls = inputs.mixed()
    assert [wl.params for wl in wls] == ["128f", "192f", "256f"]
    assert sum(wl.count for wl in wls) == 32768
    frac = np.array([wl.count for wl in wls]) / 32768
    assert np.all(np.abs(frac - np.array([0.5, 0.3, 0.2])) < 0.02)
    assert [wl.num_keys for wl in wls] == [32, 19, 13]
    allidx = np.sort(np.concatenate([wl.subset for wl in wls]))
    assert np.array_equal(allidx, np.arange(32768))             # every draw lands in exactly one set
    for wl in wls:
        assert wl.lens.min() >= 16 and wl.lens.max() <= 65536
        assert wl.key_idx.max() < wl.num_keys


def test_serving_trace():
    tr = inputs.serving_trace(rate=20000, seconds=2.0, pool=4096, seed=11)
    n = len(tr["params"])
    assert abs(n - 40000) < 4 * np.sqrt(40000)                   # Poisson count
    a = tr["arrival_ns"]
    assert np.all(np.diff(a.astype(np.int64)) >= 0) and a[-1] < 2.5e9
    frac = np.bincount(tr["params"], minlength=3) / n
    assert np.all(np.abs(frac - np.array([0.6, 0.25, 0.15])) < 0.02)
    for si, ps in enumerate(("128f", "192f", "256f")):
        sel = tr["params"] == si
        assert tr["keys"][sel].max() < (614, 256, 154)[si]
        assert tr["seeds"][ps].shape == ((614, 256, 154)[si], 3 * inputs.N_BYTES[ps])
    assert tr["pool_lens"].min() >= 16 and tr["pool_lens"].max() <= 4096
    assert tr["pool_msgs"].size == int(tr["pool_lens"].sum()) and tr["pool_idx"].max() < 4096


def test_binding_tables_match_header_and_library():
    text = open(os.path.join(ROOT, "include", "hs.h")).read()
    enum = dict((k, int(v)) for k, v in re.findall(r"HS_([0-9A-Z_]+) = (\d+)", text) if not k.startswith("E"))
    assert int(re.search(r"#define HS_NUM_PARAMS (\d+)", text).group(1)) == hs.NUM_PARAMS == len(hs.PARAMS)
    for name, pid in hs.PARAMS.items():
        assert enum[name.upper().replace("-", "_")] == pid, name
        assert hs.sig_bytes(name) == hs.SIG_BY_ID[pid]
        if name != "toy":
            assert int(hs.load().hs_sk_bytes(pid)) == 4 * hs.N_BYTES[name]


def test_tuning_cache_merges_and_applies(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "device_key", lambda: "TEST-DEVICE|sm103|152SM")
    path = str(tmp_path / "tuned.json")
    autotune.save({"128f": {"fors_lanes": {"best": 4}}}, path)
    autotune.save({"192f": {"tree_min_blocks": {"best": 4}}}, path)       # another set: kept side by side
    autotune.save({"128f": {"tree_split_below": {"best": 1024}}}, path)   # same set, another knob: kept too
    autotune.save({"128f": {"fors_lanes": {"best": 2}}}, path)            # same knob: replaced
    data = json.load(open(path))["TEST-DEVICE|sm103|152SM"]
    assert set(data) == {"128f", "192f"}
    assert data["128f"] == {"tree_split_below": {"best": 1024}, "fors_lanes": {"best": 2}}
    before = {(ps, k): autotune.get(ps, k) for ps in ("128f", "192f") for k in autotune.KNOBS}
    try:
        autotune.save({"128f": {"fors_lanes": {"best": 8}, "tree_split_below": {"best": 512}},
                       "192f": {"fors_lanes": {"best": 3}}}, path)          # 3 lanes: not compiled, skipped
        applied = autotune.apply(path)
        assert "128f" in applied
        assert autotune.get("128f", "fors_lanes") == 8 and autotune.get("128f", "tree_split_below") == 512
        assert autotune.get("192f", "fors_lanes") == before[("192f", "fors_lanes")]
        with pytest.raises(hs.HSError):
            autotune.set("128f", "fors_lanes", 3)
    finally:
        for (ps, k), v in before.items():
            autotune.set(ps, k, v)


def test_binding_rejects_wrong_element_sizes_and_short_buffers():
    """The binding checks element sizes and buffer lengths before an address
    reaches the C ABI (a wrong dtype would otherwise be read past its end);
    every case below raises before any CUDA call, so it runs on the CPU."""
    import torch
    S, n = hs.sig_bytes("128f"), 16
    sk = np.zeros((2, 4 * n), np.uint8)
    pk = np.zeros((2, 2 * n), np.uint8)
    msgs = np.zeros(64, np.uint8)
    lens = np.full(2, 32, np.uint64)
    kidx = np.zeros(2, np.uint32)
    cases = [
        lambda: hs.hs_sign_batch("128f", sk, msgs, lens.astype(np.int32)),               # 4-byte lengths
        lambda: hs.hs_sign_batch("128f", sk, msgs, lens, key_idx=kidx.astype(np.int64)),  # 8-byte key indices
        lambda: hs.hs_sign_batch("128f", sk, msgs, lens, key_idx=kidx[:1]),               # one index short
        lambda: hs.hs_sign_batch("128f", sk, msgs[:63], lens),                            # lengths add to 64
        lambda: hs.hs_sign_batch("128f", sk, msgs, lens, sigs=np.zeros(2 * S - 1, np.uint8)),
        lambda: hs.hs_sign_batch("128f", sk.reshape(-1)[:100], msgs, lens, num_keys=2),    # 2 keys need 128 B
        lambda: hs.hs_sign_batch("128f", torch.zeros(2, 64, dtype=torch.int32), msgs, lens),
        lambda: hs.hs_verify_batch("128f", pk.reshape(-1)[:63], msgs, lens, np.zeros(2 * S, np.uint8), num_keys=2),
        lambda: hs.hs_verify_batch("128f", pk, msgs, lens, np.zeros(2 * S - 16, np.uint8)),
        lambda: hs.hs_verify_batch("128f", pk, msgs, lens, np.zeros(2 * S, np.uint8), ok=np.zeros(1, np.uint8)),
        lambda: hs.hs_keygen("128f", np.zeros((2, 3 * n), np.uint8), pk=np.zeros(63, np.uint8)),
        lambda: hs.hs_keygen("128f", np.zeros((2, 3 * n), np.uint16)),
        lambda: hs.hs_slh_sign_batch("128f", sk, msgs, torch.full((2,), 32, dtype=torch.int32)),
        lambda: hs.hs_sign_batch_noalloc("128f", sk, msgs, lens, np.zeros(S, np.uint8)),
        lambda: hs.hs_sign_mixed([{"params": "128f", "sk": sk, "msgs": msgs, "lens": lens,
                                   "sigs": np.zeros(S, np.uint8)}]),
    ]
    for i, call in enumerate(cases):
        with pytest.raises(ValueError):
            call()
            pytest.fail("case %d passed the checks" % i)


def test_server_binding_checks_without_a_server():
    """Replay's per-request arrays and message pool, and submit's output
    buffer, are checked in the binding before the C ABI sees them (the
    checks run before the server handle is used, so a bare object works)."""
    srv = hs.Server.__new__(hs.Server)
    srv._h = None
    z8, z32, z64 = np.zeros(4, np.uint8), np.zeros(4, np.uint32), np.zeros(4, np.uint64)
    lens = np.full(2, 10, np.uint64)
    with pytest.raises(ValueError):
        srv.replay(z8, z32[:3], z32, np.zeros(20, np.uint8), lens, z64)          # 3 keys for 4 requests
    with pytest.raises(ValueError):
        srv.replay(z8, z32, z32, np.zeros(20, np.uint8), lens, z64[:2])          # 2 arrival times
    with pytest.raises(ValueError):
        srv.replay(z8, z32, z32, np.zeros(19, np.uint8), lens, z64)              # pool lengths add to 20
    with pytest.raises(ValueError):
        srv.submit("128f", 0, b"m", out=np.zeros(hs.sig_bytes("128f") - 1, np.uint8))


def test_tree_knob_combinations_follow_the_compiled_variants():
    """TREE_Sign's per-leaf kernel is compiled for its default (min blocks
    0, the set's addition policy, one chain per thread) and for each
    alternative of one knob with the other two at their defaults; the
    library refuses other combinations, and the SHAKE sets have no policy
    or chains-per-thread alternatives.  No CUDA call is made."""
    assert autotune.options("128f", "tree_policy") == [7, 15]
    assert autotune.options("192f", "tree_policy") == [7, 15]
    assert autotune.options("128f", "tree_chains") == [1, 2]
    assert autotune.options("shake-128f", "tree_policy") == [7]
    assert autotune.options("shake-128f", "tree_chains") == [1]
    assert autotune.options("toy", "tree_chains") == [1]
    assert autotune.options("128f", "checkpoint") == [0, 1, 2, 4, 8]
    assert autotune.get("128f", "tree_policy") == 7 and autotune.get("256f", "tree_policy") == 15
    saved = {k: autotune.get("128f", k) for k in autotune.KNOBS}
    try:
        autotune.set("128f", "tree_min_blocks", 6)
        assert not autotune.try_set("128f", "tree_policy", 15)     # (6, 15, 1) is not compiled
        assert not autotune.try_set("128f", "tree_chains", 2)      # (6, 7, 2) is not compiled
        autotune.set("128f", "tree_min_blocks", 0)
        autotune.set("128f", "tree_chains", 2)
        assert not autotune.try_set("128f", "tree_policy", 15)     # (0, 15, 2) is not compiled
        assert not autotune.try_set("128f", "tree_min_blocks", 6)
    finally:
        autotune.set("128f", "tree_chains", saved["tree_chains"])
        autotune.set("128f", "tree_min_blocks", saved["tree_min_blocks"])
        autotune.set("128f", "tree_policy", saved["tree_policy"])


def test_checkpoint_stride_per_set_and_process_wide():
    """hs_set_chain_checkpoint sets every set's stride and drops per-set
    choices; HS_TUNE_CHECKPOINT sets one set's.  No CUDA call is made."""
    try:
        autotune.set("192f", "checkpoint", 4)
        assert autotune.get("192f", "checkpoint") == 4 and autotune.get("128f", "checkpoint") == 2
        hs.hs_set_chain_checkpoint(1)
        assert autotune.get("192f", "checkpoint") == 1 and autotune.get("128f", "checkpoint") == 1
        assert not autotune.try_set("128f", "checkpoint", 3)
    finally:
        hs.hs_set_chain_checkpoint(2)


def test_message_form_knob():
    """HS_TUNE_MSG_WARP_BELOW: any threshold >= 0 for the SHA-2 sets (a warp
    per message below it), 0 only for the SHAKE sets, whose message stage has
    only the thread form.  No CUDA call is made."""
    assert autotune.get("128f", "msg_warp_below") in autotune.options("128f", "msg_warp_below")
    assert autotune.options("shake-128f", "msg_warp_below") == [0]
    assert autotune.get("shake-256s", "msg_warp_below") == 0
    saved = autotune.get("192f", "msg_warp_below")
    try:
        autotune.set("192f", "msg_warp_below", 777)          # not a listed suggestion: still accepted
        assert autotune.get("192f", "msg_warp_below") == 777
        assert not autotune.try_set("192f", "msg_warp_below", -1)
        assert not autotune.try_set("shake-192f", "msg_warp_below", 64)
        autotune.set("shake-192f", "msg_warp_below", 0)
    finally:
        autotune.set("192f", "msg_warp_below", saved)
