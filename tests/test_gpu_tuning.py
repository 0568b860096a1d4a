"""Every compiled launch-shape variant gives the same signatures.

The tuning knobs (lanes per FORS tree; TREE_Sign's form, addition policy,
chains per thread and occupancy variant; the WOTS+ chain checkpoint stride,
for all sets and per set) may only change speed.  For each parameter set,
each variant signs the same seeded batch; all outputs must be byte-equal to
the default's, and the default's must equal the oracle on sampled messages.
"""
import numpy as np
import pytest

from paper_2512_23969_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ps", ["toy", "128f", "192f", "256f", "128s"])
def test_variants_identical(hs, O, ps):
    import torch
    from paper_2512_23969_gb300 import autotune
    wl = inputs.make(ps, 24, num_keys=3, lengths=("uniform", 0, 150), seed=707)
    pk, sk = hs.hs_keygen(ps, torch.from_numpy(wl.seeds).cuda())
    msgs = torch.from_numpy(wl.msgs).cuda()
    lens = torch.from_numpy(wl.lens).cuda()
    kidx = torch.from_numpy(wl.key_idx).cuda()

    def sign():
        s = hs.hs_sign_batch(ps, sk, msgs, lens, key_idx=kidx, num_keys=wl.num_keys)
        torch.cuda.synchronize()
        return s.cpu()

    saved = {k: autotune.get(ps, k) for k in autotune.KNOBS}
    ref = sign()
    osk = [O.keygen(ps, bytes(s))[1] for s in wl.seeds]
    for i in (0, 7, 23):
        assert ref[i].numpy().tobytes() == O.sign(ps, osk[wl.key_idx[i]], wl.message(i))
    try:
        # every knob's compiled values, with TREE_Sign in both of its forms
        # (a thread per chain at this batch size by default; per leaf when
        # the split threshold is 0), each alternative from the defaults
        for split in (saved["tree_split_below"], 0):
            autotune.set(ps, "tree_split_below", split)
            for knob in autotune.KNOBS:
                if knob == "tree_split_below":
                    continue
                for v in autotune.options(ps, knob):
                    autotune.set(ps, knob, v)
                    assert torch.equal(sign(), ref), (split, knob, v)
                autotune.set(ps, knob, saved[knob])
        autotune.set(ps, "tree_split_below", saved["tree_split_below"])
        for v in autotune.options(ps, "tree_split_below"):
            autotune.set(ps, "tree_split_below", v)
            assert torch.equal(sign(), ref), ("tree_split_below", v)
        autotune.set(ps, "tree_split_below", saved["tree_split_below"])
        for ck in (0, 1, 2, 4, 8):
            hs.hs_set_chain_checkpoint(ck)
            assert torch.equal(sign(), ref), ("checkpoint", ck)
    finally:
        hs.hs_set_chain_checkpoint(2)
        for k, v in saved.items():
            autotune.set(ps, k, v)


def test_tune_options_and_errors(hs):
    from paper_2512_23969_gb300 import autotune
    for ps in ("128f", "192f", "256f", "toy"):
        for knob in autotune.KNOBS:
            opts = autotune.options(ps, knob)
            assert opts and autotune.get(ps, knob) in opts
    with pytest.raises(hs.HSError):
        autotune.set("128f", "fors_lanes", 3)
