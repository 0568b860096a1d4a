"""Tree sharing within a batch (hs_set_tree_sharing) changes no signature
byte: batches with many messages per key are signed with sharing on and off
(with and without chain checkpoints, in both TREE_Sign forms) and compared
byte for byte, and sampled messages against the oracle."""
import numpy as np
import pytest

from paper_2512_23969_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("ps,count,keys", [("toy", 200, 3), ("128f", 300, 2), ("192f", 120, 2), ("256f", 150, 2),
                                           ("128s", 40, 2), ("shake-128f", 300, 2)])
def test_sharing_is_bit_exact(hs, O, ps, count, keys):
    import torch
    from paper_2512_23969_gb300 import autotune
    wl = inputs.make(ps, count, num_keys=keys, lengths=("uniform", 0, 64), seed=1200 + count, key_mode="random")
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    m, l, k = _dev(wl.msgs), _dev(wl.lens), _dev(wl.key_idx)

    def sign():
        s = hs.hs_sign_batch(ps, sk, m, l, key_idx=k, num_keys=keys)
        torch.cuda.synchronize()
        rc, flags = hs.hs_check_status()
        assert rc == 0 and flags == 0
        return s.cpu()

    saved = autotune.get(ps, "tree_split_below")
    try:
        hs.hs_set_tree_sharing(False)
        ref = sign()
        for ck in (2, 0):
            hs.hs_set_chain_checkpoint(ck)
            for split in (0, 1 << 20):
                autotune.set(ps, "tree_split_below", split)
                hs.hs_set_tree_sharing(True)
                assert torch.equal(sign(), ref), (ck, split)
                hs.hs_set_tree_sharing(False)
    finally:
        hs.hs_set_tree_sharing(False)
        hs.hs_set_chain_checkpoint(2)
        autotune.set(ps, "tree_split_below", saved)
    osk = [O.keygen(ps, bytes(s))[1] for s in wl.seeds]
    for i in (0, count - 1):
        assert ref[i].numpy().tobytes() == O.sign(ps, osk[wl.key_idx[i]], wl.message(i))
