"""Message stage at the sizes the workloads reach and beyond: lengths on
both sides of every SHA-256 (64 B), SHA-512 (128 B) and SHAKE256 (136 B)
block boundary, the 64 KB maximum of the mixed workload, and 1 MB -- packed
back to back, so most messages start at an odd address.  Every signature
must equal the oracle's, and in FIPS 205 mode too (the context prefix then
shifts every message inside its first block).  The SHA-2 sets run both
forms of the message stage: a thread per message, and a warp per message
with the blocks' schedules computed by the lanes (HS_TUNE_MSG_WARP_BELOW)."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2512_23969_gb300 import inputs

pytestmark = pytest.mark.gpu

LENS = [0, 1, 3, 55, 56, 63, 64, 65, 111, 112, 127, 128, 129, 135, 136, 137, 271, 272, 273, 1023,
        65535, 65536, 1 << 20]


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("ps", ["128f", "192f", "256f", "shake-128f", "shake-256f"])
def test_long_and_boundary_messages(hs, O, ps):
    import torch
    from paper_2512_23969_gb300 import autotune
    wl = inputs.make(ps, len(LENS), num_keys=2, lengths=LENS, seed=4100, key_mode="random")
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    d = [_dev(x) for x in (wl.msgs, wl.lens, wl.key_idx)]
    osk = [O.keygen(ps, bytes(s))[1] for s in wl.seeds]
    with ThreadPoolExecutor(16) as ex:
        want = list(ex.map(lambda i: O.sign(ps, osk[int(wl.key_idx[i])], wl.message(i)), range(len(LENS))))
        wantf = list(ex.map(lambda i: O.slh_sign(ps, osk[int(wl.key_idx[i])], b"ctx7", wl.message(i)),
                            range(len(LENS))))
    saved = autotune.get(ps, "msg_warp_below")
    forms = (0,) if ps.startswith("shake-") else (0, 1 << 20)    # a thread / a warp per message
    try:
        for below in forms:
            autotune.set(ps, "msg_warp_below", below)
            got = hs.hs_sign_batch(ps, sk, d[0], d[1], key_idx=d[2], num_keys=2).cpu().numpy()
            fips = hs.hs_slh_sign_batch(ps, sk, d[0], d[1], ctx=b"ctx7", key_idx=d[2], num_keys=2).cpu().numpy()
            for i, L in enumerate(LENS):
                assert got[i].tobytes() == want[i], (below, L)
                assert fips[i].tobytes() == wantf[i], (below, L)
            ok = hs.hs_verify_batch(ps, pk, d[0], d[1], torch.from_numpy(got).cuda(), key_idx=d[2], num_keys=2)
            assert ok.cpu().numpy().all(), below
            bad = torch.from_numpy(got).cuda()
            bad[len(LENS) - 1, 40] ^= 1               # a FORS secret of the 1 MB message's signature
            ok = hs.hs_verify_batch(ps, pk, d[0], d[1], bad, key_idx=d[2], num_keys=2)
            assert ok.cpu().numpy().tolist() == [1] * (len(LENS) - 1) + [0], below
    finally:
        autotune.set(ps, "msg_warp_below", saved)
