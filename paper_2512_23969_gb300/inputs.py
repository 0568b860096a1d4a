"""Seeded synthetic workloads (keys seeds, messages, lengths, key indices).

Shared by the tests, the benchmark and the oracle checks.  This module holds
no signing arithmetic at all: it only draws bytes and integers from
``numpy.random.default_rng``.

The paper signs fixed-length random messages (1 KB-4 KB in its input-size
study, Sec. IV); no public dataset is involved.  Recipes:
  * key seeds: ``rng.bytes(3n)`` per key, in key order;
  * messages: ``rng.bytes(L)`` per message, concatenated in order;
  * log-uniform lengths: ``floor(exp(U(ln lo, ln(hi + 1))))`` clipped to [lo, hi].
"""
from dataclasses import dataclass, field

import numpy as np

N_BYTES = {"128f": 16, "192f": 24, "256f": 32, "toy": 16, "128s": 16, "192s": 24, "256s": 32}
N_BYTES.update({"shake-" + k: v for k, v in list(N_BYTES.items()) if k != "toy"})
N_BYTES.update({"robust-" + k: N_BYTES[k] for k in ("128f", "192f", "256f")})
BASE_SEED = 23969


@dataclass
class Workload:
    """One batch: ``seeds`` (num_keys x 3n), packed ``msgs``, ``lens``, ``key_idx``."""
    name: str
    params: str
    seeds: np.ndarray          # uint8 [num_keys, 3n]
    msgs: np.ndarray           # uint8 [sum(lens)]
    lens: np.ndarray           # uint64 [count]
    key_idx: np.ndarray        # uint32 [count]
    subset: np.ndarray = field(default=None)   # message indices checked by the oracle

    @property
    def count(self):
        return int(self.lens.shape[0])

    @property
    def num_keys(self):
        return int(self.seeds.shape[0])

    @property
    def offsets(self):
        off = np.zeros(self.count + 1, dtype=np.uint64)
        np.cumsum(self.lens, out=off[1:])
        return off

    def message(self, i) -> bytes:
        off = self.offsets
        return self.msgs[int(off[i]):int(off[i + 1])].tobytes()


def log_uniform_lengths(rng, count, lo, hi):
    u = rng.uniform(np.log(lo), np.log(hi + 1), size=count)
    return np.clip(np.floor(np.exp(u)), lo, hi).astype(np.uint64)


def make(params, count, num_keys=1, lengths=32, seed=BASE_SEED, name="custom",
         subset=None, key_mode="mod"):
    """Generic seeded batch.

    ``lengths`` is an int (fixed), a ("uniform", lo, hi) or ("loguniform", lo, hi)
    tuple, or an explicit sequence.  ``key_mode`` "mod" assigns key i mod
    num_keys; "random" draws it uniformly.
    """
    rng = np.random.default_rng(seed)
    n = N_BYTES[params]
    seeds = np.frombuffer(rng.bytes(3 * n * num_keys), dtype=np.uint8).reshape(num_keys, 3 * n).copy()
    if isinstance(lengths, int):
        lens = np.full(count, lengths, dtype=np.uint64)
    elif isinstance(lengths, tuple) and lengths[0] == "uniform":
        lens = rng.integers(lengths[1], lengths[2] + 1, size=count).astype(np.uint64)
    elif isinstance(lengths, tuple) and lengths[0] == "loguniform":
        lens = log_uniform_lengths(rng, count, lengths[1], lengths[2])
    else:
        lens = np.asarray(lengths, dtype=np.uint64)
        assert lens.shape[0] == count
    total = int(lens.sum())
    msgs = np.frombuffer(rng.bytes(total), dtype=np.uint8).copy() if total else np.zeros(0, np.uint8)
    if key_mode == "mod":
        key_idx = (np.arange(count) % num_keys).astype(np.uint32)
    else:
        key_idx = rng.integers(0, num_keys, size=count).astype(np.uint32)
    sub = None
    if subset is not None:
        sub = np.sort(rng.choice(count, size=min(subset, count), replace=False))
    return Workload(name, params, seeds, msgs, lens, key_idx, sub)


def mixed(count=32768, mix=(0.5, 0.3, 0.2), keys=(32, 19, 13), lengths=("loguniform", 16, 65536),
          seed=BASE_SEED + 3, name="mixed"):
    """Mixed-parameter batch: each message draws its set from ``mix`` over
    (128f, 192f, 256f); per set, its own seeded keys and key indices drawn
    uniformly; message lengths log-uniform.  Returns one Workload per set
    (messages in draw order), with the global message index of each row in
    ``Workload.subset``."""
    rng = np.random.default_rng(seed)
    sets = ("128f", "192f", "256f")
    which = rng.choice(3, size=count, p=np.asarray(mix) / np.sum(mix))
    out = []
    for si, ps in enumerate(sets):
        idx = np.nonzero(which == si)[0]
        sub_seed = int(rng.integers(0, 2 ** 31))
        wl = make(ps, int(idx.size), keys[si], lengths, sub_seed, "%s-%s" % (name, ps), key_mode="random")
        wl.subset = idx
        out.append(wl)
    return out


def serving_trace(rate, seconds, mix=(0.6, 0.25, 0.15), keys=(614, 256, 154), lengths=(16, 4096),
                  pool=65536, seed=BASE_SEED + 4):
    """Open-loop serving load: Poisson arrivals at ``rate`` requests/s for
    ``seconds``; each request draws its set from ``mix`` over (128f, 192f,
    256f), a key uniformly among that set's keys, and a message from a pool
    of ``pool`` seeded messages with log-uniform lengths.  Returns a dict of
    arrays (params ids, key indices, pool indices, arrival times in ns) plus
    the pool and one seed row per key and set."""
    rng = np.random.default_rng(seed)
    n = int(rng.poisson(rate * seconds))
    gaps = rng.exponential(1.0 / rate, size=n)
    arrival = np.cumsum(gaps)
    arrival_ns = (arrival * 1e9).astype(np.uint64)
    which = rng.choice(3, size=n, p=np.asarray(mix) / np.sum(mix)).astype(np.uint8)
    kidx = np.zeros(n, dtype=np.uint32)
    for si in range(3):
        sel = which == si
        kidx[sel] = rng.integers(0, keys[si], size=int(sel.sum()))
    pool_lens = log_uniform_lengths(rng, pool, lengths[0], lengths[1])
    pool_msgs = np.frombuffer(rng.bytes(int(pool_lens.sum())), dtype=np.uint8).copy()
    pool_idx = rng.integers(0, pool, size=n).astype(np.uint32)
    seeds = {}
    for si, ps in enumerate(("128f", "192f", "256f")):
        seeds[ps] = np.frombuffer(rng.bytes(3 * N_BYTES[ps] * keys[si]), dtype=np.uint8).reshape(keys[si], -1).copy()
    return {"params": which, "keys": kidx, "pool_idx": pool_idx, "arrival_ns": arrival_ns,
            "pool_msgs": pool_msgs, "pool_lens": pool_lens, "seeds": seeds, "rate": rate, "seconds": seconds}


def config(index, params=None):
    """The five workload recipes (sizes of the configurations the signer is
    specified on); ``params`` picks the set for the two-set / mixed recipes.

    0: 128f, 1 key, 64 x 32 B messages (every signature checked by the oracle)
    1: 128f, 16 keys, 16384 x 32 B, key i mod 16 (oracle on a seeded 256 subset)
    2: 192f or 256f, 16 keys, 8192 messages of U{32..1024} bytes
    3/4: mixed and serving recipes are built by their own modules.
    """
    seed = BASE_SEED + index
    if index == 0:
        return make("128f", 64, 1, 32, seed, "128f-1key-64x32B")
    if index == 1:
        return make("128f", 16384, 16, 32, seed, "128f-16keys-16384x32B", subset=256)
    if index == 2:
        ps = params or "192f"
        return make(ps, 8192, 16, ("uniform", 32, 1024), seed + (0 if ps == "192f" else 100),
                    "%s-16keys-8192xU[32,1024]B" % ps, subset=32)
    raise ValueError("config %d has no plain batch recipe" % index)
