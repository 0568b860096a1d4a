"""GB300-native batched SPHINCS+-SHA2-{128f,192f,256f}-simple signer.

The signer itself is the C-ABI library ``libhs.so`` built from ``csrc/`` (see
``include/hs.h``); :mod:`paper_2512_23969_gb300.hs` is its thin Python binding
and :mod:`paper_2512_23969_gb300.inputs` holds the seeded workload generators.
Importing this package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""

PARAM_SETS = ("128f", "192f", "256f", "toy")
