"""CPU correctness oracle for the SPHINCS+ signer (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path under
``paper_2512_23969_gb300`` never imports it.
"""
