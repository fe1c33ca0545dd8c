"""Plain FP64 CPU oracle of the hybrid-dimensional VAG scheme.

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  The product path never imports it.
"""
