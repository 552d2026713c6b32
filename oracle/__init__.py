"""FP64 CPU oracle of the ReFusion per-frame path -- test infrastructure only.

Importable by the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg; never by the product package.
"""
