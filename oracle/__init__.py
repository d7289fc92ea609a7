"""FP64 CPU oracle of the DG-LES hot path (test infrastructure only).

Only tests/, the smoke check in __graft_entry__ and the CPU-baseline leg of
bench.py may import this package; the product never does.
"""
