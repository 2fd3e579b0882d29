"""FP64 CPU oracle of the iterative sampling-and-merging POD.

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline legs of bench.py, never by the library's product path.
"""
