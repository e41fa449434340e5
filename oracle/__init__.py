"""FP64 CPU oracle for projected EM in 2D SR-MRA.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg.  The CUDA product path never imports it.
"""
