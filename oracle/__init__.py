"""Plain FP64 CPU oracle of the CF-DQMC sweep.

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import, call, link or execute anything in
this package.  It shares no code with the CUDA path.
"""
