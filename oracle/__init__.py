"""FP64 CPU oracle of the IB-LB wetting time step (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py
may import this package.  It shares no code with paper_2503_20605_gb300.
"""
