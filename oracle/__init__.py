"""FP64 CPU oracle of the projective-dynamics hot path.

Test infrastructure only: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline leg may import it; the CUDA library never does.
"""
