"""CPU oracle for the MRCM / MPM-2P hot path (test infrastructure only).

Plain, slow, FP64 NumPy/SciPy statement of what the CUDA path computes. Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline``
leg and ``--impl reference`` arm) may import it. The product package never
does, and shares no code with it.
"""
