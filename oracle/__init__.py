"""CPU oracle of the hybrid symplectic step — TEST INFRASTRUCTURE ONLY.

Plain FP64 C restatement of the method (see nbref.c for the passages it
follows). Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline
and reference legs may import it. It shares no code with the CUDA library.
"""
