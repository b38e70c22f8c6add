"""Plain FP64 CPU oracle of the FSM surface generator -- test infrastructure.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import it. The product library never does.
"""
