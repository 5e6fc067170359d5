"""FP64 CPU oracle of the TDSLDA step (test infrastructure only; see oracle.py)."""
