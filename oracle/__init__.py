"""FP64 CPU oracle of the GR PIC step (test infrastructure only; see oracle.py)."""
