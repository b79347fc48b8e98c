"""FP64 CPU oracle (test infrastructure only; see cgh_oracle.py)."""
