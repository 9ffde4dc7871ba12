"""FP64 CPU oracle (test infrastructure only; see csc_oracle.py)."""
