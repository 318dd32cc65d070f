"""FP64 CPU oracle (test infrastructure; see cpals_oracle.py)."""
