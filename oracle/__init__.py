"""CPU FP64 oracle (test infrastructure only; see bt_oracle.py)."""
