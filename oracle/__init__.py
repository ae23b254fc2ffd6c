"""CPU FP64 oracle (test infrastructure only; see fsi_oracle)."""
