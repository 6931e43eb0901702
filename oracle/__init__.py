"""CPU FP64 oracle (test infrastructure only; see sphere_oracle)."""
