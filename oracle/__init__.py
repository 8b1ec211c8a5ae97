"""CPU FP64 oracle (test infrastructure only; see kd_oracle's header)."""
