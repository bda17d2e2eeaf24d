"""FP64 CPU oracle for the APC solver: test infrastructure only (see apc_oracle)."""
