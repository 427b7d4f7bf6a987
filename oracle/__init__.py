"""CPU FP64 oracle (test infrastructure only; see fftls_oracle)."""
