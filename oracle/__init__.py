"""FP64 CPU oracle (test infrastructure only; see hps_oracle)."""
