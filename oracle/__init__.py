"""FP64 CPU oracle (test infrastructure only; see lbf_oracle's header)."""
