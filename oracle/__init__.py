"""FP64 CPU oracle for the exchange path (test infrastructure; see hfx_oracle)."""
