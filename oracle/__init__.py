"""Plain FP64 CPU oracle (test infrastructure only; see pttk_oracle)."""
