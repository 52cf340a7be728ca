"""FP64 CPU oracle (test infrastructure only; see oracle/misr_oracle.h)."""
