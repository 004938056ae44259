"""FP64 CPU oracle of the Stein-MAP-Seq hot path (test infrastructure only)."""
