"""FP64 CPU oracle of the short-range MD hot path (test infrastructure only)."""
