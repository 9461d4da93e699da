"""FP64 CPU oracle of the mechanism hot path (test infrastructure only)."""
