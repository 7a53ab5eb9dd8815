"""FP64 CPU oracle of the functional-map hot path (test infrastructure only)."""
