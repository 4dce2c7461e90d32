"""Serial FP64 CPU oracle of the method (test infrastructure only)."""
