"""FP64 CPU oracle for the split-operator step (test infrastructure only)."""
