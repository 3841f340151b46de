"""FP64 CPU oracle for the mode-space Langevin step (test infrastructure only)."""
