"""FP64 CPU oracle of the fast-electron hybrid-PIC step (test infrastructure only)."""
