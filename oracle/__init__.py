"""FP64 CPU oracle of the GMCP contact pass (test infrastructure only)."""
