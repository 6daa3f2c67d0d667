"""FP64 CPU oracle of the hybrid LBM / FENE-P step (test infrastructure only)."""
