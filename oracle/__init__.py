"""FP64 CPU oracle for the RW-MI-DELBM fluid-solute step (test infrastructure only)."""
