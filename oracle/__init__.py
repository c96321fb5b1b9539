"""FP64 CPU oracle of the coupled LB + Oldroyd-B step (test infrastructure only)."""
