"""FP64 CPU oracle of the Hessian-free ray-Born update (test infrastructure only)."""
