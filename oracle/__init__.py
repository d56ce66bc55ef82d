"""FP64 CPU oracle of the RTT Monte Carlo hot path (test infrastructure only)."""
