"""Plain FP64 CPU oracle of the MBHB Whittle log-likelihood (test infrastructure only)."""
