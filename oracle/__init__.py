"""CPU oracle of the coarse-grid solve (test infrastructure only; see cgs_oracle)."""
