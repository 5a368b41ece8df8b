"""CPU oracle package (test infrastructure only; see cafs_oracle)."""
