"""CPU oracle of the FVLBM time step (test infrastructure; see oracle/fvlbm_oracle.c)."""
