"""Plain CPU oracle of the DABS hot path (test infrastructure only)."""
