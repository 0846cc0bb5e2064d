"""CPU oracle of the CCWSIM best-match search (test infrastructure only)."""
