"""CPU oracle for the position-based articulated dynamics path (test infrastructure only)."""
