"""CPU oracle of the FRW + MicroWalk method (test infrastructure only; see oracle.py)."""
