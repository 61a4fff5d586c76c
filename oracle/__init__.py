"""CPU oracle for the 2-D DWT by lifting (test infrastructure only; see oracle.py)."""
