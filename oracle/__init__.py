"""CPU oracle for masked SpGEMM -- test infrastructure only (see oracle.c)."""
