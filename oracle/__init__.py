"""CPU oracle (test infrastructure only): see oracle.py and spc_oracle.c."""
