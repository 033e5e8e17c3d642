"""CPU oracle for RANLUX++ (test infrastructure only; see ranluxpp.py and swb.c)."""
