"""Test-infrastructure oracle for the Ising-film sweep (see oracle.py)."""
