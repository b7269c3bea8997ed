"""CPU oracle (test infrastructure only): see mlc_oracle.py."""
