"""FP64 CPU oracle for TASER -- test infrastructure only (see taser_oracle.py)."""
