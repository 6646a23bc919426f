"""Writes table1_complexity.txt from the Table I formulas (Sec. V-B) via the oracle."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import taser_oracle as O  # noqa: E402

lines = ["# Table I (Sec. V-B): real-valued multiplications of TASER for t_max iterations,",
         "# evaluated from the printed formulas:",
         "#   BPSK  t_max (U^3/3 + 5U^2/2 + 37U/6 + 4)",
         "#   QPSK  t_max (8U^3/3 + 10U^2 + 37U/3 + 4)",
         "# columns: constellation U t_max multiplications"]
for const in ("bpsk", "qpsk"):
    for U in (1, 4, 8, 16, 32):
        for t in (1, 20):
            v = O.table1_mults(const, U, t)
            lines.append(f"{const} {U} {t} {int(round(v))}")
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "table1_complexity.txt"), "w") as f:
    f.write("\n".join(lines) + "\n")
