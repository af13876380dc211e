"""Writes static_cannon_q4.txt: Eq. 2 of the paper (round r of output tile
(i, j) multiplies A_{i r'} B_{r' j}, r' = r + i + j, taken modulo q) written
out for q = 4.  Uses nothing but the equation."""
import os

q = 4
lines = ["# Static-Cannon rounds of the trident outer algorithm (Alg. 1, Eq. 2),",
         "# read with the stagger taken modulo q (r' = (r + i + j) mod q), q = 4.",
         "# Each line: i j r r'  -- output tile (i, j), round r multiplies A_{i r'} B_{r' j}.",
         "# Evaluated by hand from Eq. 2; every (i, j) meets every r' exactly once."]
for i in range(q):
    for j in range(q):
        for r in range(q):
            lines.append(f"{i} {j} {r} {(r + i + j) % q}")
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "static_cannon_q4.txt"), "w") as f:
    f.write("\n".join(lines) + "\n")
