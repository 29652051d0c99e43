"""Angle quadrature (input data of the formal solution).

The paper adopts a 12-ray set of Jaume-Bestard et al. (Sect. 2.5) whose values it does not print.
The stand-in is the 24-direction level-symmetric S4 set: in each octant the three permutations of
(mu1, mu1, mu2), mu1 = 0.3500212, mu2 = sqrt(1 - 2 mu1^2) = 0.8688903, every weight 1/24.

Ordering: directions 0..11 travel upward (mu_z > 0), 12..23 downward; direction d + 12 is the
mirror of direction d in z.  Within a hemisphere the octants run (+,+), (-,+), (-,-), (+,-) in
(mu_x, mu_y) sign, each with the permutations (mu2,mu1,mu1), (mu1,mu2,mu1), (mu1,mu1,mu2).
"""
import numpy as np

MU1 = 0.3500212


def s4_quadrature():
    mu1 = MU1
    mu2 = np.sqrt(1.0 - 2.0 * mu1 * mu1)
    perms = [(mu2, mu1, mu1), (mu1, mu2, mu1), (mu1, mu1, mu2)]
    octs = [(1, 1), (-1, 1), (-1, -1), (1, -1)]
    dirs = []
    for sz in (1.0, -1.0):
        for sx, sy in octs:
            for a, b, c in perms:
                dirs.append((sx * a, sy * b, sz * c))
    dirs = np.array(dirs, dtype=np.float64)
    w = np.full(len(dirs), 1.0 / len(dirs))
    return dirs, w
