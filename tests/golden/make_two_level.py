"""Writes two_level.txt: a two-level subspace response worked by hand.

Setting: eps = (-0.1, +0.1) Ha, kT = 0.1 Ha, g = 2, N_e = 2.  By symmetry of
the two levels about 0, g (f_1 + f_2) = 2 holds at mu = 0, so x = (-1, +1).
With the Fermi function of Eq. kseqcont:
  f_1 = 1/(1 + e^-1), f_2 = 1/(1 + e^+1)
  L_12 = (f_1 - f_2)/(eps_1 - eps_2)            (divided difference)
  L_ii = -f_i (1 - f_i)/kT                      (df/deps)
For the projected perturbation X = [[0.3, 0.2], [0.2, -0.1]]:
  mu' = (L_11 X_11 + L_22 X_22)/(L_11 + L_22)   (Tr Gamma-breve^(1) = 0, §II.C)
  Gamma-breve^(1) = L o (X - mu' I)            (Eq. subspaceDensityMatResponse)
Evaluated here with mpmath at 50 digits; this script uses no project code.
"""
import os

import mpmath as mp

mp.mp.dps = 50
kT = mp.mpf("0.1")
e1, e2 = mp.mpf("-0.1"), mp.mpf("0.1")
f1 = 1 / (1 + mp.e ** (-1))
f2 = 1 / (1 + mp.e ** (1))
L12 = (f1 - f2) / (e1 - e2)
L11 = -f1 * (1 - f1) / kT
L22 = -f2 * (1 - f2) / kT
X = [[mp.mpf("0.3"), mp.mpf("0.2")], [mp.mpf("0.2"), mp.mpf("-0.1")]]
mup = (L11 * X[0][0] + L22 * X[1][1]) / (L11 + L22)
Xp = [[L11 * (X[0][0] - mup), L12 * X[0][1]], [L12 * X[1][0], L22 * (X[1][1] - mup)]]
rows = [("eps", [e1, e2]), ("kT", [kT]), ("mu", [mp.mpf(0)]), ("occ", [f1, f2]),
        ("L", [L11, L12, L12, L22]), ("X", [X[0][0], X[0][1], X[1][0], X[1][1]]),
        ("dmu", [mup]), ("Xp", [Xp[0][0], Xp[0][1], Xp[1][0], Xp[1][1]])]
here = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(here, "two_level.txt"), "w") as fh:
    fh.write("# Two-level subspace response worked by hand (see make_two_level.py).\n")
    fh.write("# Source: Fermi function of Eq. kseqcont; Loewner scaling and traceless mu'\n")
    fh.write("# of Eq. subspaceDensityMatResponse (arXiv 2211.07894 §II.C).  g = 2, N_e = 2.\n")
    for name, vals in rows:
        fh.write(name + " " + " ".join(mp.nstr(v, 25) for v in vals) + "\n")
