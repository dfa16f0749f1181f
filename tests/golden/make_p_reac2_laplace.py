"""Writes p_reac2_laplace.txt: 2D reaction probabilities p_reac = (g_ref - g_rad)/(g_ref - g_abs)
(Eq. psurv_radII) from the exact Laplace-domain boundary terms of Section 4.2 (Eqs. absPert,
refPert, radPert; a = D = 1), each difference inverted as ONE transform by Talbot's method at 30
digits (mpmath), so that nothing cancels after the inversion.  Independent of the oracle; run
``python tests/golden/make_p_reac2_laplace.py`` to regenerate (about two minutes)."""
import os

import mpmath as mp

POINTS = [  # R, R0, tau, h
    (2.5, 1.8, 0.8, 0.3), (3.0, 1.2, 0.8, 0.00796), (1.5, 1.02, 0.2, 0.3), (4.0, 3.0, 0.8, 0.00796),
    (1.2, 1.1, 0.08, 2.0), (5.0, 4.5, 0.8, 0.00796),
]


def difference(R, R0, tau, h, first, second):
    def F(p):
        q = mp.sqrt(p)
        kk = mp.besselk(0, q * R0) * mp.besselk(0, q * R)
        quot = {"abs": -mp.besseli(0, q) / mp.besselk(0, q),
                "ref": mp.besseli(1, q) / mp.besselk(1, q),
                "rad": (mp.besseli(1, q) - h / q * mp.besseli(0, q)) / (mp.besselk(1, q) + h / q * mp.besselk(0, q))}
        return (quot[first] - quot[second]) * kk / (2 * mp.pi)
    return mp.invertlaplace(F, tau, method="talbot")


def main():
    mp.mp.dps = 30
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "p_reac2_laplace.txt")
    with open(out, "w") as f:
        f.write("# 2D p_reac (Eq. psurv_radII) from Talbot inversions (30 digits) of the Laplace-domain\n")
        f.write("# differences g_ref - g_rad and g_ref - g_abs (Section 4.2); written by make_p_reac2_laplace.py\n")
        f.write("# columns: R R0 tau h p_reac\n")
        for R, R0, tau, h in POINTS:
            p = difference(R, R0, tau, h, "ref", "rad") / difference(R, R0, tau, h, "ref", "abs")
            f.write(f"{R!r} {R0!r} {tau!r} {h!r} {mp.nstr(p, 20)}\n")


if __name__ == "__main__":
    main()
