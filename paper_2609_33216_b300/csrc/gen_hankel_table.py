"""Write hankel_table.inc: Taylor coefficients of J0, Y0, J1, Y1 about the centres
x_m = 4.5 + m (m from 0 to 15) of the unit intervals covering (4, 20), degree 15, for
the mid-range branch of hankel01() (hankel.cuh).  Computed with mpmath at 40 digits and
rounded once to FP64; on |x - x_m| <= 1/2 the dropped terms are below 1e-18 (the
derivatives of J_n and Y_n are bounded there by about 1), and Horner evaluation in FP64
stays within about 2e-16 of H_0 and H_1 relative.

    python paper_2609_33216_b300/csrc/gen_hankel_table.py
"""

import os

import mpmath as mp

mp.mp.dps = 40
DEG = 15
FUNCS = [lambda x: mp.besselj(0, x), lambda x: mp.bessely(0, x),
         lambda x: mp.besselj(1, x), lambda x: mp.bessely(1, x)]


def main():
    lines = ["// Generated by gen_hankel_table.py: Taylor coefficients (degree 15) of J0, Y0, J1, Y1",
             "// about x_m (4.5 + m for m from 0 to 15); kHankelMid[m][f][n] multiplies (x - x_m)^n.",
             "static __device__ const double kHankelMid[16][4][16] = {"]
    for m in range(16):
        c = mp.mpf(4.5) + m
        lines.append("  {")
        for f in FUNCS:
            coef = mp.taylor(f, c, DEG)
            lines.append("    {" + ", ".join(repr(float(v)) for v in coef) + "},")
        lines.append("  },")
    lines.append("};")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hankel_table.inc")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print(out)


if __name__ == "__main__":
    main()
