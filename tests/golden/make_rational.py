"""Writes rational_coeffs.json: minimax coefficients of x^-1/4 (pseudofermion
action, Eq. jkjk) and x^1/8 (heatbath, Eq. hbeq) computed by the oracle only.

The interval of each case is the free spectrum [min, max] of M0^dagger M0 on the
lattice (Sec. 7.4: the g = 0 operator sets the range at weak coupling), widened
by a factor 2 on both sides for the interaction.

    python tests/golden/make_rational.py
"""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import momentum, rational  # noqa: E402

CASES = [
    # name, dims, m, degree
    ("L4_m0.5_d8", (4, 4, 4, 4), 0.5, 8),
    ("L8_m0.5_d10", (8, 8, 8, 8), 0.5, 10),
    ("L16_m0.1_d20", (16, 16, 16, 16), 0.1, 20),
]


def main():
    out = {}
    for name, dims, m, d in CASES:
        den = momentum.free_norm(dims, m)
        lo, hi = 0.5 * float(den.min()), 2.0 * float(den.max())
        entry = {"dims": list(dims), "m": m, "lo": lo, "hi": hi}
        for key, gamma in (("action", -0.25), ("heatbath", 0.125)):
            c = rational.minimax(gamma, lo, hi, d)
            entry[key] = {"gamma": gamma, "d": d, "a0": c["a0"], "alpha": list(c["alpha"]),
                          "beta": list(c["beta"]), "err": c["err"]}
            print(name, key, "err", c["err"], flush=True)
        out[name] = entry
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rational_coeffs.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
