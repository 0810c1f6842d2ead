"""Writes the stored expected values under tests/golden/ from the oracle alone.

exp_kernel_closed_form.json: eigenvalues of sigma^2 exp(-|x-x'|/ell), sigma = ell = 1, on [0, 1]
(the analytic solution cited in the Remark of Sec. 6.1, via oracle.closed_form) and the
products that form the spectrum of the separable kernel on the unit square.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import closed_form  # noqa: E402


def main():
    out = {
        "source": "oracle.closed_form (analytic 1D exponential-kernel spectrum, Remark in Sec. 6.1)",
        "unit_interval_ell1": [float(v) for v in closed_form.exp_kernel_1d(20, 1.0)],
        "unit_square_ell1": [float(v) for v in closed_form.exp_separable_box(20, 1.0, [1.0, 1.0])],
    }
    with open(os.path.join(HERE, "exp_kernel_closed_form.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
