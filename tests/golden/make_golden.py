"""Write the stored expected values of tests/golden/ from the CPU oracle's exact tools only.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact as E  # noqa: E402


def compute() -> dict:
    """Every stored value, computed afresh by oracle/exact.py."""
    b, d = E.schlogl_rates()
    bb, dd = E.birth_death_rates()
    return {
        "source": "oracle/exact.py (birth-death closed forms, truncated CME, uniformized futile-cycle CME); see each entry",
        "schlogl_mfpt_85_to_550_s": E.bd_mfpt(85, 550, b, d),
        "schlogl_mfpt_82_to_563_s": E.bd_mfpt(82, 563, b, d),
        "schlogl_p_ge_700_t5_from_82": float(E.bd_transient(b, d, 82, 5.0, 1000)[700:].sum()),
        "birth_death_mfpt_100_to_250": E.bd_mfpt(100, 250, bb, dd),
        "futile_p_s1_gt_90_t100": float(E.futile_s1_law(100.0)[91:].sum()),
        "epigenetic_mfpt_0_30_to_g1_ge_50_s": E.epigenetic_mfpt((0, 30), lambda u, v: u >= 50),
        "notes": {
            "schlogl_mfpt_82_to_563_s": "paper Sec. III.B.3 quotes approximately 5e4 s",
            "schlogl_p_ge_700_t5_from_82": "paper Sec. III.B.3 prints the CME value 1.148e-9",
            "futile_p_s1_gt_90_t100": "paper Sec. III.A prints the CME value 2.72e-18 (from S1 = S2 = 50)",
            "epigenetic_mfpt_0_30_to_g1_ge_50_s": "paper Sec. III.C prints 1.3e6 s (WE and brute-force MLE); source and target read as the g2-high state and the last g1 bin",
        },
    }


def main():
    out = compute()
    with open(os.path.join(HERE, "exact_values.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
