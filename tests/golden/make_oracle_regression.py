"""Writes oracle_regression.json: outputs of the FP64 oracle on two small seeded systems.

These values are the oracle's own, not the paper's: they pin nothing about the method (the
checks in test_oracle_pins.py do that) but make any later change of the oracle's arithmetic
visible, since test_oracle_regression.py compares the oracle with them.  Only oracle/ and the
seeded input generators are called.

    python tests/golden/make_oracle_regression.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))

import dpsynth  # noqa: E402
import oracle  # noqa: E402

CASES = {
    "water_192_seed5": ("water_config", "water_box", 5),
    "copper_500_seed6": ("copper_config", "copper_fcc", 6),
}
SAMPLE_ATOMS = (0, 1, 2, 37, 101, 150)


def system(case):
    cfg_name, box_name, seed = CASES[case]
    cfg = getattr(dpsynth, cfg_name)()
    if box_name == "copper_fcc":
        coord, typ, box = dpsynth.copper_fcc(seed, ncell=5)
    else:
        coord, typ, box = dpsynth.water_box(seed)
    return cfg, dpsynth.model_params(cfg, seed), coord, typ, box


def main():
    out = {}
    for case in CASES:
        cfg, params, coord, typ, box = system(case)
        E, Ei, F, W = oracle.Model(cfg, params).compute(coord, typ, box)
        out[case] = {"E": E, "Ei": {str(a): Ei[a] for a in SAMPLE_ATOMS},
                     "F": {str(a): list(F[a]) for a in SAMPLE_ATOMS}, "W": W.reshape(-1).tolist()}
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
