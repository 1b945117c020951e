"""Write the oracle regression fixtures in this folder.

The paper prints no worked numeric example (its models and data live in an
external repository), so the fixtures here are FP64 oracle outputs on seeded
synthetic inputs.  This script calls only the oracle and the input generators;
rerun it (python tests/golden/make_golden.py) only when the oracle's arithmetic
changes for a reason the paper justifies.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2603_01234_gb300 import inputs  # noqa: E402


def cases():
    yield "water64_periodic", inputs.random_model(seed=1), inputs.water_box(64, seed=2)
    m2 = inputs.random_model(n_types=2, hidden=8, rc_radial=6.0, rc_angular=4.0, seed=3)
    yield "cluster24_two_types", m2, inputs.random_cluster(24, seed=4, box_len=9.0, min_dist=1.2, n_types=2)
    # with the four-body (l = 2) and five-body (l = 1) descriptors
    m3 = inputs.random_model(n_types=2, hidden=8, rc_radial=6.0, rc_angular=4.5, seed=5, l_max_4b=2, l_max_5b=1)
    yield "cluster20_many_body", m3, inputs.random_cluster(20, seed=6, box_len=8.0, min_dist=1.3, n_types=2)


def main():
    for name, m, s in cases():
        r = oracle.compute(m, s)
        out = {
            "case": name,
            "how": "oracle.compute on paper_2603_01234_gb300.inputs generators (see make_golden.py)",
            "energy": r.energy,
            "virial_total": r.virial_total.tolist(),
            "site_energy_first8": r.site_energy[:8].tolist(),
            "force_first8": r.force[:, :8].tolist(),
            "virial_first4": r.virial[:, :4].tolist(),
        }
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, r.energy)


if __name__ == "__main__":
    main()
