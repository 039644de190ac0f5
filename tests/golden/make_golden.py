"""Writes tests/golden/mesh_counts.json from the oracle's grid mesher.

The unit-sphere h = 0.1 and three-shell h = 2 mm rows (5233 nodes / 25344
tets and 428185 nodes / 2447424 tets) agree with an independent count of the
Kuhn-grid rule made when the workloads were specified; the file pins the
mesher against later changes.  Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import zi_oracle as O  # noqa: E402

ROWS = [(0.1, [1.0]), (0.2, [1.0]), (0.05, [1.0]), (0.004, [0.080, 0.086, 0.092]),
        (0.002, [0.080, 0.086, 0.092])]

out = {"about": "grid Kuhn mesh counts (nodes n, tets m, boundary faces nb, tets per shell)",
       "rows": []}
for h, radii in ROWS:
    mesh = O.mesh_from_grid(h, radii)
    out["rows"].append(dict(h=h, radii=radii, n=int(mesh["nodes"].shape[0]),
                            m=int(mesh["tets"].shape[0]), nb=int(mesh["bfaces"].shape[0]),
                            labels=[int(x) for x in np.bincount(mesh["labels"], minlength=len(radii))]))
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "mesh_counts.json"), "w") as f:
    json.dump(out, f, indent=1)
print(json.dumps(out, indent=1))
