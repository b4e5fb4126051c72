"""Write tests/golden/kerr_end_points.json: the exact end points (cos theta,
phi at r_esc = 1.1 r_obs for escaping rays, at r_cap = 1.01 r_H for captured
ones) of the Kerr rays of oracle.first_integrals.KERR_END_POINT_RAYS, from the
quadratures of their first integrals (Carter's separation of Hamilton's
equations, Sec. 2.1, on the Kerr metric, Sec. 4.3). Calls only oracle/.

    python tests/golden/make_kerr_end_points.py
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle.first_integrals import KERR_END_POINT_RAYS, kerr_end_point  # noqa: E402

R_OBS = 1000.0


def rows():
    out = []
    for a, inc, esc, cap in KERR_END_POINT_RAYS:
        r_cap = 1.01 * (1.0 + math.sqrt(1.0 - a * a))
        for fate, pixels in (("escaped", esc), ("captured", cap)):
            for x, y in pixels:
                st = oracle.init_ray(a, R_OBS, inc, x, y)
                u, phi = kerr_end_point(a, 1.1 * R_OBS, st, r_cap=r_cap)
                out.append({"a": a, "incl_deg": inc, "x": x, "y": y, "fate": fate,
                            "cos_theta": u, "phi": phi})
    return out


if __name__ == "__main__":
    doc = {"source": "quadratures of the first integrals of Kerr null geodesics "
                     "(oracle/first_integrals.py), r_obs = 1000, r_esc = 1.1 r_obs, "
                     "r_cap = 1.01 r_H, written by tests/golden/make_kerr_end_points.py",
           "rays": rows()}
    with open(os.path.join(HERE, "kerr_end_points.json"), "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
