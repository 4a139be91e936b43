"""Writes the stored fingerprints under tests/golden/.

scenegen_hashes.json: SHA-256 of small generated regions (input data; must be
identical on every platform).  oracle_small.json: SHA-256 of oracle results on
small worlds, so that a build of the oracle on another platform is checked
against this one.  Calls only scenegen and oracle."""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle as orc  # noqa: E402
import scenegen as sg  # noqa: E402
from worlds import MED64, MED64_LAYERED, MULTI32, TINY32  # noqa: E402


def sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def region_fingerprints():
    out = {}
    for spec, regions in [(sg.SINGLE_128, [(0, 0, 0, 128, 128, 128)]),
                          (sg.CITY_4096, [(1024, 2048, 512, 64, 64, 512), (3000, 100, 700, 64, 64, 256)]),
                          (sg.OPEN_65536, [(40000, 12000, 0, 64, 64, 1024)]),
                          (sg.CITY_4096_LAYERED, [(1024, 2048, 512, 64, 64, 512)])]:
        w = sg.World(spec)
        for r in regions:
            d = w.dense(*r)
            zs, ys, xs = np.nonzero(d)
            xyz = np.stack([xs + r[0], ys + r[1], zs + r[2]], 1)
            out[f"{spec.name}:{r}"] = {"occ": sha(d), "mat": sha(w.materials(xyz)), "solid": int(d.sum())}
        out[f"{spec.name}:boxes"] = sha(np.array(w.boxes(), np.int64))
    return out


def oracle_fingerprints():
    out = {}
    for spec, camf, tau, tol in [(TINY32, lambda w: sg.orbit_camera(TINY32, 5, 40, 30), 1.0, None),
                                 (MULTI32, lambda w: sg.ground_camera(w, 4, 32, 20, z_lo=4, z_hi=20), 1.0, None),
                                 (MED64, lambda w: sg.ground_camera(w, 4, 64, 36, z_lo=4, z_hi=40), 4.0, None),
                                 (MED64_LAYERED, lambda w: sg.ground_camera(w, 4, 64, 36, z_lo=4, z_hi=40), 4.0,
                                  0.05)]:
        w = sg.World(spec)
        S = orc.OracleScene(w, color_tol=tol)
        cam = camf(w)
        sel = S.select(cam, tau)
        r = S.cast(cam, sel)
        fields = np.stack([r[k] for k in ("x", "y", "z", "lod", "mat", "normal", "hit", "amb")], 1)
        out[spec.name + ("" if tol is None else f"@{tol}")] = {"sel": sha(sel), "fields": sha(fields.astype(np.int32)),
                          "dist": sha(np.where(r["hit"] == 1, r["dist"], 0.0)),
                          "visits": sha(np.stack([r["v_int"], r["v_leaf"], r["resolve_bytes"]], 1))}
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "scenegen_hashes.json"), "w") as f:
        json.dump(region_fingerprints(), f, indent=1, sort_keys=True)
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(oracle_fingerprints(), f, indent=1, sort_keys=True)
    print("written")
