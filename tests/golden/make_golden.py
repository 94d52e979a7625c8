"""Write oracle_regression.json from the FP64 oracle (calls only oracle/ and the
seeded scene generators)."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2510_25660_gb300 import scenes  # noqa: E402


def compute():
    out = {}
    sc = scenes.cornell_box()
    osc = O.OracleScene(sc)
    r = osc.render(64, 64, 256, 3.5, 0.01, spp=4, seed=25660, max_depth=4, crop=(30, 34, 30, 32))
    out["cornell_steady_crop_30_34_30_32_spp4"] = r["steady"].reshape(-1).tolist()
    f = r["film"][0, 0, :, 0]
    nz = np.nonzero(f)[0]
    out["cornell_film_px30_30_bins"] = nz.tolist()
    out["cornell_film_px30_30_values_r"] = f[nz].tolist()
    pl = scenes.point_light_plane()
    r = O.OracleScene(pl).render(8, 8, 600, 0.0, 0.01, spp=1, seed=7, max_depth=2, flags=O.PIXEL_CENTER)
    out["plane_steady_r"] = r["steady"][..., 0].reshape(-1).tolist()
    out["plane_peak_bins"] = r["film"][..., 0].argmax(2).reshape(-1).tolist()
    nl = scenes.nlos_scene()
    lasers = scenes.wall_grid(2, 2)
    r = O.OracleScene(nl).render_nlos(lasers, None, False, 4096, 0.0, 0.003, spp=64, seed=3)
    out["nlos_confocal_2x2_spp64_steady"] = r["steady"].tolist()
    return out


if __name__ == "__main__":
    json.dump(compute(), open(os.path.join(HERE, "oracle_regression.json"), "w"), indent=1)
    print("wrote oracle_regression.json")
