"""Small seeded worlds shared by the tests (sizes the oracle finishes in seconds)."""
from dataclasses import replace

import scenegen as sg

# one 32^3 chunk, filled terrain + solid floating boxes, 2 LODs
TINY32 = replace(sg.SINGLE_128, name="tiny32", seed=11, wx=32, wy=32, wz=32, chunk=32, n_lods=2,
                 period0=16, h_min=4, h_max=20, n_boxes=4, box_min=2, box_max=8)

# 4x3x2 chunks of 16^3 (64x48x32), crust terrain + hollow blocks, 2 LODs
MULTI16 = replace(sg.CITY_4096, name="multi16", seed=12, wx=64, wy=48, wz=32, chunk=16, n_lods=2,
                  period0=32, h_min=6, h_max=22, crust=3, n_boxes=6, box_min=3, box_max=9)

# 3x3x2 chunks of 32^3 (96x96x64), 3 LODs, crust + hollow blocks
MULTI32 = replace(sg.CITY_4096, name="multi32", seed=13, wx=96, wy=96, wz=64, chunk=32, n_lods=3,
                  period0=64, h_min=10, h_max=40, crust=4, n_boxes=12, box_min=3, box_max=12)

# 4x4x2 chunks of 64^3 (256x256x128), 4 LODs: several tiles per ray, ragged image sizes
MED64 = replace(sg.CITY_4096, name="med64", seed=14, wx=256, wy=256, wz=128, chunk=64, n_lods=4,
                period0=128, h_min=20, h_max=90, crust=6, n_boxes=60, box_min=4, box_max=24)

# MED64 with layered (coherent) materials: the colour-block workload
MED64_LAYERED = replace(MED64, name="med64_layered", mat_mode=1)
