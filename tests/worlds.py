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

# one 32^3 chunk with no terrain, holding only cubes placed by hand (counter pins)
HAND32 = sg.WorldSpec("hand32", seed=31, wx=32, wy=32, wz=32, chunk=32, n_lods=1, octaves=1, period0=8,
                      h_min=0, h_max=0, crust=0, n_boxes=0, box_min=1, box_max=1, box_hollow=0)


def hand_world(voxels, n_lods=1, size=1):
    """HAND32 holding only the listed cubes (min corner, side `size`)."""
    return sg.World(replace(HAND32, n_lods=n_lods), boxes=[(x, y, z, size, size, size, 0) for x, y, z in voxels])


# Straight-down rays (origin (x, y, 40)) through hand-made scenes with their
# visits counted by hand: (voxels, cube side, LODs of the world, LOD cast,
# ray x, ray y, (interior visits, leaf-block visits, resolve bytes)).
HAND_CASES = [
    ([(9, 9, 9)], 2, 1, 0, 9.5, 10.5, (3, 1, 1)),
    ([(2, 2, 2), (26, 26, 26)], 2, 1, 0, 20.5, 4.5, (1, 0, 0)),
    ([(2, 2, 2), (26, 26, 26)], 2, 1, 0, 30.5, 4.5, (0, 0, 0)),
    ([(1, 1, 1), (20, 1, 1), (20, 20, 1), (17, 17, 17), (28, 28, 20), (25, 25, 25), (28, 28, 28)], 1, 1, 0,
     28.5, 28.5, (3, 1, 1 + 3 * 4 + 2 * 4 + 1 * 8)),
    ([(5, 5, 10), (5, 6, 3)], 1, 1, 0, 5.5, 6.5, (4, 2, 1)),
    ([(8, 8, 8)], 2, 2, 1, 8.5, 9.5, (2, 1, 1)),
]
