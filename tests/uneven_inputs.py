"""Seeded inputs of the 64-image uneven workload (96..320 pixels square,
C = 512), drawn in spawned worker processes.  Only the input generator is
imported here (no method arithmetic), so the workers stay light."""
from paper_2510_15602_gb300 import synth

WORKLOAD = "uneven64_c512"


def gen(idx):
    img = synth.make_image(WORKLOAD, idx)
    return img.X, img.mask, img.r


def draw_all(n, workers=8):
    import multiprocessing as mp
    import os
    w = max(1, min(n, (os.cpu_count() or 2) - 1, workers))
    if w == 1:
        return [gen(i) for i in range(n)]
    with mp.get_context("spawn").Pool(w) as pool:
        return pool.map(gen, list(range(n)))
