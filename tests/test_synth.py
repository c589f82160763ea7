"""The seeded generators: determinism, thread-count independence, recipe."""
import hashlib
import os
import subprocess
import sys

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _digest(threads: int) -> str:
    code = ("import synth, hashlib; v = synth.porous((33, 40, 29), 77)[0]; "
            "s = synth.spheres((20, 21, 22), 9, 78); "
            "print(hashlib.sha256(v.tobytes() + s.tobytes()).hexdigest())")
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    return subprocess.check_output([sys.executable, "-c", code], cwd=ROOT, env=env).decode().strip()


def test_thread_count_independent():
    assert _digest(1) == _digest(5)


def test_same_seed_same_volume():
    a = synth.porous(24, 5)[0]
    b = synth.porous(24, 5)[0]
    c = synth.porous(24, 6)[0]
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_porous_recipe():
    v, por = synth.porous(96, synth.SEED_BASE + 2)
    assert v.dtype == np.uint16
    assert 0.25 < por < 0.40          # 35% target, minus balls clipped at the faces
    lo = v[v < 7500].astype(np.float64)
    hi = v[v >= 7500].astype(np.float64)
    assert abs(lo.mean() - 3000) < 40 and abs(hi.mean() - 12000) < 60
    assert abs(lo.std() - np.sqrt(3000)) < 5 and abs(hi.std() - np.sqrt(12000)) < 8
    # pore count N = ceil(-ln(0.65) V / E[4/3 pi r^3]) with E[r^3] = (30^4 - 2^4) / 112
    er3 = (30**4 - 2**4) / 112.0
    assert synth.porous_count(1024) == int(np.ceil(-np.log(0.65) * 1024**3 / (4 / 3 * np.pi * er3)))


def test_spheres_recipe():
    v = synth.spheres(64, 10, 3)
    assert v.dtype == np.float32
    bg = v[v < 0.6]
    assert abs(bg.mean() - 0.2) < 0.01 and abs(bg.std() - 0.05) < 0.005


def test_kd_bricks_partition():
    b = synth.kd_bricks(512, 37, synth.SEED_BASE + 4)
    assert b.shape == (37, 6)
    sides = b[:, 3:] - b[:, :3]
    assert sides.min() >= 64 and sides.max() <= 256 and (sides % 16 == 0).all()
    cover = np.zeros((32, 32, 32), np.int32)     # 16-voxel cells
    for z0, y0, x0, z1, y1, x1 in b // 16:
        cover[z0:z1, y0:y1, x0:x1] += 1
    assert (cover == 1).all()
