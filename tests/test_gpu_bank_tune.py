"""The filter-bank autotuner keeps the fastest of several plans (16 x 16 or
32 x 16 tiles, z chunks of 32..256, small radii in a second launch at two
CTAs per SM) on the assumption that every plan computes the same bits. Each
plan is pinned here in its own process (HP_BANK_TUNE=<cfg>,<zchunk>) on the
same seeded input, and the outputs must agree bit for bit with each other
and lie within the tolerance of the FP64 oracle."""
import hashlib
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_filter_close

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE = (72, 80, 96)
SIGMAS = (0.7, 2.0, 4.0)

CHILD = r"""
import hashlib, json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import paper_2511_11890_b300 as hp, synth
f = synth.porous_f16(tuple(json.loads(sys.argv[2])), 21)
bank = [(k, s) for s in json.loads(sys.argv[3]) for k in (hp.G, hp.GM, hp.LOG)]
bricks = [((0, 0, 0), (40, 48, 96)), ((0, 48, 0), (40, 80, 96)), ((40, 0, 0), (72, 80, 64)),
          ((40, 0, 64), (72, 80, 96))]
outs = hp.filterbank3d(torch.from_numpy(f).cuda(), bank, bricks=bricks, out_dtype=hp.HP_F32)
torch.cuda.synchronize()
arrs = [o.cpu().numpy() for o in outs]
np.save(sys.argv[4], np.stack(arrs))
print(json.dumps({"kernels": int(hp.stats()["bank_kernels"]),
                  "sha": hashlib.sha256(np.stack(arrs).tobytes()).hexdigest()}))
"""


@pytest.mark.parametrize("dummy", [0])
def test_every_tuning_plan_same_bits(tmp_path, dummy):
    pins = ["0,32", "0,256", "1,64", "1,256", "2,128", "2,256"]
    shas, kernels = {}, {}
    first = None
    for pin in pins:
        out = tmp_path / f"bank_{pin.replace(',', '_')}.npy"
        env = dict(os.environ, HP_BANK_TUNE=pin)
        res = subprocess.run([sys.executable, "-c", CHILD, ROOT, json.dumps(SHAPE), json.dumps(SIGMAS),
                              str(out)], env=env, capture_output=True, text=True, timeout=600)
        assert res.returncode == 0, res.stderr[-2000:]
        rec = json.loads(res.stdout.strip().splitlines()[-1])
        shas[pin], kernels[pin] = rec["sha"], rec["kernels"]
        if first is None:
            first = np.load(out)
    assert len(set(shas.values())) == 1, shas
    assert kernels["2,256"] == 2 and kernels["1,256"] == 1, kernels
    f = synth.porous_f16(SHAPE, 21)
    ref = oracle.filterbank3d(f, [(k, s) for s in SIGMAS for k in (oracle.G, oracle.GM, oracle.LOG)])
    for i, r in enumerate(ref):
        assert_filter_close(first[i], r, f"plan outputs, filter {i}")
