"""The check build (the library compiled with -DROI_CHECK: index checks on every ray-sample
column and every staged gather bin of the hot kernels) over the paths the parity tests
cover: single-launch SIRT and CP solves, one launch per operator, batches solved by single
blocks and by teams with whole-staged and band-streamed images, served requests, and the
filtered sinograms on the tensor cores (first rows of the sinogram tiles).  No
index may leave its range, and every result equals the product build's bit for bit (the
checks only read the indices)."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import hashlib, json
import numpy as np
import torch
import paper_1604_02292_gb300 as R
from paper_1604_02292_gb300 import synth, workloads as WL

res = {}
w = WL.WORKLOADS["roi_sirt_128"]
rr = R.RoiRecon(*w.geometry())
rr.set_sinogram(torch.from_numpy(WL.sinogram(w, 0)).cuda())
rr.fbp()
region = (64.0, 60.0, 16.0, 8.0)
res["sirt"] = rr.solve_local(region, R.ROI_SIRT_NONNEG, iters=20)[0]
res["cp"] = rr.solve_local(region, R.ROI_TV_CP, iters=20, lam=0.02)[0]
rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, 0)
res["cp_ops"] = rr.solve_local(region, R.ROI_TV_CP, iters=10, lam=0.02)[0]
res["sirt_ops"] = rr.solve_local((10.0, 10.0, 20.0, 10.0), R.ROI_SIRT_NONNEG, iters=10)[0]
rr.set_option(R.ROI_OPT_SINGLE_LAUNCH, 1)

N, NA, ND = 400, 90, 400
ph = synth.random_phantom(N, 12, texture=False, seed=5)
p = synth.analytic_sinogram(ph, NA, ND).astype(np.float32)
big = R.RoiRecon(N, NA, ND)
big.set_sinogram(torch.from_numpy(p).cuda())
big.fbp()
regions = [(200.0, 200.0, 100.0, 50.0), (100.0, 120.0, 20.0, 10.0), (300.0, 250.0, 45.0, 22.0),
           (380.0, 20.0, 30.0, 15.0)]
params = [dict(reg=R.ROI_SIRT_NONNEG, iters=6), dict(reg=R.ROI_TV_CP, iters=6, lam=0.02),
          dict(reg=R.ROI_SIRT_NONNEG, iters=6, weighting=1), dict(reg=R.ROI_TV_CP, iters=6, lam=0.05)]
outs, _ = big.solve_batch(regions, params)  # few regions: teams of blocks
for k, o in enumerate(outs):
    res[f"team{k}"] = o
many = [(40.0 + 4.0 * (k % 80), 60.0 + 3.0 * (k // 2 % 90), 12.0 + (k % 5), 6.0) for k in range(84)]
outs, _ = big.solve_batch(many + regions, [dict(reg=R.ROI_TV_CP, iters=3, lam=0.02)] * (len(many) + len(regions)))
for k, o in enumerate(outs):
    res[f"single{k}"] = o
big.sync()
rng = np.random.default_rng(9)
fu = torch.from_numpy(rng.standard_normal((40, NA, 2 * ND - 1)).astype(np.float32)).cuda()
fp = torch.from_numpy(rng.standard_normal((NA, ND)).astype(np.float32)).cuda()
res["filter_conv"] = big.filter_conv(fu, fp)  # tensor cores (Toeplitz tiles of the sinogram rows)
with R.Server(team_blocks=8, teams=4, large_side=200) as s:
    s.add(big)
    ids = {s.submit(0, r, prm): k for k, (r, prm) in enumerate(zip(regions, params))}
    s.drain(300000.0)
    for c in s.poll():
        assert c["status"] == R.ROI_OK
        res[f"served{ids[c['id']]}"] = s.take(c["id"], (c["box"][3], c["box"][2]))
torch.cuda.synchronize()
count, site, index = R.roi_recon_check_report()
out = {"count": count, "site": site, "index": index, "lib": R.lib()._name}
out["hashes"] = {k: hashlib.sha256(np.ascontiguousarray(v.cpu().numpy() if torch.is_tensor(v) else v).tobytes()).hexdigest()
                 for k, v in res.items()}
print(json.dumps(out))
"""


def _run(check):
    env = dict(os.environ)
    env.pop("ROI_RECON_CHECK", None)
    if check:
        env["ROI_RECON_CHECK"] = "1"
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_check_build_finds_no_out_of_range_index_and_matches_the_product_build():
    chk = _run(True)
    assert chk["lib"].endswith("libroi_recon_check.so")
    assert chk["count"] == 0, chk
    prod = _run(False)
    assert prod["lib"].endswith("libroi_recon.so")
    assert prod["count"] == 0
    assert chk["hashes"] == prod["hashes"]
