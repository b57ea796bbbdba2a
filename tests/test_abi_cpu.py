"""CPU checks of the C-ABI library: it builds, loads, exports every declared symbol,
and its host-side ROI plan agrees with the oracle's box rule and with the rows of
W_L that the oracle finds non-zero.  No compute call needs a GPU here."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_1604_02292_gb300 as R
from paper_1604_02292_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "roi_recon.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(roi_(?:recon|server)_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    R.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", R._build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(\w+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    assert sorted(R.EXPORTS) == declared


@pytest.mark.parametrize("region", [
    (64.0, 64.0, 16.0, 8.0), (63.5, 20.0, 16.0, 8.0), (10.2, 120.7, 16.5, 0.0), (0.0, 0.0, 3.0, 1.0),
    (127.0, 64.0, 40.0, 20.0), (50.3, 77.9, 0.4, 0.0),
])
def test_plan_box_matches_oracle_rule(region):
    pl = R.plan(128, 64, 128, region)
    assert pl.box == oracle.roi_box(128, *region)
    assert pl.window_stride % 4 == 0 and pl.window_stride >= pl.window_max


@pytest.mark.parametrize("N,na,nd,region", [
    (128, 64, 128, (64.0, 64.0, 16.0, 8.0)),
    (128, 64, 128, (30.0, 90.0, 16.0, 8.0)),
    (96, 37, 150, (10.0, 50.0, 12.0, 4.0)),
    (64, 45, 48, (32.0, 32.0, 20.0, 10.0)),   # detector narrower than the grid
])
def test_plan_windows_cover_nonzero_rows(N, na, nd, region):
    """Every ray with a non-zero row of W_L (oracle row sums) lies in its angle's window,
    and the window is tight to within a couple of bins."""
    pl = R.plan(N, na, nd, region)
    g = oracle.Geometry(N, na, nd)
    rows, _ = oracle.rowcol_sums(g, pl.box)
    slack = []
    for a in range(na):
        nz = np.nonzero(rows[a] > 0)[0]
        lo, hi = pl.d0[a], pl.d0[a] + pl.width[a]
        assert pl.width[a] <= pl.window_max
        if nz.size:
            assert nz.min() >= lo and nz.max() < hi, (a, nz.min(), nz.max(), lo, hi)
            slack.append((nz.min() - lo) + (hi - 1 - nz.max()))
    assert max(slack) <= 2


def test_plan_rejects_bad_regions():
    for region in [(64.0, 64.0, 0.0, 8.0), (64.0, 64.0, -1.0, 0.0), (64.0, 64.0, 5.0, -1.0),
                   (500.0, 500.0, 5.0, 1.0), (float("nan"), 3.0, 4.0, 1.0)]:
        with pytest.raises(R.RoiError):
            R.plan(128, 64, 128, region)


def test_plan_rejects_bad_geometry():
    g = R.Geometry(0, 64, 128, None, R.ROI_F32)
    info = R.SolveInfo()
    assert R.roi_recon_plan(g, R.Region(1, 1, 1, 0), info, None, None) == R.ROI_EINVAL
    g = R.Geometry(128, 64, 128, None, 7)  # unknown storage type
    assert R.roi_recon_plan(g, R.Region(1, 1, 1, 0), info, None, None) == R.ROI_EINVAL
    g = R.Geometry(128, 64, 128, None, R.ROI_F32, 5)  # unknown image storage type
    assert R.roi_recon_plan(g, R.Region(1, 1, 1, 0), info, None, None) == R.ROI_EINVAL
    g = R.Geometry(128, 64, 128, None, R.ROI_BF16)  # 16-bit storage plans like float32
    assert R.roi_recon_plan(g, R.Region(64, 64, 8, 4), info, None, None) == R.ROI_OK
    g = R.Geometry(128, 64, 128, None, R.ROI_BF16, R.ROI_F16)  # any sinogram / image pair
    assert R.roi_recon_plan(g, R.Region(64, 64, 8, 4), info, None, None) == R.ROI_OK


def test_create_rejects_bad_geometry_without_touching_the_gpu():
    g = R.Geometry(-5, 64, 128, None, R.ROI_F32)
    s, h = R.roi_recon_create(g, 0)
    assert s == R.ROI_EINVAL and not h


def test_poisson_noise_model():
    """Largest expected count is I0 (at p = 0); the noisy data are unbiased to first order."""
    p = np.linspace(0.0, 50.0, 20001)
    n = synth.poisson_noise(p, 1e6, seed=1)
    assert abs(float(np.mean(n - p))) < 0.05
    assert np.array_equal(synth.poisson_noise(p, 0, seed=1), p)
    a = synth.poisson_noise(p, 1e3, seed=3)
    b = synth.poisson_noise(p, 1e3, seed=3)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", [R.ROI_F32, R.ROI_BF16])
@pytest.mark.parametrize("region", [(1000.0, 900.0, 16.0, 8.0), (1024.0, 1024.0, 256.0, 128.0),
                                    (5.0, 2040.0, 100.0, 50.0)])
def test_server_footprint_host_only(region, storage):
    """The server's per-request budget: three float windows [N_theta][stride], four float box
    arrays and the two padded projector images in the storage type (rows padded to 16 bytes),
    each rounded to 256 bytes; the result area is the box."""
    N, na, nd = 2048, 180, 2048
    dev, host, side = R.server_footprint(N, na, nd, region, storage)
    pl = R.plan(N, na, nd, region)
    w, h = pl.box[2], pl.box[3]
    assert side == max(w, h)
    r256 = lambda n: (n + 255) // 256 * 256
    es = 4 if storage == R.ROI_F32 else 2
    ld = lambda e: (e + 4 + 16 // es - 1) // (16 // es) * (16 // es)
    expect = 3 * r256(4 * na * pl.window_stride) + 4 * r256(4 * w * h) + r256(es * h * ld(w)) + r256(es * w * ld(h))
    assert dev == expect
    assert host == r256(4 * w * h)


def test_server_footprint_rejects_bad_input():
    with pytest.raises(R.RoiError):
        R.server_footprint(256, 96, 272, (900.0, 900.0, 5.0, 1.0))
    with pytest.raises(R.RoiError):
        R.server_footprint(256, 96, 272, (100.0, 100.0, -1.0, 1.0))
    with pytest.raises(R.RoiError):
        R.server_footprint(0, 96, 272, (100.0, 100.0, 5.0, 1.0))
    with pytest.raises(R.RoiError):
        R.server_footprint(256, 96, 272, (100.0, 100.0, 5.0, 1.0), storage=9)


def test_alloc_failure_hook_arguments():
    """The allocation-failure hook is host-only: negative counts are refused, 0 turns it off."""
    assert R.roi_recon_test_fail_alloc(-1) == R.ROI_EINVAL
    assert R.roi_recon_test_fail_alloc(3) == R.ROI_OK
    assert R.roi_recon_test_fail_alloc(0) == R.ROI_OK
