"""Space-point distortion correction (location-dependent calibration: the
paper's Abstract; online calibration: Sec. 3).  Clusters of config-1 shape are
distorted by a smooth synthetic space-charge field (|d| <= 10 cm); the per-sector
64^3 trilinear grid undoes it.  Parity: corrected coordinates against the FP64
oracle element by element; tracks against the oracle tracking the oracle's
corrected clusters; and the correction's gain over tracking without it."""
import numpy as np
import pytest

import oracle
import trackeval
from paper_1910_12214_b300 import synth
from gpu_helpers import compare_tracks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def distorted():
    cl = synth.make_config1(seed=5)
    d = synth.make_distortion(seed=5, n_sectors=1, single_sector=True)
    grid, bounds = synth.correction_grid(d)
    return cl, synth.distort(cl, d), grid, bounds


class _C:
    def __init__(self, cl, y, z):
        self.x, self.row, self.item_off = cl.x, cl.row, cl.item_off
        self.item_sector, self.item_event, self.item_core = cl.item_sector, cl.item_event, None
        self.y, self.z = y, z
        self.mc = cl.mc


def _track(cl, mode, grid=None, bounds=None):
    from paper_1910_12214_b300 import tpc
    with tpc.Tracker() as t:
        if grid is not None:
            t.set_grid_correction(grid, bounds)
        t.set_correction(mode)
        t.load(cl).track()
        trk, ids = t.get_tracks()
        cy, cz = t.corrected()
        q = t.debug_dump(0).reshape(-1, 3)
    return trk, ids, cy, cz, q


def test_grid_correction_matches_oracle_elementwise(distorted):
    cl, dcl, grid, bounds = distorted
    _, _, cy, cz, _ = _track(dcl, "grid", grid, bounds)
    oy, oz = oracle.correct_clusters(dcl, grid, bounds)
    assert np.max(np.abs(cy - oy)) < 2e-4 and np.max(np.abs(cz - oz)) < 2e-4


def test_tracks_on_corrected_clusters_match_oracle(distorted):
    cl, dcl, grid, bounds = distorted
    trk, ids, cy, cz, q = _track(dcl, "grid", grid, bounds)
    oy, oz = oracle.correct_clusters(dcl, grid, bounds)
    ocl = _C(dcl, oy, oz)
    ref = oracle.run(ocl)
    # FP32 and FP64 corrections may round to a different 2^-10 cm quantum
    same = np.mean((ref["sorted_qy"] == q[:, 0]) & (ref["sorted_qz"] == q[:, 1]))
    assert same > 0.99
    r = compare_tracks(ocl, trk, ids, ref)
    assert r["matched"] >= 0.995 and r["param_ok"] >= 0.995, r


def test_correction_restores_tracking(distorted):
    from paper_1910_12214_b300 import tpc
    cl, dcl, grid, bounds = distorted
    trk0, ids0, *_ = _track(cl, "none")
    trk_n, ids_n, *_ = _track(dcl, "none")
    trk_g, ids_g, *_ = _track(dcl, "grid", grid, bounds)
    e0 = trackeval.efficiency(cl, tpc.tracks_to_trk_i(trk0), ids0)
    en = trackeval.efficiency(cl, tpc.tracks_to_trk_i(trk_n), ids_n)
    eg = trackeval.efficiency(cl, tpc.tracks_to_trk_i(trk_g), ids_g)
    chi_n = trk_n["chi2"].sum() / trk_n["ndf"].sum()
    chi_g = trk_g["chi2"].sum() / trk_g["ndf"].sum()
    print("eff undistorted", e0["eff"], "distorted none", en["eff"], "grid", eg["eff"], "chi2/ndf", chi_n, chi_g)
    assert eg["eff"] >= e0["eff"] - 0.02
    # the uncorrected distortion (up to 10 cm) shows in the fit quality; the
    # correction brings chi2/ndf back to about 1
    assert chi_g < 1.3 and chi_n > 1.5 * chi_g
