"""The learned BF16 surrogate of the grid correction: its gradients against the
FP64 oracle on the same BF16-rounded batch, its tensor-core inference against
the oracle's forward pass, its residual against the grid (which judges it) and
against the exact inverse of the field, bit-identical resume from a checkpoint,
and what the trained network gains in tracking over no correction."""
import math

import numpy as np
import pytest

import oracle
import trackeval
from paper_1910_12214_b300 import synth

pytestmark = pytest.mark.gpu
OW1, OB1, OW2, OB2, OW3, OB3 = 0, 192, 256, 4352, 4416, 4608
SLICES = {"W1": slice(OW1, OB1), "b1": slice(OB1, OW2), "W2": slice(OW2, OB2), "b2": slice(OB2, OW3),
          "W3": slice(OW3, OB3), "b3": slice(OB3, 4611)}


@pytest.fixture(scope="module")
def world():
    cl = synth.make_config1(seed=9)
    d = synth.make_distortion(seed=9, n_sectors=1, single_sector=True)
    grid, bounds = synth.correction_grid(d)
    return cl, synth.distort(cl, d), d, grid, bounds


def _tracker(grid, bounds, **kw):
    from paper_1910_12214_b300 import tpc
    t = tpc.Tracker(**kw)
    t.set_grid_correction(grid, bounds)
    return t


def test_gradients_match_fp64_oracle(world):
    _, _, _, grid, bounds = world
    P = oracle.mlp_init(11, 0)
    rng = np.random.default_rng(0)
    P[OB1:OW2] = rng.normal(0, 0.2, 64)
    P[OB2:OW3] = rng.normal(0, 0.2, 64)
    P[OB3:] = rng.normal(0, 0.2, 3)
    with _tracker(grid, bounds) as t:
        t.surrogate_set_params(0, P)
        assert np.array_equal(t.surrogate_params(0), P)
        g_gpu, loss_gpu = t.surrogate_grad(0, seed=5, step=17, batch=512)
    x, tg = oracle.mlp_batch(5, 0, 17, 512, grid[0])
    g_ref, loss_ref = oracle.mlp_grad(P, x, tg)
    assert abs(loss_gpu - loss_ref) <= 1e-2 * loss_ref
    for name, sl in SLICES.items():
        err = np.linalg.norm(g_gpu[sl] - g_ref[sl]) / np.linalg.norm(g_ref[sl])
        assert err <= 2e-2, (name, err)


def test_tensor_core_inference_matches_oracle_forward(world):
    _, dcl, _, grid, bounds = world
    P = oracle.mlp_init(12, 0)
    P[OB3:] = [0.0, 0.3, -0.2]
    with _tracker(grid, bounds) as t:
        t.surrogate_set_params(0, P)
        t.set_correction("mlp")
        t.load(dcl).track()
        cy, cz = t.corrected()
    x0, x1, v0, v1, z0, z1 = (float(v) for v in bounds[0])
    xr = np.rint((85.0 + np.arange(152) * (161.0 / 151.0)) * 1024.0) / 1024.0
    x = xr[dcl.row]
    y = dcl.y.astype(np.float64)
    z = dcl.z.astype(np.float64)
    v = y / (x * math.tan(math.radians(10.0)))
    inp = np.stack([(x - x0) * (2 / (x1 - x0)) - 1, (v - v0) * (2 / (v1 - v0)) - 1, (z - z0) * (2 / (z1 - z0)) - 1], 1)
    out = oracle.mlp_forward(P, inp)
    ey = np.abs(cy - (y + 10.0 * out[:, 1]))
    ez = np.abs(cz - (z + 10.0 * out[:, 2]))
    scale = 10.0 * np.abs(out[:, 1:]).max()
    assert np.max(ey) <= 1e-2 * scale and np.max(ez) <= 1e-2 * scale, (ey.max(), ez.max(), scale)


def test_checkpoint_resume_is_bit_identical(world, tmp_path):
    _, _, _, grid, bounds = world
    with _tracker(grid, bounds) as a:
        a.surrogate_train(40 * 1024, seed=3)
        straight = a.surrogate_params(0)
    with _tracker(grid, bounds) as b:
        b.surrogate_train(40 * 1024, seed=3, max_steps=15)
        b.surrogate_save(tmp_path / "ckpt.bin")
    with _tracker(grid, bounds) as c:
        c.surrogate_load(tmp_path / "ckpt.bin")
        c.surrogate_train(40 * 1024, seed=3)
        resumed = c.surrogate_params(0)
    assert np.array_equal(straight, resumed)


def test_trained_surrogate_residual_and_tracking_gain(world):
    from paper_1910_12214_b300 import tpc
    cl, dcl, d, grid, bounds = world
    with _tracker(grid, bounds) as t:
        mx, rms = t.surrogate_train(40_000_000, seed=1)  # 10M samples x 4 epochs
        # residual against the exact inverse of the field at the distorted clusters
        t.set_correction("mlp")
        t.load(dcl).track()
        cy, cz = t.corrected()
        trk_m, ids_m = t.get_tracks()
        t.set_correction("grid")
        t.track()
        trk_g, ids_g = t.get_tracks()
        t.set_correction("none")
        t.track()
        trk_n, ids_n = t.get_tracks()
    xr = np.rint((85.0 + np.arange(152) * (161.0 / 151.0)) * 1024.0) / 1024.0
    sig = dcl.mc >= 0
    yt, zt = synth.exact_correction(d, 0, xr[dcl.row[sig]], dcl.y[sig], dcl.z[sig])
    ex = np.hypot(cy[sig] - yt, cz[sig] - zt)
    effs = {k: trackeval.efficiency(cl, tpc.tracks_to_trk_i(tr), ids)
            for k, (tr, ids) in dict(mlp=(trk_m, ids_m), grid=(trk_g, ids_g), none=(trk_n, ids_n)).items()}
    chi = {k: float(tr["chi2"].sum() / tr["ndf"].sum()) for k, tr in dict(mlp=trk_m, grid=trk_g, none=trk_n).items()}
    print("SURROGATE residual vs grid max %.3f rms %.3f cm; vs exact max %.3f rms %.3f cm" %
          (mx, rms, ex.max(), math.sqrt(np.mean(ex ** 2))), {k: round(v["eff"], 4) for k, v in effs.items()}, chi)
    assert rms < 0.1 and mx < 0.5
    assert effs["mlp"]["eff"] > effs["none"]["eff"] + 0.3
    assert effs["mlp"]["eff"] >= effs["grid"]["eff"] - 0.03
    assert chi["mlp"] < 0.7 * chi["none"]
