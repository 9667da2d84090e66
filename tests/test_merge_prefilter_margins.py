"""The merger's FP32 prefilter (continuity and dz, ahead of the exact tests) must
never reject a pair the exact tests accept.  A numpy float32 model of the
kernel's evaluation, with the kernel's margins (1e-5 relative and absolute
terms, about 20 times a rounding-error bound of the FP32 evaluation), against
the FP64 tests on pairs placed within 1e-9 to 1e-3 of both limits, for radii
of 5 cm to 10 km."""
import math

import numpy as np

KB = 0.299792458e-2 * 0.5
f32 = np.float32


def exact(g, a, b):
    """The FP64 continuity and dz tests of the merger (sector-track reading)."""
    ref, oth = (a, b) if g["VQ"][a] <= g["VQ"][b] else (b, a)
    L = math.hypot(g["X"][oth] - g["X"][ref], g["Y"][oth] - g["Y"][ref])
    d = abs(math.hypot(g["X"][oth] - g["XC"][ref], g["Y"][oth] - g["YC"][ref]) - g["R"][ref])
    dlim = 1 + 3 * KB * math.sqrt(g["VQ"][ref]) * L * L
    i, o = (a, b) if g["RAD"][a] <= g["RAD"][b] else (b, a)
    c = math.hypot(g["X"][o] - g["X"][i], g["Y"][o] - g["Y"][i])
    Rb = 0.5 * (g["R"][a] + g["R"][b])
    arc = c * (1 + c * c / (24 * Rb * Rb))
    dz = abs(g["Z"][o] - (g["Z"][i] + g["TGL"][i] * arc))
    return d <= dlim and dz <= 2.0


def prefilter(g, a, b):
    """float32 model of the kernel's prefilter (False: certainly incompatible)."""
    G = {k: v.astype(np.float32) for k, v in g.items()}
    e, kBf = f32(1e-5), f32(KB)
    r, o = (a, b) if G["VQ"][a] <= G["VQ"][b] else (b, a)
    dxl, dyl = G["X"][o] - G["X"][r], G["Y"][o] - G["Y"][r]
    L2 = f32(dxl * dxl + dyl * dyl)
    ex, ey = G["X"][o] - G["XC"][r], G["Y"][o] - G["YC"][r]
    d = abs(np.sqrt(f32(ex * ex + ey * ey)) - G["R"][r])
    kv = f32(3) * kBf * np.sqrt(G["VQ"][r])
    Q = abs(G["X"][o]) + abs(G["Y"][o]) + abs(G["X"][r]) + abs(G["Y"][r])
    Mc = abs(G["X"][o]) + abs(G["Y"][o]) + abs(G["XC"][r]) + abs(G["YC"][r]) + G["R"][r]
    dlim = f32(kv * L2 + f32(1))
    if d > dlim * (f32(1) + e) + e * (kv * Q * Q + Mc) + f32(1e-6):
        return False
    if G["RAD"][a] == G["RAD"][b]:
        return True
    i, o = (a, b) if G["RAD"][a] < G["RAD"][b] else (b, a)
    cx, cy = G["X"][o] - G["X"][i], G["Y"][o] - G["Y"][i]
    c = np.sqrt(f32(cx * cx + cy * cy))
    Rb = f32(0.5) * (G["R"][a] + G["R"][b])
    t = c * c / (f32(24) * Rb * Rb)
    arc = c * (f32(1) + t)
    dz = abs(G["Z"][o] - f32(G["TGL"][i] * arc + G["Z"][i]))
    Qz = abs(G["X"][i]) + abs(G["Y"][i]) + abs(G["X"][o]) + abs(G["Y"][o])
    lim = f32(2) + e * (abs(G["Z"][o]) + abs(G["Z"][i]) + abs(G["TGL"][i]) * (arc + Qz) * (f32(2) + f32(4) * t))
    return not (dz > lim + f32(1e-6))


def test_prefilter_never_rejects_an_accepted_pair():
    rng = np.random.default_rng(5)
    accepted = 0
    with np.errstate(all="ignore"):
        for _ in range(6000):
            R = math.exp(rng.uniform(math.log(5), math.log(1e6)))
            phi = rng.uniform(0, 2 * math.pi)
            X0, Y0 = rng.uniform(80, 250) * math.cos(phi), rng.uniform(80, 250) * math.sin(phi)
            th = rng.uniform(0, 2 * math.pi)
            XC, YC = X0 + R * math.cos(th), Y0 + R * math.sin(th)
            VQ = float(np.float32(math.exp(rng.uniform(math.log(1e-8), math.log(1e-1)))))
            X1, Y1 = X0 + rng.uniform(-200, 200), Y0 + rng.uniform(-200, 200)
            L = math.hypot(X1 - X0, Y1 - Y0)
            dlim = 1 + 3 * KB * math.sqrt(VQ) * L * L
            dd = dlim * (1 + rng.choice([-1, 1]) * 10 ** rng.uniform(-9, -3)) * rng.choice([-1, 1])
            h = math.hypot(X1 - XC, Y1 - YC)
            X1, Y1 = XC + (X1 - XC) * (R + dd) / h, YC + (Y1 - YC) * (R + dd) / h  # on the continuity limit
            g = {k: np.zeros(2) for k in ("XC", "YC", "R", "X", "Y", "RAD", "Z", "TGL", "VQ")}
            g["XC"][:], g["YC"][:], g["R"][:] = XC, YC, R
            g["X"][:], g["Y"][:] = [X0, X1], [Y0, Y1]
            g["RAD"][:] = [math.hypot(X0, Y0), math.hypot(X1, Y1)]
            g["VQ"][:] = [VQ, float(np.float32(VQ * rng.uniform(1, 4)))]
            tgl = float(np.float32(rng.uniform(-1.5, 1.5)))
            g["TGL"][:] = tgl
            i, o = (0, 1) if g["RAD"][0] <= g["RAD"][1] else (1, 0)
            c = math.hypot(X1 - X0, Y1 - Y0)
            arc = c * (1 + c * c / (24 * R * R))
            z0 = float(np.float32(rng.uniform(-250, 250)))
            g["Z"][i] = z0  # and dz on its limit
            g["Z"][o] = float(np.float32(z0 + tgl * arc + rng.choice([-1, 1]) * 2 *
                                         (1 + rng.choice([-1, 1]) * 10 ** rng.uniform(-9, -3))))
            if exact(g, 0, 1):
                accepted += 1
                assert prefilter(g, 0, 1), (R, g)
    assert accepted > 100
