"""Host-side pins of the seeded input generators that both the CUDA path and
the oracle consume: every Lagrangian point lies on its surface with a unit
outward normal, the point counts follow the recipes, and the seeded case
sets are reproducible and stay inside their stated ranges."""
import numpy as np
import pytest

from paper_2607_07432_b300 import inputs


def test_cylinder_points_and_normals():
    g = inputs.cylinder((20.3, 11.7), 14.0, 44)
    X, N = g["X"], g["normals"]
    r = np.hypot(X[:, 0] - 20.3, X[:, 1] - 11.7)
    assert np.allclose(r, 7.0, atol=1e-12)
    assert np.allclose(np.hypot(N[:, 0], N[:, 1]), 1.0, atol=1e-14)
    assert np.allclose(X - np.array([20.3, 11.7]), 7.0 * N, atol=1e-12)   # outward radial
    assert g["tbc"].shape == (44,) and g["u_target"].shape == (44, 2)


@pytest.mark.parametrize("angle", [0.0, 0.6, 2.0])
def test_ellipse_points_normals_and_spacing(angle):
    a, b, n = 15.0, 6.0, 80
    g = inputs.ellipse((40.0, 30.0), a, b, angle, n)
    X, N = g["X"], g["normals"]
    c, s = np.cos(angle), np.sin(angle)
    dx, dy = X[:, 0] - 40.0, X[:, 1] - 30.0
    xr, yr = c * dx + s * dy, -s * dx + c * dy
    assert np.allclose((xr / a) ** 2 + (yr / b) ** 2, 1.0, atol=1e-6)
    # the normal is the normalised gradient of the implicit function, pointing out
    gx, gy = xr / a ** 2, yr / b ** 2
    gn = np.hypot(gx, gy)
    nr = np.stack([c * N[:, 0] + s * N[:, 1], -s * N[:, 0] + c * N[:, 1]], axis=1)
    assert np.allclose(nr, np.stack([gx / gn, gy / gn], axis=1), atol=1e-9)
    # uniform in arc length: chords between neighbours nearly equal
    ch = np.hypot(*(np.roll(X, -1, axis=0) - X).T)
    assert ch.max() / ch.min() < 1.02


def test_naca0012_shape():
    g = inputs.naca0012((100.0, 50.0), 100.0, 256)
    X, N = g["X"], g["normals"]
    x = (X[:, 0] - 100.0) / 100.0
    y = (X[:, 1] - 50.0) / 100.0
    assert x.min() > -1e-9 and abs(x.max() - 1.0) < 1e-9            # leading edge at 0, trailing edge at the chord
    assert abs(y.max() - 0.06) < 2e-3 and abs(y.min() + 0.06) < 2e-3  # 12% thickness, symmetric
    assert np.allclose(np.hypot(N[:, 0], N[:, 1]), 1.0, atol=1e-12)
    # outward: upper-surface normals point up, lower-surface ones down (away from the tips)
    mid = (x > 0.05) & (x < 0.95)
    assert np.all(N[mid & (y > 0), 1] > 0) and np.all(N[mid & (y < 0), 1] < 0)


@pytest.mark.parametrize("freq", [4, 7, 27])
def test_icosphere_count_radius_normals(freq):
    g = inputs.icosphere((64.0, 96.0, 96.0), 48.0, freq)
    X, N = g["X"], g["normals"]
    assert X.shape == (10 * freq * freq + 2, 3)                       # 7292 points at frequency 27
    assert np.allclose(np.linalg.norm(X - np.array([64.0, 96.0, 96.0]), axis=1), 24.0, atol=1e-10)
    assert np.allclose(X - np.array([64.0, 96.0, 96.0]), 24.0 * N, atol=1e-10)
    # no duplicated points
    d = np.linalg.norm(X[:, None, :] - X[None, :, :], axis=2) if freq < 10 else None
    if d is not None:
        assert np.sort(d, axis=1)[:, 1].min() > 1e-3


def test_batch_cases_seeded_and_in_range():
    a = inputs.batch_cases(64, 20260001)
    b = inputs.batch_cases(64, 20260001)
    assert a == b
    assert inputs.batch_cases(64, 20260002) != a
    for c in a:
        assert c["nx"] % 64 == 0 and 256 <= c["nx"] <= 1024 and c["ny"] == c["nx"] // 2
        assert 10.0 <= c["ref_length"] <= 60.0 and 32 <= c["n_points"] <= 512
        assert 1.0 <= c["a"] / c["b"] <= 3.0
        assert 0.1 <= c["mach"] <= 0.8 and 20.0 <= c["reynolds"] <= 200.0
        if not c["ellipse"]:
            assert c["a"] == c["b"]


def test_warmstart_cases_separation_and_bounds():
    cases = inputs.warmstart_cases(40, 20260002)
    assert cases == inputs.warmstart_cases(40, 20260002)
    for c in cases:
        nx, ny = c["shape"]
        pc = np.array(c["circle"]["center"])
        pe = np.array(c["ellipse"]["center"])
        dc, de = c["circle"]["diameter"], 2.0 * c["ellipse"]["a"]
        assert np.hypot(*(pc - pe)) >= 0.5 * (dc + de) + 10.0        # bounding circles 10 cells apart
        assert c["ellipse"]["b"] >= 3.0
        for p in (pc, pe):
            assert 0.15 * nx <= p[0] <= 0.5 * nx                      # upstream half
        assert 0.1 <= c["mach"] <= 0.45 and 20.0 <= c["reynolds"] <= 200.0


def test_two_body_mask_and_signed_distance_agree():
    case = inputs.warmstart_cases(1, 7)[0]
    geo = inputs.two_body_geometry(case, 1.0)
    mask = geo["shape"]["mask"].astype(bool)
    sd = inputs.signed_distance(case)
    assert mask.shape == sd.shape == (case["shape"][1], case["shape"][0])
    # strictly inside the union <=> negative signed distance (away from the
    # surfaces, where the ellipse distance is only approximate)
    far = np.abs(sd) > 1.0
    assert np.array_equal(mask[far], (sd < 0)[far])
    # every Lagrangian point sits on a body surface
    X = geo["X"]
    nc = int(round(np.pi * case["circle"]["diameter"]))
    c = np.array(case["circle"]["center"])
    assert np.allclose(np.hypot(*(X[:nc] - c).T), 0.5 * case["circle"]["diameter"], atol=1e-9)
