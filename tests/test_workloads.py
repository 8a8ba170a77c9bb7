"""The synthetic input recipe: sizes, regions, separation, interface clearance,
orientation and determinism of the seeded media and geometries (CPU)."""

import numpy as np

from oracle import nystrom as onys
from workloads import config_c1, config_c2, config_c4, config_c5_stream


def _signed_area(poly):
    x, y = poly[:, 0], poly[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def _clearance(poly, interfaces):
    mid = 0.5 * (poly + np.roll(poly, -1, axis=0))
    ys = np.concatenate([poly[:, 1], mid[:, 1]])
    return float(np.min(np.abs(ys[:, None] - np.asarray(interfaces)[None, :])))


def test_c1_single_circle_in_the_top_layer():
    wl = config_c1()
    assert wl.n_elements == 256 and len(wl.bodies) == 1
    b = wl.bodies[0]
    assert np.allclose(np.hypot(b[:, 0], b[:, 1] - 1.0), 0.5)
    assert b[:, 1].min() > 0.0   # top layer, above y = 0
    assert list(wl.medium.k) == [2.0, 4.0] and list(wl.medium.eta) == [1.0, 2.0]


def test_c2_recipe():
    wl = config_c2()
    med = wl.medium
    assert wl.n_elements == 65536 and len(wl.bodies) == 64
    assert list(med.interfaces) == [0.0, -2.0] and list(med.k) == [4.0, 6.0, 8.0]
    cen = np.array([b.mean(axis=0) for b in wl.bodies])
    rad = np.array([np.max(np.hypot(*(b - c).T)) for b, c in zip(wl.bodies, cen)])
    assert np.all((cen[:, 0] >= -10) & (cen[:, 0] <= 10) & (cen[:, 1] >= -4) & (cen[:, 1] <= 2))
    d = np.hypot(cen[:, None, 0] - cen[None, :, 0], cen[:, None, 1] - cen[None, :, 1])
    np.fill_diagonal(d, np.inf)
    # bounding circles at least 0.05 apart (radii from the vertices, which lie on the curves)
    assert np.all(d >= rad[:, None] + rad[None, :] + 0.05 - 1e-9)
    assert min(_clearance(b, med.interfaces) for b in wl.bodies) >= 1e-6
    crossing = [b[:, 1].min() < yi < b[:, 1].max() for b in wl.bodies for yi in med.interfaces]
    assert any(crossing)
    assert all(_signed_area(b) > 0 for b in wl.bodies)   # counter-clockwise
    again = config_c2()
    assert all(np.array_equal(a, b) for a, b in zip(wl.bodies, again.bodies))


def test_elements_have_outward_normals_and_chord_weights():
    wl = config_c2(n_bodies=6, nodes=64)
    pts, w, nrm, bid = onys.elements(wl.bodies)
    for b, poly in enumerate(wl.bodies):
        sel = bid == b
        c = poly.mean(axis=0)
        assert np.all(np.einsum("ij,ij->i", nrm[sel], pts[sel] - c) > 0)
        assert np.allclose(np.hypot(nrm[sel, 0], nrm[sel, 1]), 1.0)
        chords = np.hypot(*(np.roll(poly, -1, axis=0) - poly).T)
        assert np.allclose(w[sel], chords)


def test_c4_sizes_layers_and_angles():
    wls = config_c4()
    assert len(wls) == 16
    for i, wl in enumerate(wls):
        target = max(256, int(round(4096.0 * 32.0 ** (i / 15.0) / 256.0)) * 256)
        assert 0.98 * target <= wl.n_elements <= target
        assert wl.medium.n_layers == 2 + (i % 3)
        assert np.all((wl.medium.k >= 2.0) & (wl.medium.k <= 12.0))
        assert np.allclose(wl.angles_deg, (np.arange(32) + 0.5) * 180.0 / 32.0)
        assert min(_clearance(b, wl.medium.interfaces) for b in wl.bodies) >= 1e-6
    assert wls[0].n_elements == 4096 and wls[-1].n_elements == 131072


def test_c5_stream_recipe():
    reqs = config_c5_stream(8)
    for wl in reqs:
        assert 2 <= wl.medium.n_layers <= 4
        assert np.all((wl.medium.k >= 2.0) & (wl.medium.k <= 12.0))
        assert 5.0 <= float(wl.angles_deg[0]) <= 175.0
        nb = len(wl.bodies)
        assert 1 <= nb <= 32 and all(b.shape[0] >= 64 for b in wl.bodies)
        assert 2048 * 0.5 <= wl.n_elements <= 32768 * 1.5 + 64 * nb
        if wl.medium.n_layers > 1:
            assert min(_clearance(b, wl.medium.interfaces) for b in wl.bodies) >= 1e-6
    assert [wl.n_elements for wl in reqs] == [wl.n_elements for wl in config_c5_stream(8)]


def _polar_residual(poly, c, a, b, kk, th0):
    d = poly - np.asarray(c)[None, :]
    r, th = np.hypot(d[:, 0], d[:, 1]), np.arctan2(d[:, 1], d[:, 0])
    return np.max(np.abs(r - (a * np.sin(kk * (th - th0)) + b)))


def test_paper_example_geometries():
    # Sec. 5: the L-shape of Example 1, the peanuts of Example 2 and the flowers of Example 3
    # (r = a sin k (theta - theta0) + b about each centre), at the replay sizes
    from workloads import example1, example2, example3

    e1 = example1(12000)
    L = e1.bodies[0]
    assert L.shape[0] == 12000
    assert np.isclose(np.sum(np.hypot(*(np.roll(L, -1, axis=0) - L).T)), 12.5)   # perimeter
    assert np.isclose(_signed_area(L), 1.5 * 3.25 + 1.5 * 1.0)                  # area, counter-clockwise
    e2, e3 = example2(12000), example3(12000)
    for b, c in zip(e2.bodies, [(0.0, -1.0), (2.0, -3.0)]):
        assert _polar_residual(b, c, 0.5, 1.0, 2, np.pi / 4) < 1e-12
    centres = [(-1.5, 0.0), (1.5, 0.0), (0.0, -2.0), (-1.5, -4.0), (1.5, 4.0)]
    for b, c in zip(e3.bodies, centres):
        assert _polar_residual(b, c, 0.2, 0.7, 5, 0.0) < 1e-12
    for wl in (e1, e2, e3):
        assert all(_signed_area(b) > 0 for b in wl.bodies)
        for i in range(len(wl.bodies)):
            for j in range(i):   # disjoint bodies
                d = np.hypot(wl.bodies[i][:, None, 0] - wl.bodies[j][None, :, 0],
                             wl.bodies[i][:, None, 1] - wl.bodies[j][None, :, 1])
                assert d.min() > 0.1
    # every element centre (chord midpoint, the collocation point) of every replay size keeps
    # clear of the interfaces; vertices may lie on them (the L-shape's do)
    for make in (example1, example2, example3):
        for n in (12000, 24000, 48000, 96000, 192000):
            wl = make(n)
            mid = np.concatenate([0.5 * (b + np.roll(b, -1, axis=0)) for b in wl.bodies])
            gap = np.min(np.abs(mid[:, 1][:, None] - np.asarray(wl.medium.interfaces)[None, :]))
            assert gap >= 1e-6, (make.__name__, n, gap)
            assert wl.n_elements == n
