"""Host logic of the learned proposal's camera layouts (no GPU): which views of an
instance fill the network's slots, and the cameras of views resampled to the
network's resolution -- checked against the scene generator's own cameras and the
pinhole projection they define."""
import numpy as np
import pytest

from paper_2107_05509_gb300 import inputs as I
from paper_2107_05509_gb300 import proposal as PR


def test_view_slots_spread_and_repeat():
    assert PR.view_slots(8) == list(range(8))
    assert PR.view_slots(16) == list(range(0, 16, 2))
    assert PR.view_slots(4) == [0, 0, 1, 1, 2, 2, 3, 3]
    assert PR.view_slots(5) == [0, 0, 1, 1, 2, 3, 3, 4]
    for k in range(1, 40):
        s = PR.view_slots(k)
        assert len(s) == PR.SLOTS and s == sorted(s) and s[0] == 0 and s[-1] <= k - 1
        # every view is used when there are no more views than slots; none twice otherwise
        if k <= PR.SLOTS:
            assert set(s) == set(range(k))
        else:
            assert len(set(s)) == PR.SLOTS
    with pytest.raises(ValueError):
        PR.view_slots(0)


def _project(cam, X):
    R = cam[4:13].reshape(3, 3).astype(np.float64)
    Xc = R @ X + cam[13:16]
    return np.array([cam[0] * Xc[0] / Xc[2] + cam[2], cam[1] * Xc[1] / Xc[2] + cam[3]])


@pytest.mark.parametrize("wh", I.BATCH_RESOLUTIONS)
def test_ring_cameras_are_the_scene_cameras_rescaled(wh):
    W, H = wh
    hand = I.make_hand(0)
    target = hand.v_template.mean(0)
    cfg = I.SceneConfig("t", views=5, width=W, height=H, spp=4, edge_samples=0, elevation_deg=30.0,
                        azimuths_deg=tuple(17.0 + 72.0 * k for k in range(5)))
    native = I.pack_cameras(I.make_cameras(cfg, target))
    got = PR.ring_cameras(cfg.azimuths_deg, 30.0, cfg.radius, target, [wh] * 5, size=256)
    # extrinsics and centre as the scene generator's (float32 rounding apart)
    assert np.allclose(got[:, 4:19], native[:, 4:19], rtol=0, atol=2e-7)
    # intrinsics: a point projecting to (u, v) in the native image projects to
    # (u 256 / W, v 256 / H) in the resampled one
    rng = np.random.default_rng(1)
    for c in range(5):
        assert got[c, 0] == pytest.approx(1.2 * W * 256 / W) and got[c, 1] == pytest.approx(1.2 * W * 256 / H)
        assert got[c, 2] == pytest.approx(128.0) and got[c, 3] == pytest.approx(128.0)
        for _ in range(4):
            X = target + rng.normal(0, 0.03, 3)
            u = _project(native[c], X)
            assert np.allclose(_project(got[c], X), u * np.array([256.0 / W, 256.0 / H]), rtol=1e-5, atol=1e-3)


def test_sampled_ring_layouts_follow_the_heterogeneous_distribution():
    hand = I.make_hand(0)
    target = hand.v_template.mean(0)
    rng = np.random.default_rng(5)
    n = 400
    cams = PR.sample_ring_layouts(rng, n, target).reshape(n, PR.SLOTS, I.CAM_FLOATS)
    fy = cams[:, 0, 1]
    # fx is 1.2 x 256 for every native resolution; fy too except for 512 x 384 (4/3 of it)
    assert np.allclose(cams[..., 0], 307.2)
    frac_43 = np.isclose(fy, 409.6).mean()
    assert np.all(np.isclose(fy, 307.2) | np.isclose(fy, 409.6)) and 0.25 < frac_43 < 0.42
    # one fy per instance; cameras at 0.6 m from the target, 30 degrees up
    assert np.all(cams[:, :, 1] == fy[:, None])
    d = cams[..., 16:19] - target[None, None, :]
    assert np.allclose(np.linalg.norm(d, axis=2), 0.6, atol=1e-6)
    assert np.allclose(d[..., 1] / 0.6, np.sin(np.radians(30.0)), atol=1e-6)
    # the azimuth steps between consecutive slots are multiples of 360 / k, with k in 4..16
    az = np.degrees(np.arctan2(d[..., 0], d[..., 2]))
    steps = np.mod(np.diff(az, axis=1), 360.0)
    smallest = np.array([s[s > 1e-3].min() for s in steps])
    k = np.rint(360.0 / smallest)
    assert np.all((k >= 4) & (k <= 16)) and len(set(k.tolist())) > 8
