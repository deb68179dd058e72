"""The FSC / FCR utility (Section 4) and the random-conical-tilt workload: shell
membership is the paper's inequality (0.5 + (i-1) + eps <= |j| < 0.5 + i + eps,
eps = 1e-4), the FSC of a volume with itself (any positive scale) is 1 and with its
negative -1, the cone mask is the angular condition, and every slice of a 60-degree
tilt series misses the 30-degree cone about z."""
import numpy as np

import synth
from paper_1307_5824_gb300 import metrics as Mt


def test_shells_follow_the_paper_inequality():
    N = 10
    sh = Mt.shell_index(N)
    f = np.fft.fftfreq(N, 1.0 / N)
    for a in range(N):
        for b in range(N):
            for c in range(N):
                r = np.sqrt(f[a] ** 2 + f[b] ** 2 + f[c] ** 2)
                want = 0
                for i in range(1, N // 2):
                    if 0.5 + (i - 1) + 1e-4 <= r < 0.5 + i + 1e-4:
                        want = i
                assert sh[a, b, c] == want


def test_fsc_of_a_volume_with_itself_and_its_negative():
    V = np.random.default_rng(81).standard_normal((16, 16, 16))
    assert np.allclose(Mt.fsc(V, V), 1.0) and np.allclose(Mt.fsc(V, 3.0 * V), 1.0)
    assert np.allclose(Mt.fsc(V, -V), -1.0)
    W = np.random.default_rng(82).standard_normal((16, 16, 16))
    assert np.abs(Mt.fsc(V, W)[2:]).max() < 0.3           # independent noise: near 0
    # inside and outside a cone, each restricted FSC of V with itself is 1
    m = Mt.cone_mask(16, (0, 0, 1), 30.0)
    assert np.allclose(Mt.fsc(V, V, m)[1:], 1.0) and np.allclose(Mt.fsc(V, V, ~m), 1.0)


def test_cone_mask_is_the_angle_to_the_axis():
    N = 16
    m = Mt.cone_mask(N, (0, 0, 1), 30.0)
    f = np.fft.fftfreq(N, 1.0 / N).astype(int)
    idx = {v: i for i, v in enumerate(f)}
    def at(x, y, z):
        return bool(m[idx[z], idx[y], idx[x]])
    assert at(0, 0, 5) and at(0, 0, -5) and at(1, 0, 2)       # 0, 180, 26.6 degrees
    assert not at(2, 0, 3) and not at(5, 0, 5) and not at(3, 4, 0)   # 33.7, 45, 90 degrees
    assert not at(0, 0, 0)


def test_rct_views_lie_on_the_tilt_cone_and_miss_the_cone_about_z():
    R = synth.rct_rotations(300, 60.0, 5)
    d = R[:, 2, :]                                           # viewing directions
    assert np.allclose(d[:, 2], 0.5, atol=1e-12)             # polar angle 60 degrees
    az = np.arctan2(d[:, 1], d[:, 0])
    assert np.histogram(az, bins=6, range=(-np.pi, np.pi))[0].min() > 25   # azimuths spread
    # slice directions u = R row 0, v = R row 1: every in-plane frequency is at least 30
    # degrees from the z axis
    t = np.linspace(0, 2 * np.pi, 64, endpoint=False)
    xi = np.cos(t)[None, :, None] * R[:, None, 0, :] + np.sin(t)[None, :, None] * R[:, None, 1, :]
    ang = np.degrees(np.arccos(np.abs(xi[..., 2]) / np.linalg.norm(xi, axis=-1)))
    assert ang.min() >= 30.0 - 1e-9
    inp = synth.config_inputs("RCT", M=50, N=16)
    assert inp["groups"].shape[0] == 0 and inp["images"].shape == (50, 16, 16)
