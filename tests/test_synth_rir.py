"""Pins of the image-source room simulator used for the synthetic Table 1
sweep (input generation, not FCC arithmetic): with absorbing walls only the
direct path remains (amplitude 1 / (4 pi r) at delay r fs / c), a first-order
reflection appears where its image predicts it, and the response is
reciprocal (source and microphone swapped give the same RIR)."""
import math

import numpy as np

from paper_2204_13622_gb300 import synth

FS, C = 16000.0, 343.0


def test_direct_path_only():
    room = [6.0, 5.0, 3.0]
    src, mic = np.array([2.0, 2.0, 1.5]), np.array([2.0 + 343.0 * 40 / 16000.0, 2.0, 1.5])  # 40 samples away
    h = synth.image_source_rir(room, src, mic[None], 0.0, FS, C, 0.05).numpy()[0]
    r = 40 * C / FS
    assert np.argmax(h) == 40
    assert abs(h[40] - 1 / (4 * math.pi * r)) < 1e-6 / r
    h[40] = 0
    assert np.abs(h).max() < 1e-9


def test_first_order_floor_reflection():
    room = [20.0, 20.0, 10.0]
    src, mic = np.array([10.0, 10.0, 1.0]), np.array([12.0, 10.0, 1.0])
    h = synth.image_source_rir(room, src, mic[None], 0.5, FS, C, 0.02).numpy()[0]
    r_img = math.sqrt(2.0 ** 2 + 2.0 ** 2)  # the floor image is 1 m below the floor
    k = r_img * FS / C
    k0 = int(round(k))
    # the reflection's band-limited pulse peaks within a sample of its delay
    seg = h[k0 - 2:k0 + 3]
    assert abs(np.argmax(seg) - 2) <= 1
    assert seg.max() > 0.6 * 0.5 / (4 * math.pi * r_img)


def test_reciprocity():
    room = [7.0, 6.0, 3.5]
    a, b = np.array([1.3, 2.2, 1.1]), np.array([4.1, 3.7, 2.0])
    h1 = synth.image_source_rir(room, a, b[None], 0.7, FS, C, 0.1).numpy()[0]
    h2 = synth.image_source_rir(room, b, a[None], 0.7, FS, C, 0.1).numpy()[0]
    assert np.abs(h1 - h2).max() < 1e-6 * np.abs(h1).max()
