"""The C ray caster of the input generator (synth/raycast.c) gives the numpy casts'
float64 depths bit for bit: street frames (road, facades with window recesses, car
boxes seen through their pixel windows) and yawed tiny-scene frames."""

import numpy as np

from synth.scenes import segment_scenes, street_scene, tiny_scene


def test_c_casts_equal_numpy_casts():
    cases = [(street_scene(seed=0), (0, 57, 199)), (tiny_scene(seed=3, yaw_jitter=0.1), (0, 1, 2, 3)),
             (segment_scenes()[5], (3, 150))]
    for sc, frames in cases:
        for k in frames:
            a, b = sc.render_clean(k), sc.render_clean_numpy(k)
            assert np.array_equal(a, b), (sc.name, k, int((a != b).sum()))
            assert (a > 0).mean() > 0.3
