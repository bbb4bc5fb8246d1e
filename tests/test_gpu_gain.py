"""What the trained network gains (Section 5): the reduced-order model with the decoder trained on
GPU snapshots against the same method without it, on a held-out 2D impact scene.

* untrained: the same network at its Xavier initialisation (Appendix B), same scaling;
* linear manifold: the same network with identity activations, trained on the same snapshots for
  the same number of steps (an affine map of (X, xhat), the linear baseline of Section 5; its
  dg/dX is one constant matrix, so it moves the body as a translation of a fixed shape).

All three run the same reduced step (Algorithms 2, 3, 5, 6) for 2000 steps (fall and floor
impact) with the settings of the benchmark (FP32 decoder calls, ridge 0.1 on the increments,
reference gradient) and are scored by the accumulated relative position error against the
full-order run.  The trained network must beat both.
"""
import numpy as np
import pytest

import synth.scenes as S

pytestmark = pytest.mark.gpu
TRAIN_STEPS = 6000
STEPS = 2000


def test_trained_decoder_beats_untrained_and_linear_manifold():
    from paper_2109_12390_gb300 import pipeline as PL
    from paper_2109_12390_gb300.train import generate_snapshots
    train_sc = S.batch_2d(seed=3, n_inst=16, fixed_side=64, n_grid=128, origin_y=0.06)
    snaps = generate_snapshots(train_sc, STEPS, 10)
    assert snaps["status"] == 0
    rng = np.random.default_rng(44)
    E = float(rng.uniform(5e3, 1.5e4))
    v0 = rng.uniform(-0.5, 0.5, size=2)
    sc = S.block_2d(seed=4, side=64, dt=5e-5, origin=(0.375, 0.06), E=E, v0=v0)
    fx, _, fstat = PL.fom_positions(sc, STEPS)
    assert fstat == 0
    settings = dict(n_samples=256, seed=4, projection=0, ridge=1e-1, f_reference=1)
    errs = {}
    for name, act, steps in (("trained", 0, TRAIN_STEPS), ("linear", 1, TRAIN_STEPS), ("untrained", 0, 0)):
        dec, _ = PL.decoder_for_snapshots(snaps, 16, seed=0, activation=act)
        if steps:
            tr, hist, _ = PL.train(snaps, dec, steps=steps)
            assert np.isfinite(hist[-1][1])
            tr.close()
        dec.set_precision(True)
        errs[name] = PL.rom_error(dec, sc, fx, **settings).error_percent
    print("accumulated relative position error (%)", errs)
    # the untrained network does not represent the motion at all
    assert errs["trained"] < 0.1 * errs["untrained"], errs
    # and the nonlinear manifold beats the linear one trained on the same snapshots for as long
    assert errs["trained"] < errs["linear"], errs
