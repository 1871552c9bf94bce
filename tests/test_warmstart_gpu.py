"""What the trained network gains over the uniform start, and that it does
not change the answer.

Reduced form of the warm-start study (grid 128 x 64 instead of 512 x 256,
64 training cases instead of 2000, bodies of 6-14 cells, Ma 0.1-0.3,
Re 20-40 so that every case has a steady state): the solver generates the
training fields in one batched launch per step, the network trains on the
GPU, and on four held-out cases the warm start must reach the 0.1% drag
band of the uniform-start answer in fewer steps, while converging to the
same drag."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPE = (128, 64)
KW = dict(shape=SHAPE, d_range=(6.0, 14.0), mach_range=(0.1, 0.3), re_range=(20.0, 40.0))


def test_warm_start_shortens_the_transient():
    from paper_2607_07432_b300 import inputs, warmstart as ws
    train_cases = inputs.warmstart_cases(64, 20260002, **KW)
    held_out = inputs.warmstart_cases(4, 20260003, **KW)
    X, Y = ws.generate(train_cases, 12000)
    assert np.all(np.isfinite(Y))
    net = ws.new_network(SHAPE, max_batch=8)
    losses = ws.train(net, X, Y, 600, 8, 1e-3, lr_final=1e-4)
    assert losses[-50:].mean() < 0.05 * losses[:5].mean()
    res = [ws.compare(net, c, 16000, 50) for c in held_out]
    net.close()
    for r in res:
        assert r["steps_uniform"] is not None and r["steps_warm"] is not None, r
        # the converged answer is the plain solve's, whatever the start
        assert abs(r["warm_final"] - r["cd_inf"]) <= 1e-4 * abs(r["cd_inf"]), r
    su = np.mean([r["steps_uniform"] for r in res])
    sw = np.mean([r["steps_warm"] for r in res])
    assert sw < 0.85 * su, (sw, su, res)
