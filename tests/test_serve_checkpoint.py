"""The serving loop's checkpoint file (CPU): every field of a stopped stream survives the round
trip -- request identity, progress, per-step statistics, and a parked request's next source
modes and warm-start pressure -- and finished requests come back marked finished."""
import math

import numpy as np

from paper_1410_1942_gb300 import inputs, serve


def test_checkpoint_round_trip(tmp_path):
    reqs = serve.request_stream(3, math.inf, seed=5, hi=(64, 32, 32))
    rng = np.random.default_rng(0)
    # request 0 finished; request 1 parked after 2 steps; request 2 never admitted
    reqs[0].step, reqs[0].finished, reqs[0].done_at = 3, True, 1.5
    reqs[0].latencies, reqs[0].residuals = [0.01, 0.02, 0.03], [9e-10, 8e-10, 7e-10]
    reqs[0].iters, reqs[0].statuses = [40, 20, 15], [0, 0, 0]
    r = reqs[1]
    r.step, r.cancel_after = 2, 5
    r.latencies, r.residuals, r.iters, r.statuses = [0.1, 0.2], [5e-10, 6e-10], [30, 12], [0, 0]
    g = inputs.Grid(*r.shape, 1.0 / r.shape[2])
    r.modes = inputs.advect_modes(inputs.fourier_modes(np.random.default_rng(1)), g, inputs.DT)
    r.resume_p = rng.standard_normal((r.shape[2], r.shape[1], r.shape[0]))
    path = str(tmp_path / "stream.npz")
    serve.Server.checkpoint(path, reqs)
    back = serve.Server.load_checkpoint(path)
    assert [q.rid for q in back] == [q.rid for q in reqs]
    for a, b in zip(reqs, back):
        assert (b.arrival, b.shape, b.seed, b.step) == (a.arrival, tuple(a.shape), a.seed, a.step)
        assert (b.latencies, b.residuals, b.iters, b.statuses) == (a.latencies, a.residuals,
                                                                    a.iters, a.statuses)
        assert b.cancel_after == a.cancel_after and b.cancelled == a.cancelled
    assert back[0].finished and not back[1].finished and not back[2].finished
    assert back[0].resume_p is None and back[2].resume_p is None
    assert np.array_equal(back[1].resume_p, r.resume_p)
    assert back[1].modes == r.modes
