"""The learned warm start end to end, at a small scale: steady solutions from
the solver, a short training run of the network, and the time to a 1e-6
residual from the network's prediction against a start from rest on members
the network has not seen."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_warm_start_reaches_steady_state_sooner():
    pytest.importorskip("torch")
    from paper_2401_17183_gb300 import build as B
    B.build()
    from paper_2401_17183_gb300 import warmstart as WS
    X, Y, keep = WS.dataset(WS.family(4, 64))
    assert len(keep) == 64          # every member reached the residual
    ws = WS.WarmStart(width=32, batch=16)
    losses, _ = ws.train(X, Y, 300)
    assert losses[-1] < 0.05 * losses[0]
    test = WS.family(5, 8)
    Xt, Yt, kt = WS.dataset(test)
    pred = ws.predict(Xt)
    cold, _ = WS.run_to_steady([m[2] for m in WS.make_sims([test[k] for k in kt])])
    warm, _ = WS.run_to_steady([m[2] for m in WS.make_sims([test[k] for k in kt], init=pred)])
    assert warm.mean() < 0.7 * cold.mean(), (warm, cold)
