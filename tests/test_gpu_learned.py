"""The learned correction end to end on a reduced focused-source case: data
from the solver, training on the GPU with the library's kernels, and the
gain of coarse+net over the coarse scheme alone against the fine solution,
on an amplitude not seen in training."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_trained_network_improves_coarse_runs():
    torch = pytest.importorskip("torch")
    from paper_1311_3004_gb300 import build, learned
    build.build()
    spec = learned.SMALL
    X, T = learned.generate(spec, [0.2e6, 0.35e6, 0.5e6], log=None)
    net, info = learned.train_net(X, T, steps=600, crop=48, batch=8, lr=1e-3, log=None)
    assert info["loss_last"] < 0.5 * info["loss_first"]
    res = learned.evaluate(spec, 0.42e6, net, info)
    print(res)
    c, cn = res["coarse"], res["coarse_net"]
    assert cn["l2_rel_err"] < 0.9 * c["l2_rel_err"], (c, cn)
    net.close()
