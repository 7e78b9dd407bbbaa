"""The learned variant pick: the cost model trained on the GPU (with the
library's own kernels) on the committed GB300 timing sweep picks variants
whose time is within 10 % (geometric mean) of the exhaustive best on the
500 held-out shapes, and improves on the method without it (the single
best fixed variant per op)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_02389_gb300 import build, lift
    build.build()
    torch.cuda.set_device(0)
    lift.lift_init(0)
    return lift


def test_learned_pick_regret_and_gain(L, tmp_path):
    from paper_1502_02389_gb300 import costmodel as cm
    from paper_1502_02389_gb300 import tune
    tr = tune.load_csv(os.path.join(cm.DATA, "timings_gb300_train.csv"))
    ho = tune.load_csv(os.path.join(cm.DATA, "timings_gb300_heldout.csv"))
    assert len(tr) >= 3000 and len({(r["op"], r["n"], r["M"], r["N"]) for r in ho}) >= 499
    _, X, T, M = cm.dataset(tr)
    trainer = cm.Trainer(X, T, M, seed=0)
    hist = trainer.train(3000, 3e-3, log_every=300)
    assert hist[-1] < 0.5 * hist[0]
    w = str(tmp_path / "mlp.txt")
    cm.save(w, trainer.params(), T.shape[1], cm.offsets(tr)[0])
    res = cm.evaluate_policies(tr, ho, w, str(tmp_path / "table.txt"))
    print(res)
    assert res["mlp"]["geomean"] <= 1.10
    assert res["mlp"]["geomean"] < res["best_fixed"]["geomean"]
