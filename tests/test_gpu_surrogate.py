"""What the trained network gains over the method without it: held-out
cavities reach the residual tolerance in fewer steps from the network's
prediction than from rest, and converge to the same vorticity.  The method
decides the final state: both runs stop only at residual 1e-8 (velocity and scalar).
Small configuration (64^2 grid, 192 training cavities) so the test runs in
well under a minute."""
import pytest

torch = pytest.importorskip("torch")

from paper_1908_06742_gb300 import build as B
from paper_1908_06742_gb300 import surrogate as S

pytestmark = pytest.mark.gpu


def test_warm_start_saves_steps():
    assert torch.cuda.is_available(), "GPU test"
    B.build()
    r = S.experiment(n=64, n_train=192, n_test=16, epochs=100, batch=16, c=32, seed=5,
                     max_steps=1_500_000, log=lambda s: None)
    print({k: v for k, v in r.items() if k != "rows"})
    assert r["n_test_both_converged"] == 16
    assert r["pred_rel_err_median"] < 0.15
    assert r["steps_saved_ratio"] > 1.3, r["steps_saved_ratio"]
    assert r["omega_rel_diff_max"] < 0.05
