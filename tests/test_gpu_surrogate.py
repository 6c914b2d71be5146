"""What the trained network gains over the method without it: held-out
cavities reach the residual tolerance in fewer steps from the network's
prediction than from rest, and end with the same vorticity error against a
long-run reference of the method.  The method decides the final state: both
runs stop only at residual 1e-8 (velocity and scalar); a capped run would
count at its cap.  Small configuration (64^2 grid, 192 training cavities, the
last 96 of them warm-started by a network trained on the first 96) so the test
runs in about a minute."""
import pytest

torch = pytest.importorskip("torch")

from paper_1908_06742_gb300 import build as B
from paper_1908_06742_gb300 import surrogate as S

pytestmark = pytest.mark.gpu


def test_warm_start_saves_steps():
    assert torch.cuda.is_available(), "GPU test"
    B.build()
    r = S.experiment(n=64, n_train=192, n_test=16, epochs=100, batch=16, c=32, seed=5,
                     max_steps=1_500_000, boot=96, boot_epochs=60, log=lambda s: None)
    print({k: v for k, v in r.items() if k != "rows"})
    for row in r["rows"]:
        print(row)
    assert r["n_test_both_converged"] == 16
    assert r["pred_rel_err_median"] < 0.15
    assert r["steps_saved_ratio"] >= 2.0, r["steps_saved_ratio"]
    assert r["median_ratio"] >= 1.5, r["median_ratio"]
    assert r["omega_rel_diff_max"] < 0.05
    # equal vorticity error: warm and cold end the same distance from the reference
    assert r["omega_err_warm_median"] <= 1.5 * r["omega_err_cold_median"] + 1e-3
    # the bootstrapped training data took fewer steps per cavity than the cold data
    assert r["data_steps_warm_mean"] < r["data_steps_cold_mean"]
