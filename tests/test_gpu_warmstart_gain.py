"""What the trained warm start gains: steps to the Eq. 6 steady state (1e-9) from the network's
field against the run from rest (Sec. 2.2 i), on held-out draws, through the whole pipeline
(coarse batched runs, FP64 targets, training by the library's BF16 tensor-core kernels, the
validation-chosen fallback gate, batched evaluation at equal residual).

Small setting where the gain is known to exist: fine 128 x round(128 Ar), coarse 64 x round(64 Ar),
Re ~ U[100, 400], Ar ~ U[0.4, 2.0]; 48 training, 12 validation, 16 test draws, 20 epochs.  The
gated warm start must converge on every test draw and need at most 0.95 of the total steps of the
runs from rest (measured with 96 training draws: 0.88).
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2211_05009_gb300 import warmstart as W  # noqa: E402


def test_trained_warm_start_cuts_total_steps_to_steady_state():
    args = W.parser().parse_args(
        "--nx 128 --re-min 100 --re-max 400 --train 48 --val 12 --test 16 --epochs 20 --width 12 "
        "--max-steps 300000".split())
    rep = W.run(args)
    ev = rep["evaluation"]
    tot = ev["total_steps"]
    print(f"total steps to 1e-9 -- rest {tot['rest']}, coarse field {tot['coarse']}, network {tot['network']}, "
          f"network with fallback gate {tot['network_gated']} (gate Re < {rep['gate']['re_gate']:.0f}); "
          f"velocity error of the warm fields {rep['velocity_error']}")
    assert ev["converged"]["rest"] == ev["n"] and ev["converged"]["network_gated"] == ev["n"]
    assert tot["network_gated"] <= 0.95 * tot["rest"]
    assert rep["training"]["loss_last_epoch"] < 0.2 * rep["training"]["loss_first_epoch"]
