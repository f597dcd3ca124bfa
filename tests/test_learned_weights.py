"""The committed correction weights: shape, provenance and the held-out gain their
training recorded (CPU only; the GPU evaluation runs in bench.py and test_gpu_mlp)."""
import json
import os

import numpy as np

from oracle import mlp as ref

WEIGHTS = os.path.join(os.path.dirname(__file__), "..", "paper_1505_05341_gb300", "weights",
                       "correction_128cic_512tsc.npz")


def test_weights_file():
    z = np.load(WEIGHTS)
    assert z["params"].shape == (ref.N_PARAMS,) and z["params"].dtype == np.float32
    assert z["adam_m"].shape == z["adam_v"].shape == (ref.N_PARAMS,)
    assert np.all(np.isfinite(z["params"])) and np.all(z["adam_v"] >= 0)
    meta = json.loads(str(z["meta"]))
    assert meta["train_seeds"] == [10000, 11999] and meta["heldout_seeds"] == [20000, 20199]
    assert int(z["step"]) == meta["steps"]
    # held-out residuals against the 512^3 targets: every multipole's RMS fell
    b, a = meta["heldout_before"], meta["heldout_after"]
    assert a["rms0"] < 0.1 * b["rms0"] and a["rms4"] < 0.2 * b["rms4"]
    assert a["rms2"] < b["rms2"]
    # the direct galaxy sum entered training on small mocks, and on held-out small
    # mocks against it the monopole and hexadecapole residuals fell as well
    assert meta["direct_seeds"] == [30000, 30199] and meta["direct_rows"] > 0
    db, da = meta["direct_heldout_before"], meta["direct_heldout_after"]
    assert da["rms0"] < 0.1 * db["rms0"] and da["rms4"] < 0.3 * db["rms4"]


def test_weights_evaluate_on_cpu():
    z = np.load(WEIGHTS)
    X = np.array([[0.1, 3.0, 0.2, 0.01, 0.05], [0.95, 0.3, 0.02, 0.0, 0.74]])
    y, _ = ref.forward(ref.bf16_round(z["params"]), X)
    assert np.all(np.isfinite(y)) and np.abs(y).max() < 1.0
