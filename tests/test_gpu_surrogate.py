"""What the trained crater surrogate gains over the solver alone.

Training data: the batched FP32-mix solver on 4096 seeded draws of the impact distribution
at 400 x 400 cells, run to 20 s (`paper_2403_04267_gb300/data/surrogate_400.npz`, written
by `python -m paper_2403_04267_gb300.surrogate generate`); 256 held-out draws from a
disjoint seed range.  The network is trained here, on the GPU, by the library's own
tensor-core kernels (an ensemble of 8 networks, 12000 full-batch Adam steps each, on the
logarithms of transient depth and diameter).  The solver is the judge (its outputs are the
targets) and the fallback (draws the ensemble disagrees on go to it); the gate is calibrated
on a tenth of the training draws held back for validation, to 97 % there (a margin for the
95 % bar on unseen draws)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_04267_gb300 import salec, surrogate as S

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2403_04267_gb300", "data", "surrogate_400.npz")


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    salec.load()
    D = np.load(DATA)
    ok = D["train_status"] == 0
    X, T = D["train_X"][ok], D["train_T"][ok]
    nv = len(X) // 10
    ens = S.Ensemble(X[:-nv], T[:-nv], members=8, steps=12000)
    tau = S.calibrate_gate(ens, X[-nv:], T[-nv:])
    okh = D["heldout_status"] == 0
    return ens, tau, D["heldout_X"][okh], D["heldout_T"][okh], (X[:-nv], T[:-nv])


def test_training_fits_the_solver_data(trained):
    ens, _, _, _, (X, T) = trained
    Y, _, _ = ens.predict(X)
    ed, eD = S.crater_errors(Y, T)
    print("train fit median depth/diameter error", np.median(ed), np.median(eD))
    # the fit to its own training draws: typical errors inside the 2 % band
    assert np.median(ed) < 0.03 and np.median(eD) < 0.03


def test_surrogate_gain_on_heldout_draws(trained):
    ens, tau, Xh, Th, _ = trained
    assert tau > 0.0
    # the solver's cost per 400 x 400 run to 20 s is seconds; take a conservative 1 s
    rep = S.gain_report(ens, tau, Xh, Th, solver_s_per_run=1.0)
    print("gain report", rep)
    # the bar: accepted predictions within 2 % of the solver in both transient depth and
    # diameter for at least 95 % of the held-out draws the gate accepts
    assert rep["accepted"] >= 0.5 * rep["draws"]
    assert rep["accepted_within_tol"] >= 0.95
    assert rep["runs_per_hour_with_surrogate"] > 2.0 * rep["runs_per_hour_solver"]
