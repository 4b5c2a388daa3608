"""The learned pair scheduler on the GPU.

* The training kernels' loss and gradient equal the FP64 CPU network oracle
  (within FP32 rounding).
* A logging run records one (features, outcome) row per tested pair, and its
  outcomes agree with the exact oracle's clustering.
* A trained schedule gives the same clustering as the oracle (the network only
  orders the exact tests), and on a held-out input it runs fewer BCP tests
  than testing the same pairs in list order.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1912_06255_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1912_06255_gb300 import DBSCAN  # noqa: E402


def _check(ctx, X, eps, mp):
    r = ctx.run(torch.from_numpy(X).cuda(), eps, mp)
    torch.cuda.synchronize()
    core, labels, off, ids = oracle.dbscan(X, eps, mp)
    assert np.array_equal(r.core.cpu().numpy(), core)
    assert np.array_equal(r.labels.cpu().numpy(), labels)
    assert np.array_equal(r.border_offsets.cpu().numpy(), off)
    assert np.array_equal(r.border_ids.cpu().numpy(), ids)
    return ctx.stats()


def test_loss_grad_matches_oracle():
    ctx = DBSCAN(1000, 3)
    rng = np.random.default_rng(3)
    n = 5000
    feat = np.abs(rng.normal(size=(n, 6)).astype(np.float32)) * 3
    lab = (rng.random(n) < 0.4).astype(np.uint8)
    w = (rng.normal(size=mlp.NPARAM) * 0.2).astype(np.float32)
    ctx.set_scheduler_weights(w)
    assert np.array_equal(ctx.scheduler_weights(), w)
    loss, g = ctx.scheduler_loss_grad(torch.from_numpy(feat).cuda(), torch.from_numpy(lab).cuda())
    L, G = mlp.loss_grad(w.astype(np.float64), feat.astype(np.float64), lab.astype(np.float64))
    assert abs(loss - L) <= 1e-5 * max(1.0, abs(L))
    scale = np.abs(G).max()
    assert np.abs(g - G).max() <= 2e-4 * scale, np.abs(g - G).max() / scale


def test_logging_run_and_training():
    X = synth.random_small(41, 30000, 3, dtype=np.float32)
    eps, mp = 0.35, 10
    ctx = DBSCAN(len(X), 3, cell_bounds=False, collect_stats=True)
    ctx.enable_pair_log(1 << 20)
    st = _check(ctx, X, eps, mp)
    feat, lab = ctx.pair_log()
    # a logging run tests every listed pair once and skips none
    assert st["num_pairs_skipped"] == 0 and feat.shape[0] == st["num_pairs_tested"] == st["num_pairs_listed"] > 0
    f = feat.cpu().numpy()
    y = lab.cpu().numpy()
    assert np.all(np.isfinite(f)) and set(np.unique(y)) <= {0, 1} and 0 < y.sum() < len(y)
    assert np.all(f[:, 3] <= f[:, 4] + 1e-6)          # box min distance <= box max distance
    assert np.all((f[:, 5] >= 0) & (f[:, 5] <= 1))
    losses = ctx.train_scheduler(epochs=30, batch=2048, lr=3e-3, seed=1)
    assert len(losses) == 30 and losses[-1] < losses[0] and losses[-1] < 0.69
    L, _ = mlp.loss_grad(ctx.scheduler_weights().astype(np.float64), f.astype(np.float64), y.astype(np.float64))
    assert abs(L - losses[-1]) < 0.05


@pytest.mark.parametrize("cell_bounds", [False, True])
def test_learned_schedule_parity_and_gain(cell_bounds):
    eps, mp = 0.35, 10
    Xtr = synth.random_small(41, 30000, 3, dtype=np.float32)
    Xte = synth.random_small(42, 30000, 3, dtype=np.float32)
    ctx = DBSCAN(len(Xtr), 3, cell_bounds=cell_bounds, collect_stats=True)
    ctx.enable_pair_log(1 << 20)
    _check(ctx, Xtr, eps, mp)
    ctx.train_scheduler(epochs=30, batch=2048, lr=3e-3, seed=1)
    ctx.enable_pair_log(0)
    ctx.set_option(1, 2)  # learned
    learned = _check(ctx, Xte, eps, mp)
    ctx.set_option(1, 1)  # list order
    plain = _check(ctx, Xte, eps, mp)
    ctx.set_option(1, 0)  # size heuristic (SortBySize)
    size = _check(ctx, Xte, eps, mp)
    for s in (learned, plain, size):
        assert (s["num_pairs_tested"] + s["num_pairs_skipped"] + s["num_pairs_box_decided"]
                == s["num_candidate_pairs"])
    print(f"cell_bounds={cell_bounds}: learned tested {learned['num_pairs_tested']} "
          f"skipped {learned['num_pairs_skipped']}; list order tested {plain['num_pairs_tested']} "
          f"skipped {plain['num_pairs_skipped']}; size order tested {size['num_pairs_tested']}")
    # fewer exact tests than both list order and the paper's SortBySize order
    # (the method without the network), on an input the network never saw
    assert learned["num_pairs_tested"] < plain["num_pairs_tested"]
    assert learned["num_pairs_tested"] < size["num_pairs_tested"]


@pytest.mark.parametrize("d", [2, 4])
def test_learned_schedule_other_dims(d):
    X = synth.random_small(60 + d, 12000, d, dtype=np.float64)
    ctx = DBSCAN(len(X), d, precision="fp64", schedule="learned")
    for eps, mp in ((0.2, 6), (0.45, 25)):
        _check(ctx, X, eps, mp)


def test_pair_list_grows_when_needed():
    """More undecided pairs than the initial 16 per point: the list grows and
    the run is repeated, with the same exact result."""
    rng = np.random.default_rng(17)
    X = (rng.random((20000, 3)) * 27.0).astype(np.float32)  # about one point per cell of side eps/sqrt(3)
    eps, mp = 1.0 * np.sqrt(3.0), 2
    ctx = DBSCAN(len(X), 3, schedule="learned", cell_bounds=False)
    st = _check(ctx, X, eps, mp)
    assert st["num_pairs_listed"] > 16 * len(X)
    st2 = _check(ctx, X, eps, mp)  # the grown list is kept
    assert st2["num_pairs_listed"] == st["num_pairs_listed"]

