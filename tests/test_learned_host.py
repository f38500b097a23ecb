"""Host logic of the training loop (paper_1606_00556_gb300.learned.train) on
CPU, with a stand-in network that records the calls the loop makes: every
sample is used once per epoch, each batch holds the rows of X and Y it names,
the learning rate falls linearly from lr to lr_final, losses are read only
at the logging steps, and a batch larger than the network or the data set is
refused before any call."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


class _Net:
    def __init__(self, max_batch):
        self.max_batch = max_batch
        self.batches, self.lrs, self.wants = [], [], []

    def backward(self, x, y, mask, nout=1, want_loss=True):
        # the sample id is stored in every entry of its rows
        ids = x[:, 0, 0].float().round().long().tolist()
        assert ids == y[:, 0, 0].round().long().tolist()
        self.batches.append(ids)
        self.wants.append(want_loss)
        return float(len(self.batches)) if want_loss else None

    def adam_step(self, lr):
        self.lrs.append(lr)


def _data(n, V=5):
    ids = torch.arange(n, dtype=torch.float32)
    X = ids[:, None, None].expand(n, V, 16).to(torch.bfloat16).contiguous()
    Y = ids[:, None, None].expand(n, V, 4).contiguous()
    return X, Y


def test_each_epoch_uses_every_sample_once():
    from paper_1606_00556_gb300 import learned
    n, batch = 12, 4
    X, Y = _data(n)
    net = _Net(max_batch=4)
    learned.train(net, X, Y, steps=9, batch=batch, seed=3)
    assert all(len(b) == batch for b in net.batches)
    per_epoch = n // batch
    for e in range(3):
        seen = sum(net.batches[e * per_epoch:(e + 1) * per_epoch], [])
        assert sorted(seen) == list(range(n))


def test_learning_rate_falls_linearly_and_losses_are_read_when_logged():
    from paper_1606_00556_gb300 import learned
    X, Y = _data(10)
    net = _Net(max_batch=2)
    losses = learned.train(net, X, Y, steps=6, batch=2, lr=1e-2, lr_final=2e-3, log_every=4)
    assert np.allclose(net.lrs, np.linspace(1e-2, 2e-3, 6))
    assert net.wants == [True, False, False, False, True, True]
    assert [it for it, _ in losses] == [0, 4, 5]
    net2 = _Net(max_batch=2)
    learned.train(net2, X, Y, steps=3, batch=2, lr=1e-3)
    assert np.isclose(net2.lrs[-1], 1e-4) and not any(net2.wants)


def test_oversized_batch_is_refused():
    from paper_1606_00556_gb300 import learned
    X, Y = _data(6)
    with pytest.raises(ValueError):
        learned.train(_Net(max_batch=2), X, Y, steps=1, batch=4)
    with pytest.raises(ValueError):
        learned.train(_Net(max_batch=8), X, Y, steps=1, batch=7)
