"""Host logic of the K-step training windows (train.RolloutStream), on CPU
with a stand-in for the refined-run pair stream: window t of an episode holds
the restricted states t, t+1, ..., t+K of that episode, `episode` windows per
episode, and no window spans two episodes."""
import numpy as np

from paper_2504_14494_gb300 import lib as L
from paper_2504_14494_gb300 import train


class _FakePairs:
    """PairStream's contract: next() advances one coarse step and returns
    (state t, state t+1, taus) as buffers valid until the next call; t counts
    the pairs of the current episode (a new episode when t reaches episode)."""

    def __init__(self, device, episode, **kw):
        import torch
        self.episode = episode
        self.coarse = L.shape(2, 3, 1)
        self.t = episode
        self.ep = -1
        self.buf = [torch.zeros(54) for _ in range(2)]
        self.taus = torch.ones(1)

    def next(self):
        if self.t >= self.episode:
            self.ep += 1
            self.t = 0
            self.buf[0].fill_(1000.0 * self.ep)
        self.buf[1].fill_(1000.0 * self.ep + self.t + 1)
        src, dst = self.buf[0], self.buf[1]
        self.buf.reverse()
        self.t += 1
        return src, dst, self.taus


def test_rollout_windows_are_consecutive_states_of_one_episode(monkeypatch):
    monkeypatch.setattr(train, "PairStream", _FakePairs)
    for K, ep in ((1, 4), (2, 3), (4, 5)):
        rs = train.RolloutStream("cpu", K=K, episode=ep)
        n = rs.f_in.numel()
        for e in range(3):
            for t in range(ep):
                f_in, tg, _ = rs.next()
                assert np.all(f_in.numpy() == 1000.0 * e + t), (K, ep, e, t)
                for k in range(K):
                    assert np.all(tg[k * n:(k + 1) * n].numpy() == 1000.0 * e + t + 1 + k)


def test_channel_training_host_checks():
    """Argument checks of the channel pair bank and trainer that run before
    any device work: an even refinement factor, a bank that is not a whole
    number of batches, an unknown weighting."""
    import pytest

    with pytest.raises(ValueError):
        train.ChannelPairBank("cpu", m=2)

    class _Bank:
        nb = 10

    with pytest.raises(ValueError):
        train.ChannelTrainer("cpu", _Bank(), batch=4)
    _Bank.nb = 8
    with pytest.raises(ValueError):
        train.ChannelTrainer("cpu", _Bank(), batch=4, weighting="unknown")
