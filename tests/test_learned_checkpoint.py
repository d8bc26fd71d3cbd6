"""Training checkpoints of the learned-initial-guess network, on the CPU.

A stand-in network with the library's get_state/set_state/train_step interface
records the batches it is given, so the tests check the checkpoint file (round
trip, rejection of foreign and truncated files) and that a resumed run draws the
same shuffles and hands over the same state as an uninterrupted one. The GPU
test in test_gpu_learned.py checks the same on the real network, bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2001_04886_gb300 import learned  # noqa: E402


class FakeNet:
    """Adam-free stand-in: params += lr * mean of the batch's first feature; m counts
    steps. Deterministic, so an interrupted and an uninterrupted run can be compared."""

    def __init__(self, n=7, fail_at_step=None):
        self.num_params = n
        self.fail_at_step = fail_at_step
        self.params = np.arange(n, dtype=np.float32) * 0.5
        self.m = np.zeros(n, dtype=np.float32)
        self.v = np.ones(n, dtype=np.float32)
        self.step = 0
        self.batches = []

    def get_state(self):
        return {"params": self.params.copy(), "m": self.m.copy(), "v": self.v.copy(), "step": self.step}

    def set_state(self, st):
        self.params = np.array(st["params"], dtype=np.float32)
        self.m = np.array(st["m"], dtype=np.float32)
        self.v = np.array(st["v"], dtype=np.float32)
        self.step = int(st["step"])

    def train_step(self, x, t, lr, lossd):
        if self.step == self.fail_at_step:
            raise RuntimeError("the process dies here")
        self.batches.append(x[:, 0, 0, 0].tolist())
        self.params = self.params + np.float32(lr) * np.float32(float(x[:, 0].mean()))
        self.m = self.m + 1
        self.step += 1
        lossd.fill_(float(t.mean()))

    def status(self):
        pass


def data(S=40):
    g = torch.Generator().manual_seed(3)
    return torch.rand(S, 2, 4, 4, generator=g), torch.rand(S, 1, 4, 4, generator=g)


def test_checkpoint_round_trip(tmp_path):
    net = FakeNet()
    net.step = 11
    net.m[:] = 2.5
    p = tmp_path / "a.ckpt"
    learned.save_checkpoint(p, net, epoch=3, seed=9)
    ck = learned.load_checkpoint(p)
    assert (ck["step"], ck["epoch"], ck["seed"]) == (11, 3, 9)
    for k in ("params", "m", "v"):
        assert ck[k].dtype == np.float32 and np.array_equal(ck[k], getattr(net, k))
    assert p.stat().st_size == 40 + 12 * net.num_params
    assert not (tmp_path / "a.ckpt.tmp").exists()


def test_checkpoint_rejects_foreign_and_truncated_files(tmp_path):
    net = FakeNet()
    p = tmp_path / "b.ckpt"
    learned.save_checkpoint(p, net, 1, 0)
    raw = p.read_bytes()
    (tmp_path / "t.ckpt").write_bytes(raw[:-4])
    (tmp_path / "f.ckpt").write_bytes(b"XXXX" + raw[4:])
    (tmp_path / "v.ckpt").write_bytes(raw[:4] + np.array([2], dtype="<u4").tobytes() + raw[8:])
    for name in ("t.ckpt", "f.ckpt", "v.ckpt"):
        with pytest.raises(ValueError):
            learned.load_checkpoint(tmp_path / name)


def test_resumed_training_equals_uninterrupted(tmp_path):
    feats, targets = data()
    full = FakeNet()
    h_full = learned.train(full, feats, targets, epochs=4, batch=8, lr=0.1, seed=5)
    ck = tmp_path / "c.ckpt"
    first = FakeNet(fail_at_step=12)        # 5 steps per epoch: dies inside epoch 2
    with pytest.raises(RuntimeError):
        learned.train(first, feats, targets, epochs=4, batch=8, lr=0.1, seed=5, checkpoint=ck)
    assert learned.load_checkpoint(ck)["epoch"] == 2
    first.batches = first.batches[:10]       # the steps of the two completed epochs
    # a fresh process: a new network resumes from the file; epochs 0-1 are not repeated
    second = FakeNet()
    h_rest = learned.train(second, feats, targets, epochs=4, batch=8, lr=0.1, seed=5, checkpoint=ck, resume=True)
    assert len(h_rest) == 2 and h_rest == h_full[2:]
    assert second.batches == full.batches[len(first.batches):]
    assert np.array_equal(second.params, full.params) and second.step == full.step
    assert learned.load_checkpoint(ck)["epoch"] == 4
    with pytest.raises(ValueError):
        learned.train(FakeNet(), feats, targets, epochs=4, batch=8, seed=6, checkpoint=ck, resume=True)
