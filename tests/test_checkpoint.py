"""Checkpoint / resume and the per-iteration metrics log: host logic on the
CPU; on the GPU, a run resumed from a checkpoint follows the uninterrupted
run."""
import json
import os

import numpy as np
import pytest

from paper_2007_03800_gb300 import checkpoint as ck


def test_save_load_round_trip(tmp_path):
    rng = np.random.default_rng(0)
    D1, D2 = rng.standard_normal((8, 16)), rng.standard_normal((8, 16))
    cfg = {"p1": 8, "p2": 8, "n1": 16, "n2": 16, "s": 4, "seed": 1}
    path = str(tmp_path / "run.npz")
    ck.save(path, D1, D2, 7, cfg)
    got = ck.load(path, cfg)
    assert got["iteration"] == 7 and got["config"] == cfg
    np.testing.assert_array_equal(got["D1"], D1.astype(np.float32))
    np.testing.assert_array_equal(got["D2"], D2.astype(np.float32))
    assert not any(p.name.startswith("run.npz.tmp") for p in tmp_path.iterdir())


def test_config_hash_ignores_key_order_and_guards_resume(tmp_path):
    a = {"s": 4, "p1": 8, "eps": 0.0}
    b = {"eps": 0.0, "p1": 8, "s": 4}
    assert ck.config_hash(a) == ck.config_hash(b)
    assert ck.config_hash(a) != ck.config_hash({**a, "s": 5})
    path = str(tmp_path / "run.npz")
    ck.save(path, np.eye(2), np.eye(2), 1, a)
    with pytest.raises(ValueError):
        ck.load(path, {**a, "s": 5})


def test_metrics_log_is_json_lines(tmp_path):
    log = ck.MetricsLog(str(tmp_path / "m.jsonl"))
    log.log(iteration=1, rmse_after_D1=2.5, nnz_hist=[0, 1, 2])
    log.log(iteration=2, rmse_after_D1=2.0, nnz_hist=[0, 0, 3])
    recs = log.read()
    assert [r["iteration"] for r in recs] == [1, 2]
    for line in open(tmp_path / "m.jsonl"):
        json.loads(line)


def test_learn_rejects_a_zero_checkpoint_interval():
    with pytest.raises(ValueError):
        ck.learn(None, np.zeros((1, 2, 2)), None, None, 1, 1, every=0)


class _FailingContext:
    """Stand-in context: iterations run, the device error word reports
    SDL_ERR_NONFINITE from iteration `bad` on."""

    def __init__(self, bad):
        self.bad, self.calls = bad, 0

    def iterate(self, Y, D1, D2, s, eps=0.0, out=None, rmse_out=None):
        import torch

        from paper_2007_03800_gb300 import sdl
        self.calls += 1
        N = Y.shape[0]
        return sdl.Codes(torch.zeros((N, s), dtype=torch.int32), torch.zeros((N, s)),
                         torch.full((N,), s, dtype=torch.int32))

    def status(self):
        return -3 if self.calls >= self.bad else 0


def test_learn_stops_on_a_device_error_without_checkpointing(tmp_path):
    """A device-side error reported after an iteration stops learn() before
    that iteration is logged or checkpointed; earlier iterations stand."""
    import torch

    from paper_2007_03800_gb300 import sdl
    Y = torch.zeros((4, 2, 2))
    D1, D2 = torch.zeros((2, 3)), torch.zeros((2, 3))
    path = str(tmp_path / "ck.npz")
    log = ck.MetricsLog(str(tmp_path / "m.jsonl"))
    with pytest.raises(sdl.SDLError) as e:
        ck.learn(_FailingContext(bad=1), Y, D1, D2, 2, 3, checkpoint=path, log=log)
    assert e.value.code == -3
    assert not os.path.exists(path) and log.read() == []
    with pytest.raises(sdl.SDLError):
        ck.learn(_FailingContext(bad=3), Y, D1, D2, 2, 5, checkpoint=path, log=log)
    assert [r["iteration"] for r in log.read()] == [1, 2]
    assert ck.load(path)["iteration"] == 2


@pytest.mark.gpu
def test_learn_refuses_to_checkpoint_non_finite_data(gpu_ctx, tmp_path):
    import torch

    from paper_2007_03800_gb300 import sdl, synth
    Y, _, _, _, _ = synth.kron_model(512, 8, 8, 16, 16, 4, 20.0, seed=11)
    Y[5, 1, 1] = np.nan
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    Yg = sdl.signals(torch.tensor(Y, dtype=torch.float32, device="cuda:0"))
    D1g = sdl.dictionary(torch.tensor(D1, dtype=torch.float32, device="cuda:0"))
    D2g = sdl.dictionary(torch.tensor(D2, dtype=torch.float32, device="cuda:0"))
    path = str(tmp_path / "ck.npz")
    with pytest.raises(sdl.SDLError) as e:
        ck.learn(gpu_ctx, Yg, D1g, D2g, 4, 2, checkpoint=path)
    assert sdl.ERRORS[e.value.code] == "SDL_ERR_NONFINITE"
    assert not os.path.exists(path)


@pytest.mark.gpu
def test_resume_follows_the_uninterrupted_run(gpu_ctx, tmp_path):
    import torch

    from paper_2007_03800_gb300 import sdl, synth
    Y, _, _, _, _ = synth.kron_model(2048, 8, 8, 16, 16, 4, 20.0, seed=11)
    D1, D2 = synth.init_dictionaries(8, 8, 16, 16, seed=1)
    dev = "cuda:0"
    Yg = sdl.signals(torch.tensor(Y, dtype=torch.float32, device=dev))

    def dicts(A, B):
        return (sdl.dictionary(torch.tensor(np.asarray(A), dtype=torch.float32, device=dev)),
                sdl.dictionary(torch.tensor(np.asarray(B), dtype=torch.float32, device=dev)))

    cfg = {"shape": [8, 8, 16, 16], "s": 4, "N": 2048, "seed": 11}
    straight = ck.MetricsLog(str(tmp_path / "a.jsonl"))
    A1, A2 = dicts(D1, D2)
    ck.learn(gpu_ctx, Yg, A1, A2, 4, 4, config=cfg, log=straight)
    assert gpu_ctx.status() == 0

    path = str(tmp_path / "run.npz")
    resumed = ck.MetricsLog(str(tmp_path / "b.jsonl"))
    B1, B2 = dicts(D1, D2)
    ck.learn(gpu_ctx, Yg, B1, B2, 4, 2, config=cfg, checkpoint=path, log=resumed)
    state = ck.load(path, cfg)
    assert state["iteration"] == 2
    C1, C2 = dicts(state["D1"], state["D2"])
    ck.learn(gpu_ctx, Yg, C1, C2, 4, 4, config=cfg, checkpoint=path, log=resumed, start=state["iteration"])
    assert gpu_ctx.status() == 0
    assert ck.load(path, cfg)["iteration"] == 4

    np.testing.assert_allclose(C1.cpu().numpy(), A1.cpu().numpy(), rtol=0, atol=1e-6)
    np.testing.assert_allclose(C2.cpu().numpy(), A2.cpu().numpy(), rtol=0, atol=1e-6)
    ra, rb = straight.read(), resumed.read()
    assert [r["iteration"] for r in rb] == [1, 2, 3, 4]
    for x, y in zip(ra, rb):
        assert y["rmse_after_D2"] == pytest.approx(x["rmse_after_D2"], rel=1e-6)
        assert sum(y["nnz_hist"]) == 2048
