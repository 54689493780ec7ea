"""The autotuner: cache keys and file on CPU; timing a few (threads, block size) candidates and
planning with the winner on the GPU (the winner must still match the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_cache_keys_and_file_roundtrip(tmp_path, monkeypatch):
    from paper_1002_2469_gb300 import autotune as AT
    monkeypatch.setattr(AT, "CACHE", str(tmp_path / "tune.json"))
    k1 = AT.key_of((-1.2, 2.5, -0.8), 1 << 26, 1, device_name="GB300")
    k2 = AT.key_of((-1.2, 2.5, -0.8), (1 << 26) + 5, 1, device_name="GB300")
    k3 = AT.key_of((-1.0, 2.001, -1.0), 1 << 26, 1, device_name="GB300")
    assert k1 == k2 and k1 != k3                      # same N bucket; a longer decay length differs
    assert "form1" in k1 and AT.key_of((-1.2, 2.5, -0.8), 1 << 26, 0, device_name="GB300") != k1
    assert AT._load() == {}
    AT._save({k1: {"threads": 128, "block_size": 16, "ms": 0.37, "form": 1}})
    assert AT._load()[k1]["block_size"] == 16


@pytest.mark.gpu
def test_tune_plan_and_batch_on_the_gpu(tmp_path, monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1002_2469_gb300 import autotune as AT
    monkeypatch.setattr(AT, "CACHE", str(tmp_path / "tune.json"))
    t, N = (-1.2, 2.5, -0.8), 1 << 20
    best = AT.tune(t, N, candidates=[(64, 16), (128, 16), (128, 24)])
    assert best["threads"] in (64, 128) and best["ms"] > 0
    assert AT.tuned_opts(t, N)["block_size"] == best["block_size"]
    plan = AT.plan(t, N)
    assert plan.info["threads"] == best["threads"]
    F = np.random.default_rng(0).standard_normal(N)
    x = plan.solve(torch.from_numpy(F).cuda()).cpu().numpy()
    ref = oracle.thomas(t, F)
    assert np.max(np.abs(x - ref)) / np.max(np.abs(ref)) < 1e-12
    Ns = np.array([1000, 5000, 70000, 3])
    tb = AT.tune_batch(Ns, np.full(4, -1.0), np.full(4, 3.0), np.full(4, -0.7), candidates=[(0, 0), (64, 16)])
    assert tb["ms"] > 0
