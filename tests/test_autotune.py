"""The tile autotuner: it times every variant, selects the fastest, caches the
choice per (GPU, kernel side, image size, variant table) and reuses it."""
import json

import numpy as np
import pytest
import torch


class _FakeNative:
    """Stand-in for the binding: a table of variants; evaluations are only
    recorded, so the test can see whether any timing ran."""

    def __init__(self, costs):
        self.costs = costs
        self.selected = {}
        self.calls = []

    def kernel_variants(self, m):
        return len(self.costs)

    def kernel_variant_desc(self, m, v=-1):
        return {"warps": 8, "rows_per_warp": 4 + v, "tile_rows": 32 + 8 * v, "smem_bytes": 1000 + v}

    def select_kernel_variant(self, m, v):
        self.selected[m] = v

    def workspace(self, *a, **k):
        return None

    def loss_grad(self, *a, **k):
        self.calls.append(self.selected[a[2]])


def test_cache_key_reuse_and_table_change(tmp_path, monkeypatch):
    """CPU: a cached choice is reused without timing; a different variant
    table (rebuilt library) or image size gives a new key."""
    from paper_2104_13715_gb300 import autotune
    fake = _FakeNative([1.0, 0.5, 2.0])
    monkeypatch.setattr(autotune, "nat", fake)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda dev=None: "FakeGPU")
    path = str(tmp_path / "t.json")
    key = autotune._key(25, 4096, 4096, None)
    assert key.startswith("FakeGPU|m=25|4096x4096|")
    autotune._save({key: {"variant": 2, "times_ms": [3, 2, 1]}}, path)
    R = torch.zeros((4096, 4096))
    rec = autotune.tune(R, R, 25, None, cache_path=path)
    assert rec["variant"] == 2 and fake.selected[25] == 2 and fake.calls == []
    # another image size is a different key
    assert autotune._key(25, 2048, 2048, None) != key
    # a rebuilt table (different shapes) is a different key
    fake.kernel_variant_desc = lambda m, v=-1: {"warps": 12, "rows_per_warp": v}
    assert autotune._key(25, 4096, 4096, None) != key
    assert list(json.load(open(path))) == [key]


@pytest.mark.gpu
def test_tune_selects_the_fastest_and_caches(tmp_path):
    """GPU: every variant is timed, the minimum is selected and written to
    the cache; a second call returns the cached record without timing."""
    from paper_2104_13715_gb300 import autotune
    from paper_2104_13715_gb300 import native as nat
    from tests._helpers import field
    m = 11
    d = field(600, 700, m, seed=5)
    dev = torch.device("cuda")
    R = torch.from_numpy(d["R"]).to(dev)
    I = torch.from_numpy(d["I"]).to(dev)
    spec = nat.loss_spec()
    path = str(tmp_path / "tune.json")
    prev = nat.kernel_variant_desc(m)
    try:
        rec = autotune.tune(R, I, m, spec, cache_path=path, reps=2)
        nv = nat.kernel_variants(m)
        assert len(rec["times_ms"]) == nv
        assert rec["variant"] == int(np.argmin(rec["times_ms"]))
        assert nat.kernel_variant_desc(m) == nat.kernel_variant_desc(m, rec["variant"])
        cached = json.load(open(path))
        assert list(cached.values())[0]["variant"] == rec["variant"]
        # the second call reads the cache: no evaluation may run
        real = nat.loss_grad
        nat.loss_grad = lambda *a, **k: (_ for _ in ()).throw(AssertionError("timed again"))
        try:
            rec2 = autotune.tune(R, I, m, spec, cache_path=path)
        finally:
            nat.loss_grad = real
        assert rec2["variant"] == rec["variant"]
    finally:
        for v in range(nat.kernel_variants(m)):
            if nat.kernel_variant_desc(m, v) == prev:
                nat.select_kernel_variant(m, v)
                break
