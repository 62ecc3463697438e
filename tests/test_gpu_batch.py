"""Batched fits (dia_fit_batch): many pairs of uneven sizes and kernel sides in
one persistent launch per iteration, each pair checked against the FP64
oracle's normal-equation optimum and against the same pair fitted alone."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_13715_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def nat():
    from paper_2104_13715_gb300 import native
    return native


def _check(theta, ref, sky):
    ek = np.max(np.abs(theta[:-1] - ref[:-1])) / abs(ref[:-1].sum())
    eb = abs(theta[-1] - ref[-1]) / sky
    assert ek <= TOL and eb <= TOL, (ek, eb)


def _pairs(n, seed, side=(64, 200), m_range=(7, 25)):
    specs = synth.batch_specs(n, seed, side=side, m_range=m_range)
    return [synth.make_pair(s, 1000 * seed + k) for k, s in enumerate(specs)]


def _dev(d):
    dev = torch.device("cuda")
    return dict(R=torch.from_numpy(d["R"]).to(dev), I=torch.from_numpy(d["I"]).to(dev), m=d["m"])


@pytest.mark.parametrize("precond", [1, 0])
def test_batch_matches_oracle_and_single_fits(nat, precond):
    ds = _pairs(14, seed=1)
    assert len({nat_m for nat_m in (d["m"] for d in ds)}) >= 4     # several kernel sides
    spec = nat.loss_spec(rho="gauss", noise="fixed", var=1.0)
    opts = (nat.default_opts(timeout_s=120.0) if precond else
            nat.default_opts(timeout_s=120.0, precond=0, history=100))
    out = nat.fit_batch([_dev(d) for d in ds], spec, opts, want_diff=True)
    for k, d in enumerate(ds):
        assert out["infos"][k]["precond_used"] == precond
        th = out["thetas"][k].cpu().numpy()
        ref = oracle.normal_solve(d["R"], d["I"], d["m"])
        sky = float(np.median(d["I"]))
        _check(th, ref, sky)
        assert out["infos"][k]["status"] == 0
        D = out["diffs"][k].cpu().numpy()
        Do = oracle.diff_image(d["R"], d["I"], d["m"], th)
        assert np.max(np.abs(D - Do)) <= 1e-5 * np.max(np.abs(d["I"]))
    # the same pairs one at a time through the plain (non-graph) single-pair path
    plain = nat.default_opts(use_graph=0)
    for k in (0, 5, 9):
        d = ds[k]
        o = nat.fit(_dev(d)["R"], _dev(d)["I"], d["m"], spec, plain)
        _check(o["theta"].cpu().numpy(), oracle.normal_solve(d["R"], d["I"], d["m"]),
               float(np.median(d["I"])))


def test_batch_with_degenerate_pair(nat):
    ds = _pairs(4, seed=2, side=(64, 96), m_range=(7, 11))
    items = [_dev(d) for d in ds]
    items[2]["mask"] = torch.zeros_like(items[2]["R"], dtype=torch.uint8)
    spec = nat.loss_spec(rho="gauss", noise="fixed", var=1.0)
    out = nat.fit_batch(items, spec, nat.default_opts(timeout_s=120.0))
    assert out["infos"][2]["status"] == nat.DIA_ERR_DEGENERATE
    for k in (0, 1, 3):
        d = ds[k]
        _check(out["thetas"][k].cpu().numpy(), oracle.normal_solve(d["R"], d["I"], d["m"]),
               float(np.median(d["I"])))


def test_batch_nonlinear_loss(nat):
    """CCD negative log-likelihood in a batch: each pair at its FP64 Newton optimum."""
    ds = _pairs(5, seed=3, side=(80, 150), m_range=(7, 15))
    spec_d = dict(rho="gauss", noise="ccd", sigma0=5.0, gain=1.0, var_floor=1e-6)
    out = nat.fit_batch([_dev(d) for d in ds], nat.loss_spec(**spec_d),
                        nat.default_opts(timeout_s=120.0))
    for k, d in enumerate(ds):
        th = out["thetas"][k].cpu().numpy()
        ref = oracle.newton(d["R"], d["I"], d["m"], th,
                            oracle.LossSpec("gauss", "ccd", sigma0=5.0, gain=1.0))
        _check(th, ref, float(np.median(d["I"])))


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_every_work_item_variant_matches_the_oracle(nat, variant):
    """Each work-item size (tiles per item, per kernel-side group) gives the
    oracle's normal-equation optimum for every pair of an uneven batch."""
    ds = _pairs(9, seed=4, side=(64, 300), m_range=(3, 31))
    items = [_dev(d) for d in ds]
    spec = nat.loss_spec(rho="gauss", noise="fixed", var=1.0)
    try:
        for g in range(4):
            nat.select_batch_variant(g, variant)
        out = nat.fit_batch(items, spec, nat.default_opts(timeout_s=300.0))
    finally:
        for g in range(4):
            nat.select_batch_variant(g, 0)
    for d, th, info in zip(ds, out["thetas"], out["infos"]):
        assert info["status"] == 0, info
        _check(th.cpu().numpy(), oracle.normal_solve(d["R"], d["I"], d["m"]),
               float(np.median(d["I"])))


def test_converged_pairs_leave_the_work_list(nat):
    """A batch where one pair needs many more iterations than the others: the
    result is the same as the pair fitted in a batch of its own (the pairs
    that finished early drop out of the evaluation queue without changing
    anyone's arithmetic)."""
    ds = _pairs(6, seed=7, side=(64, 160), m_range=(7, 15))
    items = [_dev(d) for d in ds]
    spec = nat.loss_spec(rho="gauss", noise="fixed", var=1.0)
    opts = nat.default_opts(timeout_s=300.0)
    out = nat.fit_batch(items, spec, opts)
    evals = [f["evals"] for f in out["infos"]]
    k = int(np.argmax(evals))
    assert max(evals) > min(evals)
    alone = nat.fit_batch([items[k]], spec, opts)
    assert alone["infos"][0]["evals"] == evals[k]
    assert torch.equal(alone["thetas"][0], out["thetas"][k])


def test_batch_autotune_selects_and_caches(tmp_path):
    from paper_2104_13715_gb300 import autotune
    from paper_2104_13715_gb300 import native as nat
    ds = _pairs(6, seed=3, side=(64, 160), m_range=(7, 17))
    items = [_dev(d) for d in ds]
    spec = nat.loss_spec(rho="gauss", noise="fixed", var=1.0)
    path = str(tmp_path / "tb.json")
    try:
        rec = autotune.tune_batch(items, spec, iters=8, cache_path=path)
        for g, r in rec.items():
            assert r["variant"] == int(np.argmin(r["times_ms"]))
            assert nat.lib.dia_get_batch_variant(g) == r["variant"]
        rec2 = autotune.tune_batch(items, spec, iters=8, cache_path=path)
        assert {g: r["variant"] for g, r in rec2.items()} == {g: r["variant"] for g, r in rec.items()}
    finally:
        for g in range(4):
            nat.select_batch_variant(g, 0)


def test_batch_eval_timing_leaves_the_fit_unchanged(nat):
    """dia_set_batch_eval_timing: the timed launches of each group's evaluation
    kernel (before the first iteration) change no result bit; every group with
    pairs reports a positive time and exactly sum 4 m^2 (valid px) flop, the
    others zero; reps outside [0, 1000] are rejected."""
    ds = _pairs(10, seed=4, side=(64, 160), m_range=(5, 27))
    items = [_dev(d) for d in ds]
    spec = nat.loss_spec(rho="gauss", noise="fixed", var=1.0)
    opts = nat.default_opts(timeout_s=120.0)
    ref = nat.fit_batch(items, spec, opts)
    nat.set_batch_eval_timing(3)
    try:
        out = nat.fit_batch(items, spec, opts)
        bt = nat.batch_eval_timing()
    finally:
        nat.set_batch_eval_timing(0)
    for k in range(len(ds)):
        assert torch.equal(out["thetas"][k], ref["thetas"][k])
        assert out["infos"][k]["evals"] == ref["infos"][k]["evals"]
        assert out["infos"][k]["kernel_launches"] > ref["infos"][k]["kernel_launches"]
    group = lambda m: 0 if m <= 7 else 1 if m <= 15 else 2 if m <= 23 else 3
    flop = [0.0] * 4
    for d in ds:
        m, h = d["m"], d["m"] // 2
        flop[group(m)] += 4.0 * m * m * (d["R"].shape[0] - 2 * h) * (d["R"].shape[1] - 2 * h)
    for g in range(4):
        assert bt["flop"][g] == pytest.approx(flop[g], rel=1e-12)
        assert (bt["ms"][g] > 0.0) == (flop[g] > 0.0)
    with pytest.raises(nat.DiaError):
        nat.set_batch_eval_timing(-1)
    with pytest.raises(nat.DiaError):
        nat.set_batch_eval_timing(1001)
