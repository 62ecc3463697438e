"""The generated kernel-instantiation units and dispatch table are those the
variant table of csrc/gen_instances.py produces, and the packed-FMA twin pairs
that tests/test_gpu_loss_grad.py compares bit for bit name the same tile shape
(host-only: no GPU)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2104_13715_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_instances",
                                                  os.path.join(CSRC, "gen_instances.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_generated_units_match_the_variant_table(tmp_path):
    gen = _gen()
    gen.main(str(tmp_path))
    made = sorted(os.listdir(tmp_path))
    committed = sorted(f for f in os.listdir(CSRC)
                       if (f.startswith("dia_eval_m") and f.endswith(".cu")) or f == "dia_dispatch.cu")
    assert made == committed
    for f in made:
        with open(os.path.join(tmp_path, f)) as a, open(os.path.join(CSRC, f)) as b:
            assert a.read() == b.read(), f
    # every kernel side of the tiled kernel has a variant list, each group once
    sides = [m for g in gen.GROUPS for m in g]
    assert sorted(sides) == sorted(gen.VARIANTS) == list(range(1, 32, 2))


def test_packed_twin_pairs_share_their_tile_shape():
    from tests.test_gpu_loss_grad import F2_TWINS
    variants = _gen().VARIANTS
    for m, pairs in F2_TWINS.items():
        for a, b in pairs:
            va, vb = variants[m][a], variants[m][b]
            f2 = lambda t: t[4] if len(t) > 4 else 0
            assert va[:4] == vb[:4], (m, a, b)
            assert f2(va) == 0 and f2(vb) == 1, (m, a, b)
