"""The FP64 re-check in two stages (float-float hidden products, then plain
FP64 products on what they leave undecided) against plain FP64 products and
the oracle (needs a GB300)."""
import pytest

from workloads import generators as gen

from .test_gpu_parity import _check_count, _counter, _margin_at_a_corner

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_05890_gb300 as m
    return m


def _both(pkg, p, D, **opt):
    """A count with recheck_pairs 1 and 0 on the same FP32 tile (the tile fixes
    which boxes reach the re-check)."""
    out = []
    tile = {}
    for pairs in (1, 0):
        with _counter(pkg, p, record_leaves=1, recheck_pairs=pairs, **tile, **opt) as c:
            r = c.count(D)
            leaves = sorted(zip(*[x.tolist() for x in c.leaves()]))
        tile = dict(tile_boxes=r["tile"][0], tile_threads=r["tile"][1])
        out.append((r, leaves))
    return out


_VOLATILE = ("device_ms", "kernel_ms", "h2d_bytes", "d2h_bytes", "launches", "rechecked_fp64")


@pytest.mark.parametrize("name,D", [("acas", 17), ("nav", 12), ("tiny", 16)])
def test_pairs_give_the_classes_of_plain_fp64(pkg, name, D):
    """Same statistics, bracket, ties and leaf set either way; on the
    ACAS-shaped net the float-float stage decides some of the boxes it is given."""
    (a, la), (b, lb) = _both(pkg, gen.make(name), D)
    assert la == lb
    assert {k: v for k, v in a.items() if k not in _VOLATILE} == {k: v for k, v in b.items() if k not in _VOLATILE}
    assert b["rechecked_fp64"] == b["rechecked"]
    assert a["rechecked_fp64"] <= a["rechecked"]
    if name == "acas":
        assert a["rechecked"] > 0
        assert a["rechecked_fp64"] < a["rechecked"]


def test_pairs_leave_tiny_margins_to_fp64(pkg):
    """Margins of 1e-12 lie inside the float-float bound (about 1e-10 relative):
    those boxes go on to the plain FP64 stage, which decides them as the
    oracle does (four-box float64 tiles: even input count)."""
    p = _margin_at_a_corner()
    got = _check_count(pkg, p, p.depth, recheck_pairs=1)
    assert got["rechecked"] > 0 and got["tie_leaves"] == 0
    assert 0 < got["rechecked_fp64"] <= got["rechecked"]


def test_cluster_recheck_reports_plain_fp64(pkg):
    """The cluster form has one stage: all its re-checked boxes use FP64 products."""
    with _counter(pkg, gen.acas_shaped(0), recheck_cluster=1, recheck_pairs=1) as c:
        r = c.count(14)
    assert r["rechecked_fp64"] == r["rechecked"]


def test_recheck_pairs_option_is_validated(pkg):
    with pytest.raises(pkg.SlrError):
        with _counter(pkg, gen.make("tiny"), recheck_pairs=2):
            pass
