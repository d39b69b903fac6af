"""One count split into shards (every N-th subtree below a level g), run one
after another on one GPU: the shards' brackets add up to the whole count's
(needs a GB300)."""
import pytest

from workloads import generators as gen

pytestmark = pytest.mark.gpu

KEYS = ("unsafe_lo", "unsafe_hi")


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_05890_gb300 as m
    return m


def _count(pkg, p, D, **opt):
    with pkg.Counter(0) as c:
        c.set_problem(p)
        c.set_options(**opt)
        return c.count(D)


@pytest.mark.parametrize("name,D,g,N", [("acas", 14, 6, 3), ("acas", 14, 0, 2), ("acas", 14, 14, 4),
                                        ("tiny", 12, 3, 5), ("nav", 10, 4, 7), ("acas", 8, 2, 64)])
def test_shards_add_up(pkg, name, D, g, N):
    p = gen.make(name)
    whole = _count(pkg, p, D)
    parts = [_count(pkg, p, D, shard_count=N, shard_index=r, shard_level=g) for r in range(N)]
    assert sum(x["unsafe_lo"] for x in parts) == whole["unsafe_lo"]
    assert sum(x["unsafe_hi"] for x in parts) == whole["unsafe_hi"]
    for t in range(g, D + 1):
        assert sum(x["level_boxes"][t] for x in parts) == whole["level_boxes"][t]
        assert sum(x["level_unsafe"][t] for x in parts) == whole["level_unsafe"][t]
    for t in range(g):
        assert all(x["level_boxes"][t] == whole["level_boxes"][t] for x in parts)


def test_shards_on_the_wide_path_and_with_slopes(pkg):
    p = gen.make("acas")
    D, g, N = 10, 4, 3
    for opt in ({"wide": 1}, {"alpha_steps": 5}):
        whole = _count(pkg, p, D, **opt)
        parts = [_count(pkg, p, D, shard_count=N, shard_index=r, shard_level=g, **opt) for r in range(N)]
        for k in KEYS:
            assert sum(x[k] for x in parts) == whole[k], (opt, k)


def test_shard_options_checked(pkg):
    p = gen.make("tiny")
    with pkg.Counter(0) as c:
        c.set_problem(p)
        with pytest.raises(pkg.SlrError, match="EINVAL"):
            c.set_options(shard_count=2, shard_index=2, shard_level=3)
        c.set_options(shard_count=2, shard_index=1, shard_level=13)
        with pytest.raises(pkg.SlrError, match="EINVAL"):
            c.count(12)
        c.set_options(shard_count=2, shard_index=1, shard_level=3)
        c.count(12)
        with pytest.raises(pkg.SlrError, match="EUNSUPPORTED"):
            c.count_noalloc(12)
        with pytest.raises(pkg.SlrError, match="EUNSUPPORTED"):
            c.count_batch([p], [12])
