"""Checkpoint and resume of a count at a level boundary, through the C ABI:
a count stopped after level t and resumed (in the same context or a fresh
one) gives the whole count's result, level by level."""
import pytest

from workloads import generators as gen

pytestmark = pytest.mark.gpu

# timings, copies and launches cover the resumed levels only
VOLATILE = ("device_ms", "kernel_ms", "h2d_bytes", "d2h_bytes", "launches", "alpha_ms", "gemm_ms",
            "gemm_launches", "gemm_flop")


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_05890_gb300 as m
    return m


def _strip(r):
    return {k: v for k, v in r.items() if k not in VOLATILE}


@pytest.mark.parametrize("name,D,ts", [("tiny", 16, (0, 7, 15)), ("acas", 14, (0, 9, 13)), ("nav", 10, (4,))])
def test_resume_gives_the_whole_count(pkg, name, D, ts):
    p = gen.make(name)
    with pkg.Counter(0) as c:
        c.set_problem(p)
        whole = c.count(D)
        tile = dict(tile_boxes=whole["tile"][0], tile_threads=whole["tile"][1])
        c.set_options(**tile)
        whole = _strip(c.count(D))
        for t in ts:
            state = c.checkpoint(D, t)
            assert _strip(c.resume(state)) == whole, t
            with pkg.Counter(0) as fresh:       # as after a restart
                fresh.set_problem(p)
                fresh.set_options(**tile)
                assert _strip(fresh.resume(state)) == whole, t


def test_resume_tensor_core_and_wide_paths(pkg):
    p = gen.make("acas")
    for opt in (dict(precision=pkg.PREC_TC_TF32), dict(wide=1)):
        with pkg.Counter(0) as c:
            c.set_problem(p)
            c.set_options(**opt)
            whole = _strip(c.count(10))
            state = c.checkpoint(10, 6)
            assert _strip(c.resume(state)) == whole, opt


def test_checkpoint_errors(pkg):
    p = gen.make("tiny")
    with pkg.Counter(0) as c:
        c.set_problem(p)
        state = c.checkpoint(12, 5)
        for bad in (state[:-8], state[:40], b"", b"x" * len(state)):
            with pytest.raises(pkg.SlrError) as ei:
                c.resume(bad)
            assert ei.value.code == -1
        for D, t in ((12, 12), (12, -1), (0, 0)):
            with pytest.raises(pkg.SlrError) as ei:
                c.checkpoint(D, t)
            assert ei.value.code == -1
        c.set_options(recheck_pairs=0)          # the one-stage re-check
        with pytest.raises(pkg.SlrError) as ei:
            c.resume(state)
        assert ei.value.code == -1
        c.set_options(relax_mode=1)             # another result option
        with pytest.raises(pkg.SlrError) as ei:
            c.resume(state)
        assert ei.value.code == -1
        c.set_options(record_leaves=1)
        with pytest.raises(pkg.SlrError) as ei:
            c.checkpoint(12, 5)
        assert ei.value.code == -7
    with pkg.Counter(0) as other:               # another problem
        other.set_problem(gen.make("acas"))
        with pytest.raises(pkg.SlrError) as ei:
            other.resume(state)
        assert ei.value.code == -1


def test_resume_runs_the_checkpoints_tile(pkg):
    """The FP32 tile decides the products' summation order (small tiles split
    their inputs over lanes), so a fresh context left to its own autotuner
    resumes with the checkpoint's tile and reproduces the count exactly."""
    p = gen.make("acas")
    D, t = 14, 8
    with pkg.Counter(0) as probe:
        probe.set_problem(p)
        tuned = tuple(probe.count(4)["tile"])
    forced = (8, 256) if tuned != (8, 256) else (16, 256)
    with pkg.Counter(0) as c:
        c.set_problem(p)
        c.set_options(tile_boxes=forced[0], tile_threads=forced[1])
        whole = _strip(c.count(D))
        state = c.checkpoint(D, t)
    with pkg.Counter(0) as fresh:
        fresh.set_problem(p)
        got = fresh.resume(state)
        assert tuple(got["tile"]) == forced
        assert _strip(got) == whole
        assert tuple(fresh.count(4)["tile"]) == tuned      # the context keeps its own tile afterwards
