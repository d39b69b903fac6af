"""slr_count_noalloc against slr_count (needs a GB300).

slr_count_noalloc serves callers that cannot allocate GPU memory once set up
(a framework's caching allocator holding the device memory, or a real-time
loop that must not stall on cudaMalloc/cudaFree): its scratch lives in a fixed
array inside the library.  Its
counts must equal those of the allocating entry point, on two calls in a row
(the array keeps the previous call's contents, so each call must clear it).
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import pytest

from workloads import generators as gen

pytestmark = pytest.mark.gpu

KEYS = ("unsafe_lo", "unsafe_hi", "boxes", "rechecked", "tie_leaves", "depth", "levels",
        "level_boxes", "level_safe", "level_unsafe", "level_undecided")


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2312_05890_gb300 as m
    return m


@pytest.mark.parametrize("name,D", [("tiny", 16), ("acas", 17), ("nav", 12)])
def test_noalloc_count_equals_count(pkg, name, D):
    p = gen.make(name)
    with pkg.Counter(0) as c:
        c.set_problem(p)
        want = c.count(D)                 # allocating entry; also puts the network on the device
        for _ in range(2):
            got = c.count_noalloc(D)
            assert {k: got[k] for k in KEYS} == {k: want[k] for k in KEYS}


def test_noalloc_needs_a_resident_network(pkg):
    p = gen.tiny(0)
    with pkg.Counter(0) as c:
        c.set_problem(p)
        with pytest.raises(pkg.SlrError) as ei:
            c.count_noalloc(8)
        assert ei.value.code == -4
        c.count(8)
        assert c.count_noalloc(8)["unsafe_hi"] == c.count(8)["unsafe_hi"]


def test_noalloc_rejects_a_frontier_beyond_its_scratch(pkg):
    p = gen.acas_shaped(0)          # level 19 holds about 500k boxes, above the fixed 262144
    with pkg.Counter(0) as c:
        c.set_problem(p)
        c.count(4)
        with pytest.raises(pkg.SlrError) as ei:
            c.count_noalloc(20)
        assert ei.value.code == -5 and "262144" in str(ei.value)
        # the array is usable again right after the failed call
        assert c.count_noalloc(12)["unsafe_hi"] == c.count(12)["unsafe_hi"]


@pytest.mark.parametrize("opt", [dict(alpha_steps=5), dict(precision=1), dict(recheck_cluster=1), dict(wide=1)])
def test_noalloc_refuses_options_it_does_not_run(pkg, opt):
    """Slope steps, the tensor-core contraction, the cluster re-check and the
    wide path would make slr_count count differently: the entry refuses them
    (SLR_EUNSUPPORTED) instead of returning the fixed-slope FP32 count."""
    p = gen.make("acas")
    with pkg.Counter(0) as c:
        c.set_problem(p)
        c.set_options(**opt)
        c.count(6)
        with pytest.raises(pkg.SlrError) as ei:
            c.count_noalloc(6)
        assert ei.value.code == -7


def test_noalloc_leaves_free_device_memory_unchanged(pkg):
    """After the first call, repeated calls leave the device's free memory as
    it was: the entry point allocates nothing."""
    torch = pytest.importorskip("torch")
    p = gen.make("acas")
    with pkg.Counter(0) as c:
        c.set_problem(p)
        want = c.count(16)
        c.count_noalloc(16)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info(0)
        for _ in range(3):
            got = c.count_noalloc(16)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info(0)
    assert free1 == free0, (free0, free1)
    assert {k: got[k] for k in KEYS} == {k: want[k] for k in KEYS}
