"""Adaptive sampling of the tuner's size buckets (host logic, no GPU): only
the buckets needed to locate where the best variant changes are timed."""
import pytest

tune = pytest.importorskip("paper_1405_2915_gb300.tune")


def run(truth):
    sizes = list(range(len(truth)))
    calls = []

    def decide(n):
        calls.append(n)
        return truth[n]

    got = tune.adaptive_sizes(sizes, decide, key=lambda r: r)
    filled, last = [], None
    for n in sizes:
        last = got[n] if got[n] is not None else last
        filled.append(last)
    return filled, calls


def test_constant_choice_samples_only_the_coarse_grid():
    filled, calls = run(["a"] * 10)
    assert filled == ["a"] * 10
    assert sorted(calls) == [0, 3, 6, 9]


@pytest.mark.parametrize("k", range(1, 10))
def test_one_change_point_is_located_exactly(k):
    truth = ["small"] * k + ["large"] * (10 - k)
    filled, calls = run(truth)
    assert filled == truth
    assert len(calls) <= 4 + 2          # the coarse grid plus a bisection of one stride
    assert len(set(calls)) == len(calls)  # no bucket timed twice


def test_several_changes_are_all_found():
    truth = ["d", "d", "v1", "v1", "v1", "v2", "v2", "d", "d", "d"]
    filled, calls = run(truth)
    assert filled == truth


def test_empty_and_single():
    assert tune.adaptive_sizes([], lambda n: 1, key=lambda r: r) == {}
    assert tune.adaptive_sizes([5], lambda n: "x", key=lambda r: r) == {5: "x"}


def test_grid_sides_keep_aligned_rows():
    """Both timing points of a 2D bucket (4^k and about 2 * 4^k points) are
    square grids with a multiple of 4 columns; the side is off sqrt(n) by at
    most 2, so the point count by at most 4 sqrt(n) + 4."""
    for k in range(5, 15):
        for n in (4 ** k, 2 * 4 ** k):
            side = tune.grid_side(n)
            assert side % 4 == 0
            assert abs(side * side - n) <= 4 * n ** 0.5 + 4
        assert tune.grid_side(4 ** k) == 2 ** k


def test_tuner_tries_every_variant_the_library_offers():
    """The off-line tuner's candidate list of each skeleton covers exactly the
    variants the library reports (a variant the tuner never times can never
    enter the execution-plan table)."""
    import paper_1405_2915_gb300 as sk
    for name in sk.SK:
        offered = set(range(sk.skel_variant_count(name)))
        tried = {c[0] for c in tune.candidates(name)}
        assert tried == offered, (name, sorted(tried), sorted(offered))
        assert all(sk.skel_variant_name(name, v) != "?" for v in offered)


def test_set_table_entry_replaces_or_adds_a_bucket(tmp_path):
    """The validation's re-decision rewrites exactly one bucket's line of the
    execution-plan table (or adds it when the bucket was extrapolated)."""
    p = tmp_path / "t.tbl"
    p.write_text("# header\n0 3 0 10 0 0 1 256 2 0\n0 3 0 11 0 0 3 256 4 0\n")
    tune.set_table_entry(str(p), (0, 3, 0, 10, 0, 0), (-1, 0, 0, 0))
    assert p.read_text().splitlines() == ["# header", "0 3 0 10 0 0 -1 0 0 0", "0 3 0 11 0 0 3 256 4 0"]
    tune.set_table_entry(str(p), (1, 0, 0, 9, 0, 0), (-1, 0, 0, 0))
    assert p.read_text().splitlines()[-1] == "1 0 0 9 0 0 -1 0 0 0"
