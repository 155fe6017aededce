"""Local-refinement hierarchies from refined cell sets (the rebuild step of
the adaptive loop, Sec. 6.4): the builder reproduces the geometric hierarchy
exactly from its marks, and the closure makes an arbitrary marking admissible
(every neighbour of a refined cell is an element of its level, every frozen
element has a leaf parent, every active element a twig parent)."""
import numpy as np
import pytest

from paper_2608_14123_b300 import workloads as wl


def _spec():
    return wl.front_spec(np.random.default_rng(wl.SEED_BASE + 4))


@pytest.mark.parametrize("n_base,n_ref,n_root", [(4, 1, 2), (4, 2, 2), (8, 2, 4)])
def test_builder_reproduces_the_geometric_hierarchy(n_base, n_ref, n_root):
    spec = _spec()
    ref = wl.refined_hierarchy(spec, n_base=n_base, n_ref=n_ref, n_root=n_root)
    new = wl.hierarchy_from_marks(wl.geometric_marks(spec, n_base, n_ref), n_base=n_base, p=3,
                                  n_root=n_root)
    assert len(ref) == len(new)
    for a, b in zip(ref, new):
        for key in ("p", "shape", "corners", "nbr", "nbr27", "parent", "octant", "cls"):
            np.testing.assert_array_equal(np.asarray(a[key]), np.asarray(b[key]), err_msg=key)


def _check_classes(levels):
    for k in range(1, len(levels)):
        lv, up = levels[k], levels[k - 1]
        if lv["shape"] == up["shape"]:
            continue
        pc = up["cls"][lv["parent"]]
        frozen = lv["cls"] == wl.FROZEN
        assert np.all(pc[frozen] == wl.LEAF)
        assert np.all(pc[~frozen] == wl.TWIG)


def test_closure_makes_marks_admissible():
    n_base = 4
    # level 0 refines one cell; level 1 refines a child at the outer corner of
    # that cell, whose neighbours lie outside level 1
    marks = [{(1, 1, 1)}, {(3, 3, 3)}]
    with pytest.raises(AssertionError):
        wl.hierarchy_from_marks(marks, n_base=n_base, n_root=2)
    closed = wl.close_marks(marks, n_base)
    assert closed[1] == marks[1] and marks[0] < closed[0]
    # the added coarse cells are exactly the parents of the missing neighbours
    need = {((3 + ox) // 2, (3 + oy) // 2, (3 + oz) // 2)
            for ox in (-1, 0, 1) for oy in (-1, 0, 1) for oz in (-1, 0, 1)}
    assert closed[0] == {(1, 1, 1)} | need
    levels = wl.hierarchy_from_marks(closed, n_base=n_base, n_root=2)
    _check_classes(levels)
    # a closed set is a fixed point
    assert wl.close_marks(closed, n_base) == closed
