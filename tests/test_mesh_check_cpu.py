"""Host-only mesh validation (dgfas_check_mesh, run first by
dgfas_setup_levels; no GPU needed): every workload the tests and the bench
use passes; a non-reciprocal face neighbour and an element whose local axes
are rotated against its neighbours' (the kernels read a neighbour through
its opposite face in the same face-local order) are rejected with
DGFAS_ERR_MESH, arrays out of range with DGFAS_ERR_INVALID."""
import ctypes

import numpy as np
import pytest

from paper_2608_14123_b300 import dgfas
from paper_2608_14123_b300 import workloads as wl


def _check(levels):
    lib = dgfas.load()
    keep = []
    arr = (dgfas.dgfas_level * len(levels))()
    for i, lv in enumerate(levels):
        ne = lv["nbr"].shape[0]
        a = [np.ascontiguousarray(lv["corners"], dtype=np.float64),
             np.ascontiguousarray(lv["nbr"], dtype=np.int32),
             np.ascontiguousarray(lv["nbr27"], dtype=np.int32),
             np.ascontiguousarray(lv["parent"], dtype=np.int32),
             np.ascontiguousarray(lv["octant"], dtype=np.int32),
             np.ascontiguousarray(lv["cls"], dtype=np.int8)]
        keep += a
        arr[i] = dgfas.dgfas_level(lv["p"], ne,
                                   a[0].ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   a[1].ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   a[2].ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   a[3].ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   a[4].ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   a[5].ctypes.data_as(ctypes.POINTER(ctypes.c_byte)))
    mesh = dgfas.dgfas_mesh(len(levels), arr, 1.0, 0.0)
    rc = lib.dgfas_check_mesh(ctypes.byref(mesh))
    msg = lib.dgfas_last_error()
    return rc, (msg.decode() if isinstance(msg, bytes) else str(msg))


@pytest.mark.parametrize("name,levels", [
    ("config1", lambda: wl.config(1)["levels"]),
    ("config2s", lambda: wl.config(2, small=True)["levels"]),
    ("config3s", lambda: wl.config(3, small=True)["levels"]),
    ("config5s-p1", lambda: wl.config(5, small=True, root="p1")["levels"]),
    ("config4s", lambda: wl.config4(small=True)["levels"]),
    ("periodic", lambda: wl.paper_cartesian_periodic(2, "h", n=4)["levels"]),
])
def test_workloads_pass(name, levels):
    rc, msg = _check(levels())
    assert rc == dgfas.DGFAS_OK, (name, msg)


def _level():
    V = wl.perturbed_vertices(2, 0.1, np.random.default_rng(3))
    return wl.level_from_vertices(V, 2, -1, False)


def test_non_reciprocal_neighbour_is_rejected():
    lv = _level()
    nbr = lv["nbr"].copy()
    e = 0
    f = int(np.nonzero(nbr[e] >= 0)[0][0])
    nb = nbr[e, f]
    nbr[nb, f ^ 1] = -1          # the neighbour no longer points back
    n27 = lv["nbr27"].copy()     # (its 27-neighbourhood kept consistent with that)
    g = f ^ 1
    d, o = g >> 1, 2 if g & 1 else 0
    n27[nb, [o + 12, 1 + 3 * o + 9, 4 + 9 * o][d]] = -1
    rc, msg = _check([dict(lv, nbr=nbr, nbr27=n27)])
    assert rc == dgfas.DGFAS_ERR_MESH and "point back" in msg


def test_rotated_local_axes_are_rejected():
    """Element 0 relabelled by a quarter turn about its z axis: the same
    hexahedron, but its local x face now lies where its neighbour expects
    another face."""
    lv = _level()
    cr = lv["corners"].copy()
    # new corner (i, j, k) takes the old corner (j, 1 - i, k)
    perm = [((c >> 1) & 1) | ((1 - (c & 1)) << 1) | (c & 4) for c in range(8)]
    cr[0] = lv["corners"][0][perm]
    rc, msg = _check([dict(lv, corners=cr)])
    assert rc == dgfas.DGFAS_ERR_MESH and "aligned local axes" in msg


def test_out_of_range_neighbour_is_invalid():
    lv = _level()
    nbr = lv["nbr"].copy()
    nbr[1, 0] = nbr.shape[0] + 5
    rc, _ = _check([dict(lv, nbr=nbr)])
    assert rc == dgfas.DGFAS_ERR_INVALID


def test_inconsistent_27_neighbourhood_is_invalid():
    """The Schwarz gather and combine read the 27-neighbourhood: its face
    slots must hold the face neighbours and its centre the element itself."""
    lv = _level()
    n27 = lv["nbr27"].copy()
    n27[0, 13] = 1
    rc, msg = _check([dict(lv, nbr27=n27)])
    assert rc == dgfas.DGFAS_ERR_INVALID and "centre" in msg
    n27 = lv["nbr27"].copy()
    f = int(np.nonzero(lv["nbr"][0] >= 0)[0][0])
    d, o = f >> 1, 2 if f & 1 else 0
    slot = [o + 12, 1 + 3 * o + 9, 4 + 9 * o][d]
    n27[0, slot] = -1
    rc, msg = _check([dict(lv, nbr27=n27)])
    assert rc == dgfas.DGFAS_ERR_INVALID and "disagrees" in msg
