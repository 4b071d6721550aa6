"""bench.py's accounting, checked on the CPU: the distinct faces of each workload's grid (n per grid
line along a periodic axis, whose wrap face is one face; n + 1 otherwise) and the algorithmic
operation count of one launch of the headline step, the numerator of the roofline's `achieved`."""
import itertools

import numpy as np
import pytest

import bench


def faces_brute(n, periodic):
    """Faces seen from every cell: each cell has a face on either side of it along every axis, keyed by
    the ordered pair (cell on its low side, cell on its high side); the outside of the grid stands in
    for the missing cell on a boundary, and a periodic axis wraps."""
    D = len(n)
    faces = set()
    for c in itertools.product(*[range(k) for k in n]):
        for d in range(D):
            for s in (-1, 1):
                m = list(c)
                m[d] += s
                if periodic[d]:
                    m[d] %= n[d]
                    other = tuple(m)
                elif 0 <= m[d] < n[d]:
                    other = tuple(m)
                else:
                    other = ("outside", s, c)
                faces.add((d, other, c) if s < 0 else (d, c, other))
    return len(faces)


@pytest.mark.parametrize("n,periodic", [((7,), [True]), ((7,), [False]), ((5, 3), [True, False]),
                                         ((4, 6), [False, True]), ((3, 4, 5), [True, True, True]),
                                         ((3, 4, 2), [False, True, False]), ((2, 2), [True, True])])
def test_faces_of_matches_brute_force(n, periodic):
    bc = [[0, 0] if p else [1, 1] for p in periodic]
    assert bench.faces_of(n, bc) == faces_brute(n, periodic)


def test_faces_of_the_bench_workloads():
    assert bench.faces_of((1024, 1024), [[0, 0], [0, 0]]) == 2_097_152
    assert bench.faces_of((256, 256, 256), [[0, 0]] * 3) == 3 * 256 ** 3
    assert bench.faces_of((1024, 384), [[3, 4], [2, 3]]) == 787_840
    assert bench.faces_of((400,), [[1, 1]]) == 401


def test_headline_operations_per_launch():
    """1674 operations per distinct face (2D, multi-dimensional, MUSCL-2) and 168 per cell: 3.687e9
    per launch of the 1024^2 step, the figure that the bench's `achieved` divides by the launch time."""
    from paper_1302_2132_gb300 import gks
    per_face = sum(gks.face_op_count(2, True, True)[:3]) + sum(gks.recon_op_count(2, "muscl2")[:3])
    per_cell = bench.CELL_OPS + sum(gks.cell_op_count(2)[:3])
    assert (per_face, per_cell) == (1674, 168)
    ops = bench.faces_of((1024, 1024), [[0, 0], [0, 0]]) * per_face + 1024 * 1024 * per_cell
    assert ops == 3_686_793_216
    assert np.isclose(ops / 119.10e-6 / 1e12, 30.955, rtol=1e-4)  # the default bench line: 119.10 us
