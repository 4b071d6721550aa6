"""The step kernel's tile geometry, read on the CPU from the kernel's own templates by a host harness
compiled with nvcc: the ring cells that the ring phase evaluates (turbulent relaxation time and
limited slopes of the tile and its first halo ring) are exactly the cells that the tile's faces read,
each once, and the face counts that the tile shapes were chosen for hold."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1302_2132_gb300", "csrc")
SO = os.path.join(HERE, "_build", "libtile_host.so")

TILES = [(1, v) for v in range(3)] + [(2, v) for v in range(9)] + [(3, v) for v in range(4)]


@pytest.fixture(scope="module")
def harness():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = os.path.join(HERE, "tile_host_harness.cu")
    hdrs = [os.path.join(CSRC, f) for f in ("gks_step.cuh", "gks_flux.cuh")]
    os.makedirs(os.path.dirname(SO), exist_ok=True)
    if not os.path.exists(SO) or os.path.getmtime(SO) < max(os.path.getmtime(f) for f in [src] + hdrs):
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1",
                               "-Xcompiler", "-fPIC", "-shared", "-I", CSRC, "-o", SO + ".tmp", src])
        os.replace(SO + ".tmp", SO)
    L = ctypes.CDLL(SO)
    P = ctypes.POINTER(ctypes.c_int)
    L.tile_info.argtypes = [ctypes.c_int, ctypes.c_int, P]
    L.tile_ring_slots.argtypes = [ctypes.c_int, ctypes.c_int, P]
    return L


def info(L, D, V):
    o = (ctypes.c_int * 13)()
    assert L.tile_info(D, V, o) == 13
    keys = ["X", "Y", "Z", "T", "RX", "RY", "RZ", "NR", "NFX", "NFY", "NFZ", "NF", "NU"]
    return dict(zip(keys, list(o)))


def ring_slots(L, D, V, nr):
    o = (ctypes.c_int * nr)()
    n = L.tile_ring_slots(D, V, o)
    assert 0 < n <= nr
    return np.array(list(o)[:n])


def cells_read_by_faces(D, t):
    """Ring-box indices of the two cells beside every face of the tile (ring coordinates: the tile's
    cell (i, j, k) is (i + 1, j + 1, k + 1) in the ring box), enumerated face by face."""
    X, Y, Z = t["X"], t["Y"], t["Z"]
    RX, RY = t["RX"], t["RY"]
    out = set()
    ext = [X, Y if D >= 2 else 1, Z if D >= 3 else 1]
    for a in range(D):
        n = list(ext)
        n[a] += 1  # faces along axis a: one more than cells
        for k in range(n[2]):
            for j in range(n[1]):
                for i in range(n[0]):
                    f = [i, j, k]
                    for side in (0, 1):  # the cell below the face and the cell above it
                        c = [f[0] + 1, f[1] + (1 if D >= 2 else 0), f[2] + (1 if D >= 3 else 0)]
                        c[a] += side - 1
                        out.add((c[2] * RY + c[1]) * RX + c[0])
    return out


@pytest.mark.parametrize("D,V", TILES)
def test_ring_phase_covers_the_cells_the_faces_read(harness, D, V):
    t = info(harness, D, V)
    assert t["RX"] == t["X"] + 2 and t["NR"] == t["RX"] * t["RY"] * t["RZ"]
    s = ring_slots(harness, D, V, t["NR"])
    assert len(s) == t["NU"]
    assert len(set(s.tolist())) == len(s), "a ring cell is evaluated twice"
    assert s.min() >= 0 and s.max() < t["NR"]
    need = cells_read_by_faces(D, t)
    if D == 3:
        # the 3D ring phase skips the edge and corner cells of the ring box: exactly the face cells
        assert set(s.tolist()) == need
        X, Y, Z, RX, RY = t["X"], t["Y"], t["Z"], t["RX"], t["RY"]
        ri, rj, rk = s % RX, (s // RX) % RY, s // (RX * RY)
        n0 = X * Y * Z
        assert np.all((ri[:n0] >= 1) & (ri[:n0] <= X) & (rj[:n0] >= 1) & (rj[:n0] <= Y)
                      & (rk[:n0] >= 1) & (rk[:n0] <= Z)), "tile cells come first"
        lay = [slice(n0, n0 + 2 * Y * Z), slice(n0 + 2 * Y * Z, n0 + 2 * Y * Z + 2 * X * Z),
               slice(n0 + 2 * Y * Z + 2 * X * Z, len(s))]
        for r, hi, sl in ((ri, X + 1, lay[0]), (rj, Y + 1, lay[1]), (rk, Z + 1, lay[2])):
            half = (sl.stop - sl.start) // 2
            assert np.all(r[sl][:half] == 0) and np.all(r[sl][half:] == hi), "x, y, z layers, low side first"
    else:
        # 1D and 2D evaluate the whole ring box, in order
        assert np.array_equal(s, np.arange(t["NR"]))
        assert need <= set(s.tolist())
        assert t["NR"] - len(need) == (4 if D == 2 else 0)  # only the 2D box corners are not read


@pytest.mark.parametrize("D,V,faces,threads", [
    (2, 0, 1007, 256), (2, 1, 967, 256), (2, 2, 2047, 512), (2, 3, 1787, 256), (2, 4, 1202, 256),
    (2, 5, 3547, 512), (2, 8, 1397, 256), (3, 1, 944, 256), (3, 2, 896, 256)])
def test_tile_face_counts(harness, D, V, faces, threads):
    t = info(harness, D, V)
    assert t["NF"] == faces and t["T"] == threads
    assert t["NF"] == t["NFX"] + t["NFY"] + t["NFZ"]
    if D == 2 and V in (0, 1, 2, 3, 5):
        # these shapes fill their rounds of one face per thread to at least 94% (32 x 21 is chosen for
        # whole waves instead: 91%)
        rounds = -(-faces // threads)
        assert faces / (rounds * threads) >= 0.94


@pytest.mark.parametrize("shape,D,V,tiles", [((1024, 1024), 2, 3, 1216), ((1024, 384), 2, 8, 608)])
def test_tile_counts_fill_whole_waves(harness, shape, D, V, tiles):
    """The 32 x 27 tile cuts a 1024^2 grid into four full waves of two CTAs on each of 152 SMs, the
    32 x 21 tile a 1024 x 384 grid into two."""
    t = info(harness, D, V)
    n = -(-shape[0] // t["X"]) * -(-shape[1] // t["Y"])
    assert n == tiles and n % (2 * 152) == 0
