"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, loads,
exports every entry point include/sllbm.h declares, and its host-side tables (velocity
set, precomputed streaming table = the uniform-mesh form of Psi_i) agree with the
oracle's independent departure search."""
import math
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2012_05537_gb300 import build as B
from paper_2012_05537_gb300 import sllbm as S

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "sllbm.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return S.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sllbm_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_entry_point_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_default_params_and_strerror(lib):
    p = S.sllbm_default_params()
    assert (p.Ma, p.Re, p.Pr, p.gamma, p.T0, p.rho0) == (0.5, 1600.0, 0.7, 1.4, 1.0, 1.0)
    assert p.storage == S.F32 and p.collide == 1 and p.tgv_C < 0
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert S.strerror(code) != "unknown error"
    assert S.strerror(-99) == "unknown error"


def test_library_velocity_set_equals_oracle(lib):
    xi, w = S.sllbm_velset_d3q45()
    xo, wo = O.velset()
    assert np.max(np.abs(xi - xo)) <= 1e-15
    assert np.max(np.abs(w - wo)) <= 1e-17


@pytest.mark.parametrize("p,cells,dt,direction", [(2, 8, 0.05, 0), (3, 16, 0.13, 1),
                                                  (4, 32, 0.021, 2), (4, 7, 0.9, 0),
                                                  (3, 64, 0.2, 2)])
def test_stream_table_matches_oracle_departure_search(lib, p, cells, dt, direction):
    """Row a0 (precompute): the library's per-(velocity, local node) cell shift and
    Lagrange weights equal the oracle's literal departure search in every cell."""
    h = 2 * math.pi / cells
    shift, wt = S.sllbm_stream_table(p, h, dt, direction)
    xi, _ = O.velset()
    g = O.Grid(cells=(cells, cells, cells), p=p, dt=dt)
    x = O.node_coords(g, direction)
    for c in (0, cells // 2, cells - 1):
        for a in range(p):
            for i in range(45):
                y = x[c * p + a] - dt * xi[i, direction]
                cf = math.floor(y / h)
                r = 2 * (y / h - cf) - 1
                assert cf - c == shift[i, a] or abs(r + 1) < 1e-9 or abs(r - 1) < 1e-9
                if cf - c == shift[i, a]:
                    assert np.allclose(wt[i, a], O.lagrange(p, r), atol=1e-12)


def test_stream_table_rejects_bad_arguments(lib):
    with pytest.raises(S.SllbmError):
        S.sllbm_stream_table(5, 0.1, 0.1, 0)
    with pytest.raises(S.SllbmError):
        S.sllbm_stream_table(3, -0.1, 0.1, 0)
