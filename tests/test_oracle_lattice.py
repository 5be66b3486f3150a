"""Oracle pins: lattice tables, equilibrium and forcing moments (closed forms).

These check the oracle's building blocks against the paper's printed tables
and against moment identities that hold exactly for D3Q19 (c_s^2 = 1/3).
"""
import itertools

import numpy as np
import pytest

import oracle
from conftest import golden

CS2 = 1.0 / 3.0


def test_lattice_matches_printed_table():
    g = golden("d3q19_section2.txt")
    e, w, _ = oracle.lattice()
    assert np.array_equal(e[:, 0], np.array(g["ex"][0], dtype=int))
    assert np.array_equal(e[:, 1], np.array(g["ey"][0], dtype=int))
    assert np.array_equal(e[:, 2], np.array(g["ez"][0], dtype=int))
    assert np.allclose(w, g["w"][0], rtol=0, atol=1e-16)


def test_opposite_directions():
    e, _, opp = oracle.lattice()
    for i in range(19):
        assert np.array_equal(e[opp[i]], -e[i])
    # the diagonal pairs are not (2k-1, 2k)
    assert [opp[i] for i in (7, 8, 11, 12, 15, 16)] == [10, 9, 14, 13, 18, 17]


def test_isotropy_up_to_fourth_order():
    e, w, _ = oracle.lattice()
    e = e.astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, e), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, e, e), CS2 * np.eye(3), atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, e, e, e), 0.0, atol=1e-16)
    d = np.eye(3)
    iso4 = CS2 * CS2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                        + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e), iso4, atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(seed):
    """Eq. 2: zeroth, first and second moments are rho, rho u, rho (u u + c_s^2 I)."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.02, 1.5)
    u = rng.uniform(-0.1, 0.1, 3)
    e, _, _ = oracle.lattice()
    e = e.astype(float)
    f = oracle.feq(rho, u)
    assert abs(f.sum() - rho) < 1e-14
    assert np.allclose(e.T @ f, rho * u, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib->ab", f, e, e), rho * (np.outer(u, u) + CS2 * np.eye(3)), atol=1e-14)


@pytest.mark.parametrize("seed", range(5))
def test_forcing_moments(seed):
    """Eq. 9: sum S_i = 0, sum e_i S_i = F, sum e_i e_i S_i = u F + F u."""
    rng = np.random.default_rng(100 + seed)
    u = rng.uniform(-0.1, 0.1, 3)
    F = rng.uniform(-1e-2, 1e-2, 3)
    e, _, _ = oracle.lattice()
    e = e.astype(float)
    S = oracle.source(u, F)
    assert abs(S.sum()) < 1e-16
    assert np.allclose(e.T @ S, F, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", S, e, e), np.outer(u, F) + np.outer(F, u), atol=1e-16)


def test_mirror_map_matches_printed_left_boundary_rule():
    g = golden("physics_section3.txt")
    m = oracle.mirror_map(0)
    for a, b in g["mirror_x"]:
        assert m[int(a)] == int(b)


def test_mirror_map_reflects_normal_component():
    e, _, _ = oracle.lattice()
    for axis in range(3):
        m = oracle.mirror_map(axis)
        for i in range(19):
            r = e[i].copy()
            r[axis] = -r[axis]
            assert np.array_equal(e[m[i]], r)
    # z planes: the five outward directions map to the five inward ones
    mz = oracle.mirror_map(2)
    assert [mz[i] for i in (6, 13, 14, 17, 18)] == [5, 11, 12, 15, 16]


def test_all_pairs_distinct():
    e, _, _ = oracle.lattice()
    assert len({tuple(v) for v in e}) == 19
    assert all(sum(abs(c) for c in v) <= 2 for v in e)
    assert sum(1 for v, c in itertools.product(range(19), range(3)) if e[v][c] != 0) == 30
