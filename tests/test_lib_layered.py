"""The library's set-up of the AIM grid step inside a layer of a stratified background
(bem_layered_grid_tables, host code: Table I's layered media) against the oracle
(oracle/layered.py) and, over a ground plane, against image theory in closed form. No GPU."""
import math

import numpy as np
import pytest

from oracle import layered as L, operators as op
from paper_2108_03991_gb300 import api, build

KINDS = ((0, "xx"), (1, "zz"), (2, "phi"))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return api.lib()


@pytest.mark.parametrize("kind,name", KINDS)
def test_tables_match_the_oracle(lib, kind, name):
    """A lossy three-layer stack on a ground plane under air, full wave (20 THz, k0 R ~ 1):
    both the Toeplitz and the Hankel tables to 1e-11 of their largest entry."""
    freq = 2e13
    layers = [(1.0, 4.0 - 0.2j), (2.0, 2.2), (0.7, 11.9 - 3j)]
    origin, h, n = (0.1, -0.3, 1.2), (0.4, 0.5, 0.3), (5, 4, 4)
    T, H = api.layered_grid_tables(layers, freq, origin, h, n, kind)
    g = L.LayeredGrid(L.Stack(op.k0_of(freq), layers, top_eps=1.0), name, origin, h, n)
    assert np.max(np.abs(T - g.T)) < 1e-11 * np.max(np.abs(g.T))
    assert np.max(np.abs(H - g.H)) < 1e-11 * np.max(np.abs(g.H))


@pytest.mark.parametrize("kind,sign", [(0, -1.0), (1, 1.0), (2, -1.0)])
def test_ground_plane_is_image_theory(lib, kind, sign):
    """One lossy layer of the top medium on the ground plane: T is the free-space kernel at the
    layer's wavenumber and H the image term, -G(R_i) for x, y and charges, +G(R_i) for z, in
    closed form."""
    freq, eps = 3e13, 3.0 - 0.1j
    origin, h, n = (0.0, 0.0, 0.4), (0.3, 0.35, 0.25), (4, 3, 3)
    T, H = api.layered_grid_tables([(2.0, eps)], freq, origin, h, n, kind, top_eps=eps)
    k = op.k0_of(freq) * np.sqrt(eps)
    k = -k if k.imag > 0 else k
    nx, ny, nz = n
    dx, dy = np.meshgrid(np.arange(nx) * h[0], np.arange(ny) * h[1], indexing="xy")
    rho = np.hypot(dx, dy)
    for r in range(2 * nz - 1):
        R = np.hypot(rho, (r - (nz - 1)) * h[2])
        with np.errstate(divide="ignore", invalid="ignore"):
            ref = np.where(R > 0, np.exp(-1j * k * R) / (4 * math.pi * R), 0.0)
        assert np.max(np.abs(T[r] - ref)) < 1e-11 * np.max(np.abs(T))
        Ri = np.hypot(rho, 2 * origin[2] + r * h[2])
        refh = sign * np.exp(-1j * k * Ri) / (4 * math.pi * Ri)
        assert np.max(np.abs(H[r] - refh)) < 1e-11 * np.max(np.abs(H))


def test_table_one_bus_stack(lib):
    """Table I's bus background at 10 GHz (lossy silicon, oxide, air), a grid in the oxide."""
    freq = 1e10
    layers = [(495.0, op.eps_rc(10.0, freq, 11.9)), (30.0, 4.0)]
    origin, h, n = (0.0, 0.0, 500.0), (5.0, 5.0, 4.0), (4, 3, 4)
    g = L.LayeredGrid(L.Stack(op.k0_of(freq), layers, top_eps=1.0), "phi", origin, h, n)
    T, H = api.layered_grid_tables(layers, freq, origin, h, n, 2)
    assert np.all(np.isfinite(T)) and np.all(np.isfinite(H))
    assert np.max(np.abs(T - g.T)) < 1e-10 * np.max(np.abs(g.T))
    assert np.max(np.abs(H - g.H)) < 1e-10 * np.max(np.abs(g.H))


def test_errors(lib):
    layers = [(1.0, 4.0), (2.0, 2.2)]
    with pytest.raises(api.BemError) as ei:   # node planes across the interface at z = 1
        api.layered_grid_tables(layers, 1e10, (0, 0, 0.8), (0.3, 0.3, 0.3), (3, 3, 3), 0)
    assert ei.value.code == -3
    with pytest.raises(api.BemError) as ei:
        api.layered_grid_tables([(0.0, 4.0)], 1e10, (0, 0, 0.1), (0.3, 0.3, 0.3), (3, 3, 1), 0)
    assert ei.value.code == -1
    with pytest.raises(api.BemError) as ei:
        api.layered_grid_tables(layers, 1e10, (0, 0, 1.5), (0.3, 0.3, 0.3), (3, 3, 2), 3)
    assert ei.value.code == -1


@pytest.mark.parametrize("kind,name", KINDS)
def test_kernel_tables_match_the_oracle(lib, kind, name):
    """The reflected parts at arbitrary (rho, z - z') and (rho, z + z') points, the tables the
    near-region entries of objects inside a layer interpolate: 1e-11 of the largest entry, in
    the middle layer of the lossy three-layer stack."""
    freq = 2e13
    layers = [(1.0, 4.0 - 0.2j), (2.0, 2.2), (0.7, 11.9 - 3j)]
    st = L.Stack(op.k0_of(freq), layers, top_eps=1.0)
    rho = np.linspace(0.0, 2.7, 11)
    for part, arg in ((0, np.linspace(-1.7, 1.7, 7)), (1, np.linspace(2.3, 5.7, 7))):
        got = api.layered_kernel_table(layers, freq, 1, kind, part, rho, arg)
        # the layer: z from 1 to 3 um (thickness 2); decay of each row's reflected terms
        zeta = [min(a - 2 * 1.0, 2 * 3.0 - a) if part == 1 else 2 * 2.0 - abs(a) for a in arg]
        ref = np.stack([st.sommerfeld(lambda kr, a=a: st.spectral(1, kr, "TH"[part], a, name),
                                      rho, z) for a, z in zip(arg, zeta)])
        assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def test_kernel_table_rejects_points_outside_the_layer(lib):
    layers = [(1.0, 4.0), (2.0, 2.2)]
    for part, arg in ((0, [2.5]), (1, [1.5])):
        with pytest.raises(api.BemError) as ei:
            api.layered_kernel_table(layers, 1e10, 1, 0, part, [0.0, 1.0], arg)
        assert ei.value.code == -1
