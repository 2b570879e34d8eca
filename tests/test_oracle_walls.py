"""Pins of the oracle's no-slip walls (Sec. 3.7, boundary conditions) and of
the dipole-wall set-up (Sec. 4.1), against closed forms that do not go
through the oracle's formulas:

* the slowest Stokes mode of a channel between two walls, u_x = sin(pi y / H),
  decays at the rate nu pi^2 / H^2 (nu = c_s^2 (tau - 1/2));
* the rest state is a fixed point of the walls in closed boxes;
* the dipole of eq_dipole1 / eq_dipole2 has kinetic energy 2 and enstrophy
  800 on [-1, 1]^2 (integrals of the analytic fields by quadrature here); the
  oracle's initial state, kinetic energy and wall-aware enstrophy must match.
"""
import numpy as np
import pytest

import oracle as O
from paper_1505_06900_gb300 import workloads as W


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q27, O.D3Q19])
def test_channel_wave_decays_at_the_stokes_rate(lattice):
    H, tau = 32, 0.8
    D = 2 if lattice == O.D2Q9 else 3
    shape = (4, H + 1, 1 if D == 2 else 2)
    rho, u = W.channel_wave(*shape, u0=0.01, dims=D)
    f = O.init(lattice, shape, tau, rho, u, walls=2)
    mode = np.sin(np.pi * np.arange(H + 1) / H)
    steps, amps, done = [200, 400, 600, 800], [], 0
    for s in steps:
        f = O.step(lattice, shape, tau, f, s - done, walls=2)
        done = s
        _, uu, _ = O.fields(lattice, shape, f, walls=2)
        prof = uu[0, 0, :, 0]
        assert abs(prof[0]) < 1e-15 and abs(prof[-1]) < 1e-15  # no slip on the wall nodes
        amps.append(np.dot(prof, mode) / np.dot(mode, mode))
    rate = -np.polyfit(steps, np.log(amps), 1)[0]
    expected = (tau - 0.5) / 3.0 * np.pi ** 2 / H ** 2
    assert abs(rate / expected - 1.0) < 1e-3, rate / expected - 1.0


@pytest.mark.parametrize("lattice,shape,walls", [(O.D2Q9, (5, 6, 1), 3),
                                                 (O.D3Q27, (4, 5, 3), 7),
                                                 (O.D3Q27, (4, 5, 3), 5),
                                                 (O.D3Q19, (4, 5, 3), 7)])
def test_rest_state_is_a_fixed_point_of_the_walls(lattice, shape, walls):
    D = 2 if lattice == O.D2Q9 else 3
    nx, ny, nz = shape
    f = O.init(lattice, shape, 0.7, np.ones((nz, ny, nx)), np.zeros((D, nz, ny, nx)),
               walls=walls)
    g = O.step(lattice, shape, 0.7, f, 5, walls=walls)
    r, u, p = O.fields(lattice, shape, g, walls=walls)
    assert np.abs(r - 1.0).max() < 1e-14
    assert np.abs(u).max() < 1e-15 and np.abs(p).max() < 1e-15


def test_dipole_initial_energy_and_enstrophy():
    N = 125
    m = 2001
    X = np.linspace(-1.0, 1.0, m)
    x, y = np.meshgrid(X, X)
    ux, uy = W.dipole_velocity(x, y)
    # vorticity of each Gaussian monopole: +-omega_e (1 - r^2/r0^2) exp(-r^2/r0^2)
    (x1, y1), (x2, y2) = W.DIPOLE_CENTRES
    s1 = ((x - x1) ** 2 + (y - y1) ** 2) / W.DIPOLE_R0 ** 2
    s2 = ((x - x2) ** 2 + (y - y2) ** 2) / W.DIPOLE_R0 ** 2
    om = W.DIPOLE_OMEGA_E * ((1 - s1) * np.exp(-s1) - (1 - s2) * np.exp(-s2))
    wq = np.ones(m)
    wq[0] = wq[-1] = 0.5
    Wq = np.outer(wq, wq) * (2.0 / (m - 1)) ** 2
    E_exact = 0.5 * np.sum(Wq * (ux ** 2 + uy ** 2))
    Om_exact = 0.5 * np.sum(Wq * om ** 2)
    assert abs(E_exact - 2.0) < 1e-5 and abs(Om_exact - 800.0) < 1e-2  # Clercx normalisation

    u_lb = W.dipole_u_lb(N)
    rho, u = W.dipole_2d(N)
    n = 2 * N + 1
    shape = (n, n, 1)
    f = O.init(O.D2Q9, shape, W.dipole_tau(N), rho, u, walls=3)
    E = O.diagnostics(O.D2Q9, shape, f, walls=3)[-1] / u_lb ** 2 / N ** 2
    Om = O.enstrophy(O.D2Q9, shape, f, walls=3) / u_lb ** 2
    assert abs(E / E_exact - 1.0) < 1e-5
    # second-order differences on 12.5 nodes per monopole radius
    assert abs(Om / Om_exact - 1.0) < 0.015, Om / Om_exact - 1.0
