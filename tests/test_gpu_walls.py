"""No-slip walls (Sec. 3.7, boundary conditions) on the GPU, against the FP64
oracle, and the dipole-wall benchmark (Sec. 4.1) against the enstrophy peaks
the paper prints.

Populations that stream in from outside the domain are undefined on both
sides after an update (NaN in the oracle, stale values in the store), so the
element-wise comparisons cover the defined ones; the macroscopic fields
(which on a wall node are those of its closed state) are compared everywhere.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from _common import max_rel_to_weight, rel_l2, shifted
from paper_1505_06900_gb300 import binding as B
from paper_1505_06900_gb300 import dipole
from paper_1505_06900_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

VARIANT = {B.COLLIDE_RR: O.RR, B.COLLIDE_REG2: O.REG2, B.COLLIDE_BGK: O.BGK}

# (lattice, shape, walls): closed boxes (edges and corners), channels, and
# walls on other axes, with sizes that are not multiples of a block
CASES = [(O.D2Q9, (12, 9, 1), 3), (O.D2Q9, (10, 7, 1), 2), (O.D2Q9, (7, 11, 1), 1),
         (O.D3Q27, (8, 6, 5), 7), (O.D3Q27, (6, 7, 5), 2), (O.D3Q27, (5, 6, 7), 5),
         (O.D3Q19, (8, 6, 5), 7), (O.D3Q19, (5, 6, 7), 5)]


def defined(lattice, shape, walls):
    """[Q, nz, ny, nx] mask of the populations whose source node x - xi_i is
    inside the domain."""
    c, _ = O.lattice_tables(lattice)
    nx, ny, nz = shape
    dims = (nx, ny, nz)
    m = np.ones((c.shape[0], nz, ny, nx), bool)
    for i in range(c.shape[0]):
        for a in range(3):
            if (walls >> a) & 1 and c[i, a] != 0:
                idx = [slice(None)] * 3
                idx[2 - a] = 0 if c[i, a] == 1 else dims[a] - 1
                m[(i,) + tuple(idx)] = False
    return m


def d_of(lattice):
    return 2 if lattice == O.D2Q9 else 3


@pytest.mark.parametrize("lattice,shape,walls", CASES)
@pytest.mark.parametrize("collision", [B.COLLIDE_RR, B.COLLIDE_REG2, B.COLLIDE_BGK])
@pytest.mark.parametrize("nsteps", [1, 2])
def test_walled_updates_match_the_oracle(lattice, shape, walls, collision, nsteps):
    """From the same initial fields, nsteps updates (parity 0, then 1)."""
    D = d_of(lattice)
    tau = 0.63
    rho, u = W.as_f32(*W.random_field(shape, D, seed=17 + walls, a_rho=0.01, a_u=0.03))
    f = O.init(lattice, shape, tau, rho, u, variant=VARIANT[collision], walls=walls)
    f = O.step(lattice, shape, tau, f, nsteps, variant=VARIANT[collision], walls=walls)
    r_o, u_o, p_o = O.fields(lattice, shape, f, variant=VARIANT[collision], walls=walls)
    with B.Solver(lattice, shape, tau, collision=collision, walls=walls) as s:
        s.init_fields(torch.from_numpy(rho.astype(np.float32)).cuda(),
                      torch.from_numpy(u.astype(np.float32)).cuda())
        s.step(nsteps)
        df = s.populations().cpu().numpy().astype(np.float64)
        r_g, u_g, p_g = (t.cpu().numpy().astype(np.float64) for t in s.moments())
    m = defined(lattice, shape, walls)
    ref = shifted(lattice, f)
    assert max_rel_to_weight(lattice, np.where(m, df, 0.0), np.where(m, ref, 0.0)) <= 1e-6
    assert np.abs(r_g - r_o).max() <= 1e-6
    assert np.abs(u_g - u_o).max() <= 1e-6
    assert np.abs(p_g - p_o).max() <= 1e-6
    # no slip: the wall nodes report u = 0
    for a in range(D):
        if (walls >> a) & 1:
            first = [slice(None)] * 3
            first[2 - a] = 0
            assert np.all(u_g[(slice(None),) + tuple(first)] == 0.0)


@pytest.mark.parametrize("lattice", [O.D2Q9, O.D3Q27, O.D3Q19])
def test_channel_wave_decays_at_the_stokes_rate(lattice):
    """u_x = sin(pi y / H) between walls decays at nu pi^2 / H^2 (closed form)."""
    H, tau = 32, 0.8
    D = d_of(lattice)
    shape = (4, H + 1, 1 if D == 2 else 2)
    rho, u = W.as_f32(*W.channel_wave(*shape, u0=0.01, dims=D))
    mode = np.sin(np.pi * np.arange(H + 1) / H)
    amps, steps, done = [], [200, 400, 600, 800], 0
    with B.Solver(lattice, shape, tau, walls=B.WALL_Y) as s:
        s.init_fields(torch.from_numpy(rho.astype(np.float32)).cuda(),
                      torch.from_numpy(u.astype(np.float32)).cuda())
        for k in steps:
            s.step(k - done)
            done = k
            prof = s.moments()[1][0, 0, :, 0].cpu().numpy().astype(np.float64)
            amps.append(np.dot(prof, mode) / np.dot(mode, mode))
    rate = -np.polyfit(steps, np.log(amps), 1)[0]
    expected = (tau - 0.5) / 3.0 * np.pi ** 2 / H ** 2
    assert abs(rate / expected - 1.0) < 1e-3, rate / expected - 1.0


def test_dipole_run_matches_the_oracle():
    """300 updates of the dipole at N = 32 (tau = 0.5015, Ma ~ 0.7 peak)."""
    N, nsteps = 32, 300
    n = 2 * N + 1
    shape = (n, n, 1)
    tau = W.dipole_tau(N)
    rho, u = W.as_f32(*W.dipole_2d(N))
    f = O.init(O.D2Q9, shape, tau, rho, u, walls=3)
    f = O.step(O.D2Q9, shape, tau, f, nsteps, walls=3)
    r_o, u_o, _ = O.fields(O.D2Q9, shape, f, walls=3)
    en_o = O.enstrophy(O.D2Q9, shape, f, walls=3)
    with B.Solver(B.D2Q9, shape, tau, walls=3) as s:
        s.init_fields(torch.from_numpy(rho.astype(np.float32)).cuda(),
                      torch.from_numpy(u.astype(np.float32)).cuda())
        s.step(nsteps)
        r_g, u_g, _ = (t.cpu().numpy().astype(np.float64) for t in s.moments())
        en_g = s.enstrophy()
    assert rel_l2(u_g, u_o) <= 1e-5
    assert rel_l2(r_g, r_o) <= 1e-6
    assert abs(en_g / en_o - 1.0) <= 1e-4


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "dipole_wall_enstrophy.json")


@pytest.mark.parametrize("N,tol", [(500, 0.05), (1000, 0.01)])
def test_dipole_enstrophy_peaks_match_the_paper(N, tol):
    """The two enstrophy maxima of the dipole-wall collisions against the
    reference values printed in Sec. 4.1, at N = 500 (1001^2 nodes, 150,000
    updates to t = 0.75) and N = 1000 (2001^2 nodes, 600,000 updates)."""
    golden = json.load(open(GOLDEN))
    assert (W.DIPOLE_OMEGA_E, W.DIPOLE_R0, W.DIPOLE_RE) == (
        golden["omega_e"], golden["r0"], golden["re"])
    r = dipole.run(N, t_end=0.75)
    print({k: v for k, v in r.items() if k != "history"})
    assert abs(r["energy0"] - 2.0) < 1e-4
    assert abs(r["omega0"] / 800.0 - 1.0) < 2e-3
    (p1, p2) = r["peaks"]
    ref1, ref2 = golden["enstrophy_peaks"]
    assert 0.3 < p1["t"] < 0.36 and abs(p1["enstrophy"] / ref1 - 1.0) < tol
    assert 0.55 < p2["t"] < 0.7 and abs(p2["enstrophy"] / ref2 - 1.0) < tol


def test_dipole_at_mach_0_7_stays_stable_with_rr_only():
    """Sec. 4.1 runs the dipole at a peak Mach number of 0.7 (U_lb = 0.032,
    Re = 2500) with the recursive model; the order-2 regularized model of
    Sec. 3.8.1, whose shear modes the paper finds unstable at high velocity,
    blows up on the same run."""
    r = dipole.run(250, t_end=0.75, u_lb=0.032)
    assert all(np.isfinite(p["enstrophy"]) for p in r["peaks"])
    assert abs(r["peaks"][0]["enstrophy"] / 3313.0 - 1.0) < 0.2
    with pytest.raises(B.LBError):
        dipole.run(250, t_end=0.75, u_lb=0.032, collision=B.COLLIDE_REG2)
