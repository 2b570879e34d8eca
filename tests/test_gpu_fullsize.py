"""Parity at the benchmark's full size: D3Q27 (and D3Q19), FP32 store, 512^3
cells, the same kernels and launch configuration that bench.py times.

The oracle cannot update 134M cells, so sampled cells are checked one by one:
after one update the population i of cell x must equal the oracle's collision
of cell x - xi_i; after two updates, the oracle's collision of the cells
around x - xi_i composed twice. Samples include the periodic corners and
edges. Global mass and momentum are checked at every size (conservation)."""
import numpy as np
import pytest

import oracle as O
from paper_1505_06900_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = 512
TAU = W.taylor_green_3d_tau(N, 0.1, 1600.0)  # the benchmark's relaxation time


@pytest.mark.parametrize("lattice", [O.D3Q27, O.D3Q19])
def test_sampled_cells_at_512_cubed(lattice):
    from paper_1505_06900_gb300 import binding as B
    c, w = O.lattice_tables(lattice)
    q = len(w)
    free = torch.cuda.mem_get_info()[0]
    need = 3 * q * N ** 3 * 4
    if free < need * 1.2:
        pytest.skip(f"needs {need / 1e9:.0f} GB of free device memory")
    gen = torch.Generator(device="cuda").manual_seed(1234)
    wt = torch.tensor(w, dtype=torch.float32, device="cuda").view(q, 1, 1, 1)
    df = torch.randn((q, N, N, N), generator=gen, device="cuda", dtype=torch.float32)
    df.mul_(0.05 * wt)
    rng = np.random.default_rng(5)
    samples = [(0, 0, 0), (N - 1, N - 1, N - 1), (0, N - 1, 255), (N - 1, 0, 1), (300, 0, N - 1)]
    samples += [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(15)]

    # inputs of the oracle: the 5x5x5 neighbourhood of every sample, read from
    # the seeded input tensor (not from the library)
    def hood(x, y, z):
        ix = torch.tensor([(x + d) % N for d in range(-2, 3)], device="cuda")
        iy = torch.tensor([(y + d) % N for d in range(-2, 3)], device="cuda")
        iz = torch.tensor([(z + d) % N for d in range(-2, 3)], device="cuda")
        sub = df.index_select(3, ix).index_select(2, iy).index_select(1, iz)
        return sub.cpu().numpy().astype(np.float64) + w.reshape(q, 1, 1, 1)  # [Q, z, y, x]

    hoods = {s: hood(*s) for s in samples}

    with B.Solver(lattice, (N, N, N), TAU) as s:
        s.set_populations(df)
        d0 = s.diagnostics()
        got = []
        for k in range(2):
            s.step(1)
            out = s.populations()
            idx = torch.tensor([[(z * N + y) * N + x for (x, y, z) in samples]], device="cuda")
            got.append(out.view(q, -1).index_select(1, idx[0]).cpu().numpy().astype(np.float64))
            del out
            torch.cuda.empty_cache()
        d2 = s.diagnostics()
    del df
    torch.cuda.empty_cache()

    for si, smp in enumerate(samples):
        h = hoods[smp]
        cache = {}

        def post(dx, dy, dz):
            key = (dx, dy, dz)
            if key not in cache:
                cache[key] = O.collide_cell(lattice, h[:, 2 + dz, 2 + dy, 2 + dx], TAU)
            return cache[key]

        # one update: f_i(x) = post(x - xi_i)_i
        ref1 = np.array([post(-c[i, 0], -c[i, 1], -c[i, 2])[i] for i in range(q)]) - w
        assert np.max(np.abs(got[0][:, si] - ref1) / w) <= 1e-6, smp

        # two updates: f_i(x) = collide(f(x - xi_i, t+1))_i
        ref2 = np.zeros(q)
        for i in range(q):
            yx, yy, yz = -c[i, 0], -c[i, 1], -c[i, 2]
            fy = np.array([post(yx - c[j, 0], yy - c[j, 1], yz - c[j, 2])[j] for j in range(q)])
            ref2[i] = O.collide_cell(lattice, fy, TAU)[i] - w[i]
        assert np.max(np.abs(got[1][:, si] - ref2) / w) <= 1e-6, smp

    # conservation at full size
    assert abs(d2[0] - d0[0]) <= 1e-12 * d0[0]
    assert np.allclose(d2[1:4], d0[1:4], rtol=0, atol=1e-3)


def _sample_two_steps(lattice, N3, df_dev, samples, tau, storage=None):
    """Run two updates from df_dev ([Q, nz, ny, nx] shifted populations on the
    device) and return the logical populations of the sampled cells after each."""
    from paper_1505_06900_gb300 import binding as B
    nx, ny, nz = N3
    q = df_dev.shape[0]
    got = []
    kw = {} if storage is None else {"storage": storage}
    with B.Solver(lattice, N3, tau, **kw) as s:
        s.set_populations(df_dev)
        for _ in range(2):
            s.step(1)
            out = s.populations()
            idx = torch.tensor([(z * ny + y) * nx + x for (x, y, z) in samples], device="cuda")
            got.append(out.view(q, -1).index_select(1, idx).cpu().numpy().astype(np.float64))
            del out
            torch.cuda.empty_cache()
    return got


def test_sampled_cells_d2q9_2048_squared():
    """D2Q9 2048^2 (the double-shear-layer size), FP32 store: sampled cells
    after one and two updates against the oracle's collisions."""
    from paper_1505_06900_gb300 import binding as B
    n = 2048
    c, w = O.lattice_tables(O.D2Q9)
    tau = W.double_shear_2d_tau(n, 0.1)
    gen = torch.Generator(device="cuda").manual_seed(77)
    wt = torch.tensor(w, dtype=torch.float32, device="cuda").view(9, 1, 1, 1)
    df = torch.randn((9, 1, n, n), generator=gen, device="cuda", dtype=torch.float32) * (0.05 * wt)
    rng = np.random.default_rng(7)
    samples = [(0, 0, 0), (n - 1, n - 1, 0), (0, n - 1, 0), (n - 1, 0, 0)]
    samples += [(int(rng.integers(0, n)), int(rng.integers(0, n)), 0) for _ in range(30)]
    host = {}
    for (x, y, _) in samples:
        ix = torch.tensor([(x + d) % n for d in range(-2, 3)], device="cuda")
        iy = torch.tensor([(y + d) % n for d in range(-2, 3)], device="cuda")
        host[(x, y)] = (df[:, 0].index_select(2, ix).index_select(1, iy).cpu().numpy()
                        .astype(np.float64) + w.reshape(9, 1, 1))
    got = _sample_two_steps(B.D2Q9, (n, n, 1), df, samples, tau)
    for si, (x, y, _) in enumerate(samples):
        h = host[(x, y)]
        cache = {}

        def post(dx, dy):
            if (dx, dy) not in cache:
                cache[(dx, dy)] = O.collide_cell(O.D2Q9, h[:, 2 + dy, 2 + dx], tau)
            return cache[(dx, dy)]

        ref1 = np.array([post(-c[i, 0], -c[i, 1])[i] for i in range(9)]) - w
        assert np.max(np.abs(got[0][:, si] - ref1) / w) <= 1e-6
        ref2 = np.array([O.collide_cell(O.D2Q9, np.array(
            [post(-c[i, 0] - c[j, 0], -c[i, 1] - c[j, 1])[j] for j in range(9)]), tau)[i]
            for i in range(9)]) - w
        assert np.max(np.abs(got[1][:, si] - ref2) / w) <= 1e-6


def test_sampled_cells_f16_store_at_512_cubed():
    """D3Q27 512^3 with the FP16 store (the shared-memory tiled kernel the
    benchmark's FP16 variant times): one update of sampled cells, stored value
    within one FP16 unit in the last place (plus 1e-6) of the oracle's."""
    from paper_1505_06900_gb300 import binding as B
    c, w = O.lattice_tables(O.D3Q27)
    free = torch.cuda.mem_get_info()[0]
    if free < 40e9:
        pytest.skip("needs 40 GB of free device memory")
    gen = torch.Generator(device="cuda").manual_seed(99)
    g16 = (0.05 * torch.randn((27, N, N, N), generator=gen, device="cuda")).to(torch.float16)
    rng = np.random.default_rng(9)
    samples = [(0, 0, 0), (N - 1, N - 1, N - 1), (127, 128, 5), (128, 0, N - 1)]
    samples += [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(12)]
    hoods = {}
    for (x, y, z) in samples:
        ix = torch.tensor([(x + d) % N for d in (-1, 0, 1)], device="cuda")
        iy = torch.tensor([(y + d) % N for d in (-1, 0, 1)], device="cuda")
        iz = torch.tensor([(z + d) % N for d in (-1, 0, 1)], device="cuda")
        sub = g16.index_select(3, ix).index_select(2, iy).index_select(1, iz)
        hoods[(x, y, z)] = w.reshape(27, 1, 1, 1) * (1.0 + sub.cpu().numpy().astype(np.float64))
    with B.Solver(B.D3Q27, (N, N, N), TAU, storage=B.STORE_F16) as s:
        s.set_state(g16.contiguous().view(torch.uint8).reshape(-1), 0)
        del g16
        torch.cuda.empty_cache()
        s.step(1)
        out = s.populations()
        idx = torch.tensor([(z * N + y) * N + x for (x, y, z) in samples], device="cuda")
        got = out.view(27, -1).index_select(1, idx).cpu().numpy().astype(np.float64)
        del out
    for si, smp in enumerate(samples):
        h = hoods[smp]
        ref = np.array([O.collide_cell(O.D3Q27, h[:, 1 - c[i, 2], 1 - c[i, 1], 1 - c[i, 0]], TAU)[i]
                        for i in range(27)])
        g_ref = ref / w - 1.0
        g_got = got[:, si] / w
        ulp = 2.0 ** (np.floor(np.log2(np.maximum(np.abs(g_ref), 2.0 ** -14))) - 10)
        assert np.all(np.abs(g_got - g_ref) <= ulp + 1e-6), smp


def test_sampled_cells_fused_closure_at_256_cubed():
    """The fused learned-closure update at 256^3, the coarse grid of the
    learned form, launched as lb_step launches it (one persistent block per
    SM), one update at each AA parity. For sampled cells (both 128-cell tiles
    of a row at their edges, the periodic faces and random cells): the 27
    neighbours' features the kernel read against the standardised oracle
    moments of the state before the update (one BF16 unit), both hidden
    activations and the 17 predictions against the FP64 network with the
    bounds of the network tests, and the cell's 27 post-update populations,
    where streaming puts them, against the oracle's corrected collision with
    the kernel's predictions (1e-6 of the weights)."""
    from oracle import closure as C
    from paper_1505_06900_gb300 import binding as B
    from _common import f64_state
    from test_gpu_closure import bf16_params, check_forward_chain

    n, theta, o_scale = 256, 0.3, 2e-5
    shape = (n, n, n)
    tau = W.taylor_green_3d_tau(n, 0.3, 1600.0)
    rho, u = W.random_field(shape, 3, seed=81, a_rho=0.005, a_u=0.03)
    rng = np.random.default_rng(82)
    p = bf16_params(rng, (0.05, 0.15, 0.3))
    cvel, w = O.lattice_tables(O.D3Q27)
    # sampled cells: tile edges x = 0, 127, 128, 255 and neighbours, periodic faces
    edge = [0, 1, 126, 127, 128, 129, 254, 255]
    cells = [(x, y, z) for x in edge for y, z in ((0, 0), (255, 255), (0, 131), (77, 255))]
    cells += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(64)]
    xs_, ys_, zs_ = (np.array(v) for v in zip(*cells))
    S = len(cells)
    # the 27 neighbours of each sampled cell, neighbour nb = (dx+1) + 3(dy+1) + 9(dz+1)
    nb_x = np.stack([(xs_ + (k % 3 - 1)) % n for k in range(27)], 1)
    nb_y = np.stack([(ys_ + ((k // 3) % 3 - 1)) % n for k in range(27)], 1)
    nb_z = np.stack([(zs_ + (k // 9 - 1)) % n for k in range(27)], 1)
    net = B.MLP(C.pack(p))
    with B.Solver(B.D3Q27, shape, tau) as s:
        s.init_fields(torch.from_numpy(rho.astype(np.float32)).cuda(),
                      torch.from_numpy(u.astype(np.float32)).cuda())
        r_d, u_d, pi_d = s.moments()
        mom = torch.cat([(r_d - 1.0).reshape(1, -1), u_d.reshape(3, -1), pi_d.reshape(6, -1)])
        mean = mom.double().mean(1).cpu().numpy().astype(np.float32)
        inv = (1.0 / (mom.double().std(1) + 1e-12)).cpu().numpy().astype(np.float32)
        del r_d, u_d, pi_d, mom
        net.set_scaling(mean, inv, np.full(17, o_scale, np.float32))
        s.set_closure(net, bound=1e6, dead_zone=theta)
        m64, i64 = mean.astype(np.float64), inv.astype(np.float64)
        o64 = np.full(17, np.float32(o_scale), np.float64)
        for parity in (0, 1):
            pre = s.populations()
            nbf = pre[:, torch.from_numpy(nb_z.reshape(-1)).cuda(),
                      torch.from_numpy(nb_y.reshape(-1)).cuda(),
                      torch.from_numpy(nb_x.reshape(-1)).cuda()].cpu().numpy()
            del pre
            tr, xs = s.closure_step_trace()
            sel = torch.from_numpy(np.asarray([(z * n + y) * n + x for x, y, z in cells])).cuda()
            trs = tr.index_select(0, sel).cpu().numpy().astype(np.float64)
            feat = xs[torch.from_numpy(nb_z.reshape(-1) + 1).cuda(),
                      torch.from_numpy(nb_y.reshape(-1) + 1).cuda(),
                      torch.from_numpy(nb_x.reshape(-1) + 1).cuda()].float().cpu().numpy()
            del tr, xs
            post = s.populations()
            # features: standardised oracle moments of each neighbour, one BF16 unit
            f_nb = f64_state(O.D3Q27, nbf.reshape(27, 1, 1, -1))
            z_ref = (C.moment_field(f_nb).reshape(10, -1).T - m64) * i64  # [27 S, 10]
            ulp = 2.0 ** (np.floor(np.log2(np.maximum(np.abs(z_ref), 1e-30))) - 7)
            assert np.all(np.abs(feat[:, :10] - z_ref) <= ulp + 1e-5), parity
            assert np.all(feat[:, 10:] == 0)
            # the network, layer by layer, from the features the kernel read
            X = np.zeros((S, 288))
            X[:, :270] = feat[:, :10].reshape(S, 27, 10).reshape(S, 270)
            Y = np.zeros((S, 32))
            Y[:, :17] = trs[:, 128:145]
            check_forward_chain(X, p, trs[:, :64], trs[:, 64:128], Y)
            # the update: oracle collision of each cell with the kernel's predictions
            yd = np.sign(Y[:, :17]) * np.maximum(np.abs(Y[:, :17]) - theta, 0.0)
            assert np.count_nonzero(yd) > 0.1 * yd.size
            f_cell = f_nb.reshape(27, S, 27)[:, :, 13]  # neighbour 13 is the cell itself
            for c_i, (x, y, z) in enumerate(cells):
                ref = O.collide_cell_closure(f_cell[:, c_i], tau, yd[c_i] * o64)
                gx = (x + cvel[:, 0]) % n
                gy = (y + cvel[:, 1]) % n
                gz = (z + cvel[:, 2]) % n
                got = post[torch.arange(27).cuda(), torch.from_numpy(gz).cuda(),
                           torch.from_numpy(gy).cuda(),
                           torch.from_numpy(gx).cuda()].cpu().numpy().astype(np.float64)
                err = np.max(np.abs(got + w - ref) / w)
                assert err <= 1e-6, (parity, (x, y, z), err)
            del post
        assert s.closure_fallbacks() == 0
    net.close()
