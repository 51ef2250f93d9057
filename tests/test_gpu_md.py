"""GPU parity of the Langevin dynamics driver (Section 4.3, BAOAB) with the
forces of the library plus Section 5.2's LJ model, against the oracle's
step on the oracle's forces; CUDA-graph replays equal plain steps."""
import numpy as np
import pytest

from oracle import ewald2d, lattice, md, soe_ewald2d, walls

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qslab():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01521_gb300 as q
    q.load()
    return q


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _spread(n, box, seed, dmin=1.05, zpad=1.0):
    """n points with pairwise distances >= dmin (x, y periodic), z inside
    [zpad, Lz - zpad]."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        p = np.array([rng.uniform(0, box[0]), rng.uniform(0, box[1]), rng.uniform(zpad, box[2] - zpad)])
        ok = True
        for o in out:
            d = p - o
            d[0] -= box[0] * round(d[0] / box[0])
            d[1] -= box[1] * round(d[1] / box[1])
            if d @ d < dmin * dmin:
                ok = False
                break
        if ok:
            out.append(p)
    return np.array(out)


BOX = (36.0, 36.0, 12.0)
ALPHA, RC = 0.35, 12.0
SW = (0.01, -0.01)
PARAMS = md.MDParams(dt=0.002, mass=1.0, gamma=1.0, kT=1.0, lj_eps=1.0, lj_sigma=1.0,
                     wall_eps=1.0, wall_sigma=0.5, seed=5)


def _oracle_forces(q, soe, kc, modes=None):
    s, w = soe

    def f(pos):
        if modes is None:
            lr = soe_ewald2d.soe_full(pos, q, BOX, ALPHA, s, w, kc=kc)
        else:
            lr = soe_ewald2d.soe_rbe(pos, q, BOX, ALPHA, s, w, *modes)
        ps = walls.wall_potential(pos, q, BOX, *SW)
        rs = ewald2d.realspace(pos, q, BOX, ALPHA, RC)
        lj = md.lj_pairs(pos, BOX, PARAMS.lj_eps, PARAMS.lj_sigma)
        lw = md.lj_walls(pos, BOX, PARAMS.wall_eps, PARAMS.wall_sigma)
        F = lr["F"] + ps["F"] + rs["F"] + lj["F"] + lw["F"]
        E = [lr["E"] + ps["E"], rs["E"] + lj["E"], lw["E"]]
        return F, E
    return f


def _slab(qslab, prec, soe, kc=None, rbe=None):
    slab = qslab.QSlab(0, prec).configure(BOX, ALPHA, soe, kcut=kc, rbe=rbe, rcut=RC)
    slab.set_walls(*SW)
    slab.md_configure(PARAMS.dt, PARAMS.mass, PARAMS.gamma, PARAMS.kT,
                      (PARAMS.lj_eps, PARAMS.lj_sigma), (PARAMS.wall_eps, PARAMS.wall_sigma),
                      PARAMS.seed)
    return slab


def test_md_fp64_full_k_matches_oracle(qslab, soe16):
    n = 160
    pos0 = _spread(n, BOX, 3)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    vel0 = np.random.default_rng(4).normal(size=(n, 3))
    kc = lattice.kcut_for_tail(ALPHA, 1e-10)
    slab = _slab(qslab, "fp64", soe16, kc=kc)
    pos = torch.tensor(pos0, device="cuda")
    vel = torch.tensor(vel0, device="cuda")
    tq = torch.tensor(q, device="cuda")
    F, E = slab.md_forces(pos, tq, vel)
    force_fn = _oracle_forces(q, soe16, kc)
    Fo, Eo = force_fn(pos0)
    assert slab.status() == 0
    assert _rel(F.cpu().numpy(), Fo) < 1e-10
    e = E.cpu().numpy()
    for j in range(3):
        assert abs(e[j] - Eo[j]) <= 1e-10 * max(abs(Eo[j]), 1.0), j
    assert abs(e[3] - 0.5 * (vel0 ** 2).sum()) <= 1e-12 * e[3]
    x, v, Fx = pos0, vel0, Fo
    for step in range(3):
        E = slab.md_step(pos, vel, tq, F, 1)
        x, v, Fx = md.baoab_step(x, v, Fx, BOX, PARAMS, step, lambda p: force_fn(p)[0])
        assert slab.status() == 0
        assert _rel(pos.cpu().numpy(), x) < 1e-12
        assert _rel(vel.cpu().numpy(), v) < 1e-10
        assert _rel(F.cpu().numpy(), Fx) < 1e-10
    assert qslab.qslab_md_get_step(slab.h) == 3
    e = E.cpu().numpy()
    assert abs(e[3] - 0.5 * (v ** 2).sum()) <= 1e-10 * e[3]
    slab.close()


def test_md_fp32_rbe_metropolis_step(qslab, soe16):
    """FP32C, random batch with the Metropolis sampler: one step against the
    oracle's step with the modes the device drew for the new forces."""
    n = 240
    pos0 = _spread(n, BOX, 8)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    vel0 = np.random.default_rng(9).normal(size=(n, 3))
    slab = _slab(qslab, "fp32c", soe16, rbe=(100, 21)).sampler("metropolis", 2)
    pos = torch.tensor(pos0, device="cuda", dtype=torch.float32)
    vel = torch.tensor(vel0, device="cuda", dtype=torch.float32)
    tq = torch.tensor(q, device="cuda", dtype=torch.float32)
    F, _ = slab.md_forces(pos, tq, vel)
    slab.md_step(pos, vel, tq, F, 10)
    x0, v0, F0 = (t.double().cpu().numpy() for t in (pos, vel, F))
    slab.md_step(pos, vel, tq, F, 1)
    assert slab.status() == 0
    mx, my, _ = slab.sampled_modes()
    call = slab.rng_state()[1] - 1
    omx, omy = lattice.metropolis_modes(100, 21, call, ALPHA, BOX[0], BOX[1], thin=2)
    assert (mx == omx).all() and (my == omy).all()
    force_fn = _oracle_forces(q, soe16, None, modes=(omx, omy))
    x, v, Fx = md.baoab_step(x0, v0, F0, BOX, PARAMS, 10, lambda p: force_fn(p)[0])
    assert np.abs(pos.double().cpu().numpy() - x).max() < 2e-5
    assert _rel(vel.double().cpu().numpy(), v) < 1e-5
    rms = lambda a: float(np.sqrt((a ** 2).mean()))
    assert rms(F.double().cpu().numpy() - Fx) < 1e-4 * rms(Fx)
    slab.close()


def test_md_graph_replay_equals_plain_steps(qslab, soe16):
    n = 200
    pos0 = _spread(n, BOX, 12)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    vel0 = np.random.default_rng(13).normal(size=(n, 3))
    res = []
    for graphed in (False, True):
        slab = _slab(qslab, "fp32c", soe16, rbe=(64, 3))
        pos = torch.tensor(pos0, device="cuda", dtype=torch.float32)
        vel = torch.tensor(vel0, device="cuda", dtype=torch.float32)
        tq = torch.tensor(q, device="cuda", dtype=torch.float32)
        F, _ = slab.md_forces(pos, tq, vel)
        if graphed:
            g = qslab.GraphedMD(slab, pos, vel, tq, F, 4)       # 4 steps in the warm-up
            g.replay()
            E = g.replay()
        else:
            for _ in range(3):
                E = slab.md_step(pos, vel, tq, F, 4)
        torch.cuda.synchronize()
        assert slab.status() == 0
        assert qslab.qslab_md_get_step(slab.h) == 12
        res.append([t.cpu().numpy().copy() for t in (pos, vel, F, E)])
        slab.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_md_input_errors(qslab, soe16):
    slab = qslab.QSlab(0, "fp64").configure(BOX, ALPHA, soe16, kcut=1.0)
    pos = torch.tensor(_spread(10, BOX, 1), device="cuda")
    q = torch.tensor(np.array([1.0, -1.0] * 5), device="cuda")
    with pytest.raises(qslab.QslabError) as e:            # not configured
        slab.md_forces(pos, q)
    assert e.value.code == qslab.QSLAB_ERR_NOT_CONFIGURED
    for bad in [dict(dt=0.0), dict(dt=0.01, mass=-1.0), dict(dt=0.01, gamma=-1.0),
                dict(dt=0.01, lj=(1.0, 0.0))]:
        with pytest.raises(qslab.QslabError):
            slab.md_configure(**bad)
    qslab.qslab_set_rcut(slab.h, 1.0)                     # below the LJ cut-off 2^(1/6)
    slab.md_configure(0.01)
    with pytest.raises(qslab.QslabError) as e:
        slab.md_forces(pos, q)
    assert e.value.code == qslab.QSLAB_ERR_INVALID_ARG
    slab.close()


def _cation_profile(qslab, soe, rbe, nsteps, seed):
    """z-histogram (1-wide bins) of Section 5.2's cation-only system: 436
    cations in 100 x 100 x 30, top wall at -0.0436 (neutralising), LJ
    particles and walls, alpha = 0.3, rc = 4/alpha, Langevin at kT = 1,
    dt = 0.005; averaged over the last two thirds of the run."""
    import workloads
    sl = workloads.cations_walls()
    rng = np.random.default_rng(seed)
    g = (np.arange(8) + 0.5) * 12.5
    gx, gy, gz = np.meshgrid(g, g, 2.0 + np.arange(7) * 4.3, indexing="ij")
    pos0 = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1)[:sl.N] + rng.uniform(-1, 1, (sl.N, 3))
    slab = qslab.QSlab(0, "fp32c").configure(sl.box, 0.3, soe, rbe=rbe, rcut=4 / 0.3)
    if rbe is not None:
        slab.sampler("metropolis", 1)
    slab.set_walls(*sl.walls)
    slab.md_configure(0.005, 1.0, 1.0, 1.0, (1.0, 1.0), (1.0, 0.5), seed)
    pos = torch.tensor(pos0, device="cuda", dtype=torch.float32)
    vel = torch.tensor(rng.normal(size=(sl.N, 3)), device="cuda", dtype=torch.float32)
    q = torch.tensor(sl.q, device="cuda", dtype=torch.float32)
    F, _ = slab.md_forces(pos, q, vel)
    chunk = 100
    gr = qslab.GraphedMD(slab, pos, vel, q, F, chunk)
    hist = np.zeros(30)
    nchunks = nsteps // chunk
    for k in range(nchunks):
        gr.replay()
        if k >= nchunks // 3:
            hist += np.histogram(pos[:, 2].cpu().numpy(), bins=30, range=(0.0, 30.0))[0]
    assert slab.status() == 0
    slab.close()
    return hist / hist.sum()


def test_md_cation_layer_rbe_matches_full_k(qslab, soe16):
    """Section 5.2, cation-only system (the concentration profile of its
    Fig. 5(b), qualitatively): the cations gather in a layer at the
    neutralising wall, and the random-batch run (P = 100, Metropolis
    sampler) gives the same profile as the full k-sum."""
    rb = _cation_profile(qslab, soe16, (100, 7), 30_000, 3)
    fk = _cation_profile(qslab, soe16, None, 30_000, 4)
    for p in (rb, fk):
        assert p[25:].sum() > 0.4            # most cations within 5 of the top wall
        assert p[:15].sum() < 0.25           # a dilute bulk at the uncharged wall's side
        assert (np.diff(p[15:29]) > -0.01).all()   # rising towards the charged wall
    assert abs(rb[25:].sum() - fk[25:].sum()) < 0.03
    assert abs((rb * np.arange(30)).sum() - (fk * np.arange(30)).sum()) < 0.5
