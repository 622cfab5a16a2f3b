"""GPU parity of the learned-proposal extension (Metropolis–Hastings bond
moves, the BF16 tensor-core network, the event log) against the oracle.

- MH with the uniform proposal: bit-exact bond tables and move counters
  against the oracle's MH sweep on frozen configurations, over all eight
  checkerboard colours.
- Both proposals reach the exact Boltzmann arm populations of frozen stars
  (the learned one only through its Hastings factor).
- The network: forward, loss and gradient against an FP64 evaluation of the
  same BF16-rounded operands (FP32 summation order apart) and against the
  exact FP64 oracle (relative 1e-2 per tensor or the BF16 operands' own
  error, cosine > 0.999); training lowers the loss.
- The event log of a plain sweep equals the oracle's events bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from oracle.features import FeatureState, sweep_events
from synth import random_frozen, colloid_linker, telechelic

from _stars import star_arm_ranks, star_expectation, star_occupancy, stars_case, block_mean_se

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def snapmod(torch):
    from paper_2609_21204_b300 import build
    build.build()
    import paper_2609_21204_b300 as m
    return m


def _mh_cases():
    return {
        "ab_v1": lambda: random_frozen(seed=21, n=9000, box=22.0, overlap_factor=0.6, r_max=1.4, eps=1.0),
        "ab_v3_2": lambda: random_frozen(seed=22, n=9000, box=22.0, overlap_factor=0.6, r_max=1.5,
                                         valence=(3, 2), r_min=0.4, eps=2.0),
        "colloid_linker": lambda: colloid_linker(seed=23, n_c=4000, n_l=16000, eps=3.0),
        "telechelic": lambda: telechelic(seed=24, n_chains=300, n_x=600, eps=1.0),
    }


MH_STATS = ("form_attempts", "form_accepts", "break_attempts", "break_accepts")


@pytest.mark.parametrize("name", list(_mh_cases()))
def test_mh_uniform_bit_exact(snapmod, name):
    s = _mh_cases()[name]()
    precision = "fp64" if name == "ab_v1" else "mixed"
    sim = snapmod.from_system(s, precision=precision)
    orc = oracle.OracleSystem(s)
    sim.set_mh(1)
    tot = dict.fromkeys(MH_STATS, 0)
    for step in list(range(24)) + [1000, 123456789]:
        sim.set_step(step)
        sim.mh_sweep()
        st = orc.mh_sweep(step=step)
        for k in MH_STATS:
            tot[k] += st[k]
        assert np.array_equal(sim.bonds(), orc.bonds()), (name, step)
    g = sim.stats()
    for k in MH_STATS:
        assert g["mh_" + k] == tot[k], (name, k, g["mh_" + k], tot[k])
    assert tot["form_accepts"] > 0 and tot["break_accepts"] > 0
    b = sim.bonds()
    occ = np.bincount(b[:, :2].ravel(), minlength=s.n)
    assert np.all(occ <= np.asarray(s.valence)[s.types])


def _run_stars(snapmod, mode, mlp=None, sweeps=8000, burn=800):
    s = stars_case(n_stars=512, seed=12)
    sim = snapmod.from_system(s, precision="fp64")
    sim.set_mh(mode, mlp, eps_u=0.05)
    rank = star_arm_ranks(s)
    samples = []
    for t in range(sweeps):
        sim.set_step(t)
        sim.mh_sweep()
        if t >= burn and t % 8 == 7:
            b = sim.bonds()
            dp = np.full((s.n, 4), -1, np.int64)
            dp[b[:, 0], 0] = b[:, 1]
            dp[b[:, 1], 0] = b[:, 0]
            samples.append(star_occupancy(dp, s, rank))
    mean, se = block_mean_se(np.array(samples))
    return s, mean, se, sim.stats()


@pytest.mark.parametrize("mode", [1, 2])
def test_mh_stars_reach_boltzmann_populations(snapmod, mode):
    mlp = snapmod.Mlp(omlp.init(seed=5, scale=3.0).astype(np.float32)) if mode == 2 else None
    s, mean, se, st = _run_stars(snapmod, mode, mlp)
    expect = star_expectation(s, math.exp(s.reactions[0].eps))
    assert np.all(np.abs(mean - expect) < 4 * se + 0.01), (mode, mean, expect, se)
    assert st["mh_form_accepts"] > 1000 and st["mh_break_accepts"] > 1000


# ------------------------------------------------------------------ network
@pytest.mark.parametrize("rows", [1, 15, 16, 1037, 70000])
def test_mlp_forward(snapmod, torch, rows):
    rng = np.random.default_rng(rows)
    X = rng.normal(size=(rows, omlp.NF)).astype(np.float32)
    theta = omlp.init(seed=3, scale=1.5).astype(np.float32)
    m = snapmod.Mlp(theta)
    assert np.array_equal(m.weights(), theta)
    dX = torch.from_numpy(X).cuda()
    dy = torch.full((rows + 3,), 7.0, device="cuda")
    m.forward(dX.data_ptr(), rows, dy.data_ptr())
    torch.cuda.synchronize()
    y = dy.cpu().numpy()
    assert np.all(y[rows:] == 7.0)          # nothing written past the rows
    y = y[:rows].astype(np.float64)
    emu, _ = omlp.forward_bf16(theta.astype(np.float64), X.astype(np.float64))
    ref, _ = omlp.forward(theta.astype(np.float64), X.astype(np.float64))
    scale = 1.0 + np.abs(ref).max()
    assert np.abs(y - emu).max() <= 2e-3 * scale, np.abs(y - emu).max()
    assert np.abs(y - ref).max() <= 5e-2 * scale, np.abs(y - ref).max()


def _random_events(rng, n_events, nmax=16):
    sizes = rng.integers(1, nmax + 1, n_events)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    X = rng.normal(size=(off[-1], omlp.NF)).astype(np.float32)
    # the label is the candidate with the smallest |feature 1| (learnable)
    lab = np.array([np.argmin(np.abs(X[off[e]:off[e + 1], 1])) for e in range(n_events)], np.int32)
    return X, off, lab


def test_mlp_loss_and_gradient(snapmod, torch):
    """Against the FP64 evaluation of the same BF16 operands: relative 2e-3
    per tensor (FP32 summation order).  Against the exact FP64 oracle: cosine
    > 0.999 and relative 1e-2 per tensor, or 1.5x the BF16 operands' own
    error where cancellation in the gradient sum makes that larger (W1)."""
    rng = np.random.default_rng(7)
    X, off, lab = _random_events(rng, 700)
    theta = omlp.init(seed=4).astype(np.float32)
    m = snapmod.Mlp(theta)
    dX, doff, dlab = (torch.from_numpy(a).cuda() for a in (X, off, lab))
    loss, g = m.loss_grad(dX.data_ptr(), X.shape[0], doff.data_ptr(), dlab.data_ptr(), len(lab))
    t64, X64 = theta.astype(np.float64), X.astype(np.float64)
    loss_o, g_o = omlp.loss_and_grad(t64, X64, off, lab)
    loss_b, _, g_b = omlp.loss_and_grad_bf16(t64, X64, off, lab)
    assert abs(loss - loss_b) <= 1e-4 * abs(loss_b), (loss, loss_b)
    assert abs(loss - loss_o) <= 1e-2 * abs(loss_o), (loss, loss_o)
    assert np.all(omlp.unpack(g.astype(np.float64))["W1"][omlp.NF:] == 0.0)
    gp, gop, gbp = (omlp.unpack(v.astype(np.float64)) for v in (g, g_o, g_b))
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    for name in ("W1", "b1", "W2", "b2", "w3"):
        a, o, b = (d[name][:omlp.NF].ravel() if name == "W1" else d[name].ravel() for d in (gp, gop, gbp))
        cos = a @ o / (np.linalg.norm(a) * np.linalg.norm(o))
        assert rel(a, b) <= 2e-3, (name, rel(a, b))
        assert rel(a, o) <= max(1e-2, 1.5 * rel(b, o)) and cos > 0.999, (name, rel(a, o), rel(b, o), cos)
    assert abs(gp["b3"][0]) <= 1e-5     # softmax gradients sum to zero per event


def test_mlp_training_lowers_loss(snapmod, torch):
    rng = np.random.default_rng(8)
    X, off, lab = _random_events(rng, 20000)
    m = snapmod.Mlp(omlp.init(seed=6).astype(np.float32))
    dX, doff, dlab = (torch.from_numpy(a).cuda() for a in (X, off, lab))
    args = (dX.data_ptr(), X.shape[0], doff.data_ptr(), dlab.data_ptr(), len(lab))
    before, _ = m.loss_grad(*args)
    losses = m.train(*args, epochs=15, batch_events=512, lr=2e-3, seed=1)
    after, _ = m.loss_grad(*args)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.6 * losses[0] and after < 0.5 * before, (before, after, losses)


# ---------------------------------------------------------------- event log
def test_event_log_matches_oracle(snapmod):
    s = random_frozen(seed=31, n=4000, box=15.0, overlap_factor=0.6, r_max=1.4, valence=(2, 2), eps=1.0)
    sim = snapmod.from_system(s, precision="mixed")
    orc = oracle.OracleSystem(s)
    sim.log_events(100000)
    total = 0
    for step in (0, 1, 2, 77):
        state = FeatureState(orc.pos, s.box, s.types, s.valence, orc.dp.reshape(s.n, 4).copy(),
                             s.reactions[0], s.bond_types[s.reactions[0].bond_type].r0)
        sim.set_step(step)
        sim.bond_update()
        _, tr = orc.sweep(step=step, trace=True)
        assert np.array_equal(sim.bonds(), orc.bonds())
        ev_o = sweep_events(state, tr["prop"], tr["matched"], tr["formed"])
        feat, off, lab = sim.get_events(clear=True)
        ev_g = [(feat[off[e]:off[e + 1]], int(lab[e])) for e in range(len(lab))]
        key = lambda ev: (ev[0].tobytes(), ev[1])
        assert sorted(map(key, ev_g)) == sorted(map(key, ev_o)), (step, len(ev_g), len(ev_o))
        total += len(ev_o)
    assert total > 200
    assert sim.stats()["events_logged"] == total


# ------------------------------------------------------------ MD in MH mode
def test_md_with_mh_moves_keeps_invariants(snapmod):
    s = colloid_linker(seed=41, n_c=2000, n_l=8000, eps=4.0)
    sim = snapmod.from_system(s, precision="mixed")
    mlp = snapmod.Mlp(omlp.init(seed=9).astype(np.float32))
    val = np.asarray(s.valence)[s.types]
    for mode, steps in ((2, 300), (1, 200), (0, 50), (2, 50)):
        sim.set_mh(mode, mlp if mode == 2 else None)
        sim.step(steps)
        b = sim.bonds()
        occ = np.bincount(b[:, :2].ravel(), minlength=s.n)
        assert np.all(occ <= val)
        assert np.all(s.types[b[:, 0]] != s.types[b[:, 1]])
        assert np.all(np.isfinite(sim.positions()))
    st = sim.stats()
    assert st["mh_form_accepts"] > 100 and st["mh_break_accepts"] > 0
    assert b.shape[0] > 1000


def test_mh_argument_checks(snapmod):
    s = random_frozen(seed=51, n=200, box=7.0, overlap_factor=0.6)
    sim = snapmod.from_system(s)
    with pytest.raises(snapmod.SnapError):
        sim.mh_sweep()                     # MH mode is off
    with pytest.raises(snapmod.SnapError):
        sim.set_mh(2)                      # learned proposal without a network
    with pytest.raises(snapmod.SnapError):
        sim.set_mh(3)
    with pytest.raises(snapmod.SnapError):
        sim.set_step(-1)
    with pytest.raises(snapmod.SnapError):
        sim.get_events()                   # logging is off
    small = random_frozen(seed=52, n=50, box=4.0, overlap_factor=0.6)
    with pytest.raises(snapmod.SnapError):
        snapmod.from_system(small).set_mh(1)   # fewer than 2 MH cells per axis


# ------------------------------------------------- what the network gains
def _train_on_plain_events(snapmod, torch, sim, sweeps, epochs, seed=1):
    """Log formation events of plain sweeps at frozen positions, hold out a
    tenth, train the network on the rest; returns it with held-out metrics."""
    sim.log_events(1_000_000)
    for t in range(sweeps):
        sim.set_step(t)
        sim.bond_update()
    feat, off, lab = sim.get_events(clear=True)
    sim.log_events(0)
    E = len(lab)
    Et = int(0.9 * E)
    dX, doff, dlab = (torch.from_numpy(a).cuda() for a in (feat, off, lab))
    m = snapmod.Mlp(omlp.init(seed=seed).astype(np.float32))
    m.train(dX.data_ptr(), int(off[Et]), doff.data_ptr(), dlab.data_ptr(), Et, epochs=epochs,
            batch_events=1024, lr=2e-3, seed=seed + 1)
    # held-out cross-entropy and top-1 accuracy of the network and of uniform choice
    y = torch.empty(int(off[E]), device="cuda")
    m.forward(dX.data_ptr(), int(off[E]), y.data_ptr())
    torch.cuda.synchronize()
    y = y.cpu().numpy().astype(np.float64)
    ce, hit, ce_u, hit_u = [], [], [], []
    for e in range(Et, E):
        z = y[off[e]:off[e + 1]]
        z = z - z.max()
        lp = z - np.log(np.exp(z).sum())
        ce.append(-lp[lab[e]])
        hit.append(np.argmax(z) == lab[e])
        n = off[e + 1] - off[e]
        ce_u.append(np.log(n))
        hit_u.append(1.0 / n)
    return m, dict(events=E, ce=np.mean(ce), ce_uniform=np.mean(ce_u), top1=np.mean(hit), top1_uniform=np.mean(hit_u))


def test_trained_proposal_gain_on_competing_partners(snapmod, torch):
    """Stars whose arms compete for one centre: the network trained on the
    plain method's formation events predicts its choice far better than a
    uniform pick, and as an MH proposal it raises the accepted fraction of
    moves while the arm populations stay at their Boltzmann values."""
    from synth import frozen_stars
    s = frozen_stars(seed=21, n_stars=512, arms=6, r_lo=0.95, r_hi=1.3, k=400.0, eps=0.0, r_max=1.35,
                     min_sep=0.5)
    sim = snapmod.from_system(s, precision="fp64", p_on0=0.5)
    m, met = _train_on_plain_events(snapmod, torch, sim, sweeps=2000, epochs=20)
    assert met["ce"] < 0.25 * met["ce_uniform"] and met["top1"] > 0.95 > met["top1_uniform"], met
    rank = star_arm_ranks(s)
    expect = star_expectation(s, math.exp(s.reactions[0].eps))
    acc = {}
    for mode in (1, 2):
        sim.set_bonds(np.zeros((0, 2), np.int64))
        sim.set_mh(mode, m if mode == 2 else None, eps_u=0.05)
        st0 = sim.stats()
        samples = []
        for t in range(8000):
            sim.set_step(t)
            sim.mh_sweep()
            if t >= 800 and t % 8 == 7:
                b = sim.bonds()
                dp = np.full((s.n, 4), -1, np.int64)
                dp[b[:, 0], 0] = b[:, 1]
                dp[b[:, 1], 0] = b[:, 0]
                samples.append(star_occupancy(dp, s, rank))
        st = sim.stats()
        d = {k: st["mh_" + k] - st0["mh_" + k] for k in MH_STATS}
        acc[mode] = (d["form_accepts"] + d["break_accepts"]) / (d["form_attempts"] + d["break_attempts"])
        mean, se = block_mean_se(np.array(samples))
        assert np.all(np.abs(mean - expect) < 4 * se + 0.01), (mode, mean, expect, se)
    assert acc[2] > 1.05 * acc[1], acc


def test_trained_proposal_on_dense_gel_keeps_bonded_fraction(snapmod, torch):
    """Dense colloid-linker gel (number density 0.8): trained on plain-run
    events, the learned MH proposal and the uniform one give the same bonded
    fraction under Langevin dynamics within the statistical error."""
    s = colloid_linker(seed=61, n_c=4000, n_l=16000, rho=0.8, eps=6.0)
    sim = snapmod.from_system(s, precision="mixed")
    sim.step(300)
    sim.log_events(1_000_000)
    sim.step(300)
    feat, off, lab = sim.get_events(clear=True)
    sim.log_events(0)
    assert len(lab) > 5000
    dX, doff, dlab = (torch.from_numpy(a).cuda() for a in (feat, off, lab))
    m = snapmod.Mlp(omlp.init(seed=2).astype(np.float32))
    losses = m.train(dX.data_ptr(), len(feat), doff.data_ptr(), dlab.data_ptr(), len(lab), epochs=40,
                     batch_events=1024, lr=2e-3, seed=3)
    assert losses[-1] < 0.6 * losses[0], losses
    state = sim.get_state()
    nb = {}
    for mode in (1, 2):
        sim.set_state(state)
        sim.set_mh(mode, m if mode == 2 else None)
        series = []
        for _ in range(60):
            sim.step(50)
            series.append(sim.stats()["n_bonds"])
        h = np.array(series[20:], float)
        nb[mode] = block_mean_se(h, nblocks=10)
    (m1, e1), (m2, e2) = nb[1], nb[2]
    assert abs(m1 - m2) < 4 * math.hypot(e1, e2) + 1e-3 * m1, nb
