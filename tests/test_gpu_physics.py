"""Physics of the GPU path at scale, against what the paper states (not the oracle).

* Fig. decay / Eqs. OmN, collmatD1Q3, D1Q3relax: the ensemble mean of the
  non-conserved moment pi relaxes as the mean-field recursion of one binary
  collision at a time predicts; the closed form with the constant that
  Eq. 1Ddecay implies (sqrt 8, reading c6) follows it, the printed 2 sqrt 6
  does not.  Without streaming the system relaxes to the local equilibrium,
  which lies slightly below the global one (the text after Eq. local).
* Fig. 1dPoisson (Sec. III.A): with an even number of rest particles at every
  site that parity never changes; n_0 follows the Poisson law restricted to
  even values while n_-1 and n_+1 stay Poisson.
"""
import math

import numpy as np
import pytest

from paper_1706_01094_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_01094_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1706_01094_gb300 import mclg  # noqa: E402


def pi_moment(n):
    """Ensemble mean of pi = sqrt(2) (n_-1 - n_0 / 2 + n_+1) (Sec. IV.A)."""
    m = n.astype(np.float64).mean(axis=1)
    return math.sqrt(2.0) * (m[0] - m[1] / 2 + m[2])


def mean_field(f, collisions, lam=1.0):
    """f^(n+1) = f^(n) + Omega^(1)(f^(n)) with Omega^(1) of Eq. collmatD1Q3."""
    f = np.array(f, dtype=np.float64)
    rho = f.sum()
    out = [f.copy()]
    for _ in range(collisions):
        d = f[1] ** 2 / 8 - 2 * f[0] * f[2]
        f = f + lam / rho ** 2 * np.array([d, -2 * d, d])
        out.append(f.copy())
    return out


def closed_form(pi0, n, rho, const):
    """Eq. D1Q3relax at u = 0 with the given constant (sqrt 8 or 2 sqrt 6) times rho."""
    a = const * rho
    return a * pi0 / (math.exp(n / rho) * (a + pi0) - pi0)


@pytest.mark.parametrize("sampler", [0, 1])
@pytest.mark.parametrize("start", [(0, 300, 0), (150, 0, 150)])
def test_pi_decay_follows_mean_field(start, sampler):
    R, Lr, C, steps = 1000, 1000, 10, 40
    L = np.full(R, Lr, dtype=np.uint32)
    n0 = np.tile(np.array(start, dtype=np.uint16)[:, None], (1, R * Lr))
    rho = float(sum(start))
    mf = mean_field(start, C * steps)
    with mclg.Lattice(L, seed=2024, sampler=sampler) as lat:
        lat.set_state(n0)
        measured = [pi_moment(n0)]
        for _ in range(steps):
            lat.step(1)
            n, _ = lat.get_state()
            measured.append(pi_moment(n))
    pi0 = measured[0]
    for k in range(0, steps + 1, 4):
        f = mf[C * k]
        pmf = math.sqrt(2.0) * (f[0] - f[1] / 2 + f[2])
        # fluctuation corrections are O(1); the initial |pi| is 212 or 424
        assert abs(measured[k] - pmf) < 1.5, (k, measured[k], pmf)
    # the closed form with sqrt 8 tracks the recursion; 2 sqrt 6 is further off
    err8 = max(abs(closed_form(pi0, C * k, rho, math.sqrt(8)) - measured[k]) for k in range(steps + 1))
    err24 = max(abs(closed_form(pi0, C * k, rho, 2 * math.sqrt(6)) - measured[k])
                for k in range(steps + 1))
    assert err8 < 2.5 and err24 > 2 * err8, (err8, err24)


def test_local_equilibrium_without_streaming_is_below_global():
    R, Lr, C = 200, 1000, 10
    L = np.full(R, Lr, dtype=np.uint32)
    n0 = np.tile(np.array([100, 100, 100], dtype=np.uint16)[:, None], (1, R * Lr))
    with mclg.Lattice(L, seed=5, flags=mclg.NO_STREAM) as lat:
        lat.set_state(n0)
        lat.step(300)
        n_local, _ = lat.get_state()
    with mclg.Lattice(L, seed=5) as lat:
        lat.set_state(n0)
        lat.step(300)
        n_global, _ = lat.get_state()
    # u = 0 on average: pi^eq = 0 globally; the local equilibrium sits O(1) below
    p_loc, p_glob = pi_moment(n_local), pi_moment(n_global)
    assert abs(p_glob) < 0.3, p_glob
    assert -3.0 < p_loc < -0.3, p_loc


def test_even_rest_particles_keep_parity_and_restricted_poisson():
    R, Lr = 2000, 100  # the paper's lattice length, many independent lattices
    L = np.full(R, Lr, dtype=np.uint32)
    S = R * Lr
    g = np.random.default_rng(11)
    n = np.zeros((3, S), dtype=np.uint16)
    n[0] = g.poisson(2.0, S)
    n[2] = g.poisson(2.0, S)
    z = g.poisson(8.0, 4 * S)
    n[1] = z[z % 2 == 0][:S]                  # Poisson(8) restricted to even values
    hist = {0: np.zeros(64), 1: np.zeros(64), 2: np.zeros(64)}
    with mclg.Lattice(L, seed=3) as lat:
        lat.set_state(n)
        lat.step(300)
        for _ in range(60):
            lat.step(10)
            cur, _ = lat.get_state()
            assert (cur[1] % 2 == 0).all()     # the spurious invariant of Sec. III.A
            for i in range(3):
                hist[i] += np.bincount(np.minimum(cur[i], 63), minlength=64)[:64]
    k = np.arange(64)
    logfact = np.array([math.lgamma(v + 1) for v in k])
    for i, mu in ((0, 2.0), (2, 2.0)):
        p = np.exp(-mu + k * math.log(mu) - logfact)
        emp = hist[i] / hist[i].sum()
        sel = p > 1e-3
        assert np.all(np.abs(emp[sel] - p[sel]) < 0.02 * p[sel] + 3e-4), (i, emp[:8], p[:8])
    mu = 8.0
    p = np.where(k % 2 == 0, np.exp(-mu + k * math.log(mu) - logfact), 0.0)
    p /= p.sum()
    emp = hist[1] / hist[1].sum()
    assert emp[1::2].sum() == 0.0
    sel = p > 1e-3
    assert np.all(np.abs(emp[sel] - p[sel]) < 0.02 * p[sel] + 3e-4), (emp[:12], p[:12])


def relaxation_rate(state, flags, sampler, R=1000, Lr=100, steps=40):
    """Collide-only decay rate per step of the ensemble-mean rest count towards its
    equilibrium, from identical nodes (N and J stay fixed at every node)."""
    L = np.full(R, Lr, dtype=np.uint32)
    n0 = np.tile(np.array(state, dtype=np.uint16)[:, None], (1, R * Lr))
    means = []
    with mclg.Lattice(L, seed=31, flags=mclg.NO_STREAM | flags, sampler=sampler) as lat:
        lat.set_state(n0)
        means.append(float(n0[1].mean()))
        for _ in range(steps):
            lat.step(1)
            means.append(float(lat.get_state()[0][1].astype(np.float64).mean()))
        lat.step(400)
        tail = []
        for _ in range(20):
            lat.step(5)
            tail.append(float(lat.get_state()[0][1].astype(np.float64).mean()))
    dev = np.array(means) - np.mean(tail)
    k = np.arange(len(dev))
    use = np.abs(dev) > 4.0
    slope = np.polyfit(k[use], np.log(np.abs(dev[use])), 1)[0]
    return -slope


@pytest.mark.parametrize("sampler", [0, 1])
def test_galilean_rate_makes_relaxation_independent_of_u(sampler):
    """Eq. D1Q3relax: the pi mode relaxes with rate C lambda sqrt(1 + 3u^2) / rho per
    step near equilibrium.  With lambda = lambda~ / sqrt(1 + 3u^2) (end of Sec. IV.A)
    the rate at u = 0.3 equals the one at rest; with a constant lambda it is
    sqrt(1.27) = 1.127 times larger."""
    at_rest = (40, 220, 40)      # N = 300, J = 0, b 20 above equilibrium
    moving = (8, 194, 98)        # N = 300, J = 90 (u = 0.3), b ~ 20 above equilibrium
    r0 = relaxation_rate(at_rest, mclg.GALILEAN, sampler)
    r1 = relaxation_rate(moving, mclg.GALILEAN, sampler)
    c0 = relaxation_rate(at_rest, 0, sampler)
    c1 = relaxation_rate(moving, 0, sampler)
    assert abs(r1 / r0 - 1.0) < 0.04, (r0, r1)
    assert abs(c1 / c0 - math.sqrt(1.27)) < 0.04, (c0, c1)
    assert abs(c0 - 10.0 / 300.0) < 0.1 * 10.0 / 300.0, c0   # C lambda / N at u = 0


def eq_a_amplitude(profile):
    """Eq. A: least-squares amplitude of sin(2 pi x / L) in a profile."""
    L = profile.size
    s = np.sin(2.0 * np.pi * np.arange(L) / L)
    return float((s * profile).sum() / (s * s).sum())


def mean_field_lattice(f, steps, C=10, lam=1.0):
    """The MCLG's mean-field dynamics on one periodic lattice: C applications of the
    one-collision mean-field map of Eqs. OmN / collmatD1Q3 at every node, then the
    streaming of the evolution equation (Sec. III).  Yields rho(x) after each step."""
    f = np.array(f, dtype=np.float64)
    for _ in range(steps):
        rho = f.sum(axis=0)
        for _ in range(C):
            d = f[1] ** 2 / 8 - 2 * f[0] * f[2]
            f = f + lam / rho ** 2 * np.stack([d, -2 * d, d])
        f = np.stack([np.roll(f[0], -1), f[1], np.roll(f[2], 1)])
        yield f.sum(axis=0)


def sound_wave_deviation(rho0, sampler, R=1024, Lr=512, steps=3000, every=50):
    """Largest |A_MCLG(t) - A_mean-field(t)| / A(0) over the run, with A the Eq. A
    amplitude of the ensemble-mean density of a 10 % sine wave at density rho0."""
    x = np.arange(Lr)
    rho = rho0 * (1.0 + 0.1 * np.sin(2.0 * np.pi * x / Lr))
    L = np.full(R, Lr, dtype=np.uint32)

    def amplitude(n):
        return eq_a_amplitude(n.astype(np.float64).sum(axis=0).reshape(R, Lr).mean(axis=0) - rho0)

    amps = []
    with mclg.Lattice(L, seed=77, sampler=sampler) as lat:
        lat.init(np.tile(rho, R), np.zeros(R * Lr))
        amps.append(amplitude(lat.get_state()[0]))
        for _ in range(steps // every):
            lat.step(every)
            amps.append(amplitude(lat.get_state()[0]))
    f0 = np.stack([rho / 6, 2 * rho / 3, rho / 6])
    mf = [eq_a_amplitude(f0.sum(axis=0) - rho0)]
    for k, prof in enumerate(mean_field_lattice(f0, steps), start=1):
        if k % every == 0:
            mf.append(eq_a_amplitude(prof - rho0))
    amps, mf = np.array(amps), np.array(mf)
    a0 = 0.1 * rho0
    assert abs(mf[0] - a0) < 1e-9 * a0 and abs(amps[0] - a0) < 0.02 * a0
    assert mf.min() < -0.4 * a0 and abs(mf[-1]) < 0.8 * a0     # it oscillates and decays
    return float(np.abs(amps - mf).max() / a0)


@pytest.mark.parametrize("sampler", [0, 1])
def test_sound_wave_amplitude_approaches_mean_field(sampler):
    """A 10 % density wave on 1024 replicas of L = 512 (Eq. A fit of the
    ensemble-mean density every 50 steps, three sound periods): the MCLG's
    ensemble average follows the mean-field lattice Boltzmann dynamics of the
    same collision operator (Eqs. OmN, collmatD1Q3), up to corrections of order
    1/rho that come from averaging ac/N^2 over the node's fluctuating mass: within
    1.5 % at rho = 200, and at least twice as close as at rho = 50."""
    d50 = sound_wave_deviation(50.0, sampler)
    d200 = sound_wave_deviation(200.0, sampler)
    assert d200 < 0.015, (d50, d200)
    assert d50 > 2.0 * d200, (d50, d200)
