"""The D2Q9 lattice gas on the GPU (mclg2d_* through the C ABI): bit for bit
against the oracle, and the physics the paper states for it: relaxation to the
entropic product equilibrium of Eq. D2Q9eqdist with Poisson fluctuations (Eq.
poisson), and the decay of a shear wave at the viscosity of Eqs. Decay, nu and
tausigma."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1706_01094_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1706_01094_gb300 import mclg  # noqa: E402

PAPER = mclg.D2Q9_PAPER_LAMBDA


def run2(Lx, Ly, R, seed, n0, t0, steps, **kw):
    with mclg.Lattice2D(Lx, Ly, R, seed=seed, **kw) as lat:
        lat.set_state(n0, t=t0)
        lat.step(steps)
        out, t = lat.get_state()
        assert t == t0 + steps
    return out


@pytest.mark.parametrize("Lx,Ly,R,C,lam,flags", [
    (7, 5, 3, 10, PAPER, 0), (100, 10, 1, 10, PAPER, 0), (1, 1, 4, 10, PAPER, 0),
    (64, 33, 2, 1, PAPER, 0), (9, 13, 2, 37, ((128, 64, 32, 16, 8, 4, 2, 1, 96), 128), 0),
    (16, 16, 2, 10, ((1, 2, 3, 4, 5, 6, 7, 8, 9), 37), 0), (12, 7, 3, 10, PAPER, mclg.NO_STREAM)])
def test_d2q9_bit_exact(Lx, Ly, R, C, lam, flags):
    g = np.random.default_rng(Lx * 100 + Ly)
    n0 = g.poisson(7.0, size=(9, Lx * Ly * R)).astype(np.uint16)
    oflags = oracle.FLAG_NO_STREAM if flags & mclg.NO_STREAM else 0
    want, err = oracle.d2q9_step(Lx, Ly, R, 31, n0, 5, 9, C=C, lam=lam, flags=oflags,
                                 first_replica=2)
    assert err == 0
    got = run2(Lx, Ly, R, 31, n0, 5, 9, C=C, lam=lam, flags=flags, first_replica=2)
    assert np.array_equal(got, want)


def test_d2q9_init_and_moments_equal_oracle():
    Lx, Ly, R = 40, 25, 3
    S = Lx * Ly * R
    g = np.random.default_rng(2)
    rho = g.uniform(5, 300, S)
    ux, uy = g.uniform(-0.3, 0.3, S), g.uniform(-0.3, 0.3, S)
    want, err = oracle.d2q9_init(Lx, Ly, R, 8, rho, ux, uy)
    assert err == 0
    with mclg.Lattice2D(Lx, Ly, R, seed=8) as lat:
        lat.init(rho, ux, uy)
        got, t = lat.get_state()
        assert t == 0 and np.array_equal(got, want)
        d = [torch.empty(S, dtype=torch.int32, device="cuda") for _ in range(3)]
        tot = lat.moments(*d)
        r, jx, jy, otot = oracle.d2q9_moments(want)
        assert np.array_equal(tot, otot)
        for a, b in zip(d, (r, jx, jy)):
            assert np.array_equal(a.cpu().numpy(), b)
        lat.step(20)
        assert np.array_equal(lat.moments(), otot)   # mass and momentum conserved
    with pytest.raises(mclg.MCLGError):          # a pick whose outcomes exceed probability 1
        mclg.Lattice2D(4, 4, lam=((1, 1, 128, 128, 1, 128, 1, 1, 1), 128))


def test_d2q9_relaxes_to_poisson_fluctuations_around_the_entropic_equilibrium():
    """From a deterministic start (every node the same counts, no fluctuations)
    the lattice relaxes to the global equilibrium: time-averaged occupation means
    equal f^eq(rho, u) of Eq. D2Q9eqdist with the conserved density and velocity,
    and their variances equal the means (Eq. poisson), with the paper's rates at
    rho = 36, u = (0.1, 0.25) (the setting of Fig. n0ton4)."""
    Lx, Ly, R = 32, 10, 64
    S = Lx * Ly * R
    f0 = oracle.d2q9_feq(36.0, 0.1, 0.25)
    n0 = np.repeat(np.rint(f0).astype(np.uint16)[:, None], S, axis=1)
    N, Jx, Jy = int(n0.sum()), int((n0.T @ np.array(oracle.D2Q9_VX)).sum()), \
        int((n0.T @ np.array(oracle.D2Q9_VY)).sum())
    f = oracle.d2q9_feq(N / S, Jx / N, Jy / N)
    means, varis = [], []
    with mclg.Lattice2D(Lx, Ly, R, seed=5) as lat:
        lat.set_state(n0)
        lat.step(400)
        for _ in range(60):
            lat.step(5)
            st, _ = lat.get_state()
            x = st.astype(np.float64)
            means.append(x.mean(axis=1))
            varis.append(x.var(axis=1))
    m, v = np.mean(means, axis=0), np.mean(varis, axis=0)
    assert np.allclose(m, f, rtol=4e-3), (m, f)
    assert np.allclose(v, f, rtol=0.03), (v, f)


def test_d2q9_shear_wave_decays_at_the_predicted_viscosity():
    """u_x = A sin(2 pi y / L_y) at rho = 500 (Sec. IV.B): the amplitude of the
    x-averaged profile decays as exp(-4 pi^2 nu t / L_y^2) with nu = (tau - 1/2) / 3
    and tau from Eq. tausigma for the paper's rates; C chosen for tau = 1.5."""
    lam = [n / PAPER[1] for n in PAPER[0]]
    rate_sum = 8 * lam[0] + lam[2] + 2 * (lam[3] + lam[5] + 2 * lam[6] + 4 * lam[7])
    rho0, Lx, Ly, R, A = 500.0, 32, 64, 8, 0.1
    C = int(round(-math.log(1 - 1 / 1.5) * 9 * rho0 / rate_sum))
    tau = 1 / (1 - math.exp(-C * rate_sum / (9 * rho0)))
    nu = (tau - 0.5) / 3
    S = Lx * Ly * R
    y = np.tile(np.repeat(np.arange(Ly), Lx), R)
    ux = A * np.sin(2 * np.pi * y / Ly)
    sinus = np.sin(2 * np.pi * np.arange(Ly) / Ly)
    times, amps = [], []
    with mclg.Lattice2D(Lx, Ly, R, seed=12, C=C) as lat:
        lat.init(np.full(S, rho0), ux, np.zeros(S))
        for k in range(7):
            st, t = lat.get_state()
            x = st.astype(np.float64).reshape(9, R, Ly, Lx)
            jx = np.tensordot(np.array(oracle.D2Q9_VX, dtype=float), x, axes=1)
            uprof = (jx / x.sum(axis=0)).mean(axis=(0, 2))
            times.append(t)
            amps.append(2 / Ly * (uprof * sinus).sum())
            lat.step(50)
    slope = np.polyfit(times, np.log(amps), 1)[0]
    want = -4 * np.pi**2 * nu / Ly**2
    assert abs(slope / want - 1) < 0.06, (slope, want, tau, C)
