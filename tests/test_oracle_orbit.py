"""Pins for the oracle's orbit-dependent neighbour criterion (Sec. 6.3.1,
Eq. 24): the Kepler pericentre against closed forms and numerical orbit
integration, and the two-stage neighbour sets against brute force,
special cases and invariants."""
import math

import numpy as np
import pytest

import oracle
from paper_2006_16560_gb300 import inputs


def _rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


def _state(e, p, f, mu, R):
    """Relative position/velocity at true anomaly f of a conic (e, p)."""
    r = p / (1 + e * math.cos(f))
    x = r * np.array([math.cos(f), math.sin(f), 0.0])
    s = math.sqrt(mu / p)
    v = s * np.array([-math.sin(f), e + math.cos(f), 0.0])
    return R @ x, R @ v


@pytest.mark.parametrize("e", [0.0, 0.3, 0.9, 1.0, 2.5, 40.0])
def test_pericentre_closed_form(e):
    rng = np.random.default_rng(int(e * 10))
    for _ in range(20):
        p, mu = rng.uniform(0.1, 3), rng.uniform(0.1, 5)
        fmax = math.pi * 0.95 if e < 1 else math.acos(-1 / e) * 0.9
        f = rng.uniform(-fmax, fmax)
        x, v = _state(e, p, f, mu, _rotation(rng))
        assert oracle.pericentre(x, v, mu) == pytest.approx(p / (1 + e), rel=1e-11)


def test_pericentre_limits():
    x = np.array([0.3, -0.4, 1.2])
    assert oracle.pericentre(x, np.zeros(3), 2.0) == pytest.approx(np.linalg.norm(x), rel=1e-15)
    assert oracle.pericentre(x, -0.7 * x, 2.0) < 1e-30          # radial infall
    assert oracle.pericentre(x, 0.7 * x, 0.0) < 1e-15           # radial, no gravity
    v = np.array([1.0, 0.5, -0.2])
    b = np.linalg.norm(np.cross(x, v)) / np.linalg.norm(v)      # impact parameter
    assert oracle.pericentre(x, v, 0.0) == pytest.approx(b, rel=1e-14)
    assert oracle.pericentre(x, v, 1e-12) == pytest.approx(b, rel=1e-9)
    # circular orbit: the pericentre is the current radius
    R = _rotation(np.random.default_rng(3))
    x, v = R @ np.array([2.0, 0, 0]), R @ np.array([0, math.sqrt(0.5 / 2.0), 0])
    assert oracle.pericentre(x, v, 0.5) == pytest.approx(2.0, rel=1e-13)


def _min_separation(x, v, mu, t_end, nstep):
    """Smallest |x| along the two-body orbit, integrated both ways from the
    given state with RK4 in the regularised time s (dt = r ds, so the steps
    shrink near pericentre); the minimum is refined by a parabola through
    the three samples around it."""
    best = np.linalg.norm(x)

    def f(y):
        r = np.linalg.norm(y[:3])
        return np.concatenate([r * y[3:6], -mu * y[:3] / r ** 2, [r]])
    for sgn in (1.0, -1.0):
        y = np.concatenate([x, sgn * v, [0.0]])
        ds = t_end / np.linalg.norm(x) / nstep
        rs = [np.linalg.norm(x)]
        while y[6] < t_end and len(rs) < 40 * nstep:
            k1 = f(y)
            k2 = f(y + 0.5 * ds * k1)
            k3 = f(y + 0.5 * ds * k2)
            k4 = f(y + ds * k3)
            y = y + ds / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            rs.append(np.linalg.norm(y[:3]))
            if rs[-1] > rs[-2] and rs[-1] > 4 * rs[0]:      # receding for good
                break
        rs = np.array(rs)
        k = int(np.argmin(rs))
        if 0 < k < len(rs) - 1:
            a, b, c = rs[k - 1], rs[k], rs[k + 1]
            den = a - 2 * b + c
            rmin = b - (a - c) ** 2 / (8 * den) if den > 0 else b
        else:
            rmin = rs[k]
        best = min(best, rmin)
    return best


def test_pericentre_against_integration():
    """Brute force: the minimum separation of the numerically integrated orbit."""
    rng = np.random.default_rng(7)
    for _ in range(8):
        x = rng.normal(size=3)
        mu = rng.uniform(0.5, 2)
        vc = math.sqrt(mu / np.linalg.norm(x))
        v = rng.normal(size=3) * vc * rng.uniform(0.3, 1.2)
        r = np.linalg.norm(x)
        E = 0.5 * v @ v - mu / r
        t_end = 2 * math.pi * (mu / (-2 * E)) ** 1.5 if E < 0 else 20 * r / math.sqrt(v @ v)
        rmin = _min_separation(x, v, mu, t_end, 4000)
        assert oracle.pericentre(x, v, mu) == pytest.approx(rmin, rel=1e-6)


def test_rnb_special_cases():
    rng = np.random.default_rng(1)
    vel = rng.normal(size=(50, 3))
    s = rng.uniform(1, 3, 50)
    assert np.array_equal(oracle.neighbour_radius(np.zeros((50, 3)), 0.01, 0.5, 3.0, s), 0.01 * s)
    a = oracle.neighbour_radius(vel, 0.0, 1.0, 1.0)
    np.testing.assert_allclose(a, np.linalg.norm(vel, axis=1), rtol=1e-15)
    b = oracle.neighbour_radius(vel, 0.01, 0.25, 3.0)
    np.testing.assert_allclose(b - 0.01, 0.75 * a, rtol=1e-12)


def _sets(off, idx):
    return [set(idx[off[i]:off[i + 1]].tolist()) for i in range(len(off) - 1)]


def test_zero_velocity_reduces_to_rout_neighbours():
    d = inputs.plummer(1500, 3, masses="kroupa")
    s = oracle.radius_scale(d["mass"])
    vel = np.zeros((1500, 3))
    for mode in (oracle.ORBIT_CANDIDATES, oracle.ORBIT_ROUT):
        off, idx, _ = oracle.orbit_neighbours(d["pos"], vel, d["mass"], 0.05, 0.1, mode=mode, scale=s)
        o2, i2 = oracle.neighbours(d["pos"], 0.05, scale=s)
        assert np.array_equal(off, o2) and np.array_equal(idx, i2)


def _small_cluster(n, seed):
    d = inputs.plummer(n, seed)
    rng = np.random.default_rng(seed)
    vel = d["vel"] if "vel" in d else rng.normal(size=(n, 3)) * 0.5
    return d["pos"], vel, d["mass"]


def test_against_integrated_orbits_brute_force():
    """Tiny set: stage 1 from the plain distance test, stage 2 from the
    integrated minimum separation of every candidate pair."""
    N = 24
    pos, vel, mass = _small_cluster(N, 11)
    mass = mass * N                  # total mass N: strong pair orbits
    r_out, dt, C_r, C_v = 0.12, 0.25, 3.0, 1.5
    off, idx, ncand = oracle.orbit_neighbours(pos, vel, mass, r_out, dt, C_r, C_v)
    got = _sets(off, idx)
    sp = np.linalg.norm(vel, axis=1)
    rnb = r_out + C_r * sp * dt
    near = 0
    n_drop = 0
    memo = {}
    for i in range(N):
        cand, keep, close = set(), set(), set()
        for j in range(N):
            if j == i:
                continue
            x = pos[j] - pos[i]
            if np.linalg.norm(x) >= max(rnb[i], rnb[j]):
                continue
            cand.add(j)
            key = (min(i, j), max(i, j))
            if key not in memo:                     # the pair's orbit is symmetric
                v = vel[j] - vel[i]
                mu = mass[i] + mass[j]
                r = np.linalg.norm(x)
                E = 0.5 * v @ v - mu / r
                t_end = 2 * math.pi * (mu / (-2 * E)) ** 1.5 if E < 0 else 20 * r / math.sqrt(v @ v)
                memo[key] = _min_separation(x, v, mu, t_end, 800)
            rmin = memo[key]
            if abs(rmin - C_v * r_out) < 1e-3 * r_out:
                near += 1
                close.add(j)
                continue
            if rmin < C_v * r_out:
                keep.add(j)
        assert ncand[i] == len(cand)
        assert got[i] <= cand and got[i] - close == keep
        n_drop += len(cand - got[i])
    assert near <= 2 and n_drop > 0


def test_invariants():
    pos, vel, mass = _small_cluster(2000, 5)
    vel = vel.copy()
    vel[::97] *= 30                  # a few high-velocity particles
    s = oracle.radius_scale(mass)
    kw = dict(r_out=0.03, dt=0.02, C_r=3.0, scale=s)
    cand = _sets(*oracle.orbit_neighbours(pos, vel, mass, mode=oracle.ORBIT_CANDIDATES, **kw)[:2])
    keep = _sets(*oracle.orbit_neighbours(pos, vel, mass, C_v=1.5, **kw)[:2])
    printed = _sets(*oracle.orbit_neighbours(pos, vel, mass, C_v=1.5, mode=oracle.ORBIT_RNB, **kw)[:2])
    rout = _sets(*oracle.neighbours(pos, 0.03, scale=s))
    n_drop = 0
    for i in range(2000):
        for j in cand[i]:
            assert i in cand[j]                      # symmetric
        for j in keep[i]:
            assert i in keep[j]
        assert rout[i] <= keep[i] <= cand[i]        # r_out pairs always kept
        assert printed[i] == cand[i]                 # pericentre <= separation
        n_drop += len(cand[i] - keep[i])
    assert n_drop > 0


def test_fast_particle_keeps_only_its_path():
    """Massless field particles at rest around a fast one moving along +x:
    those ahead within C_v r_out of its line are kept, the ones to the side
    are dropped (Sec. 6.3.1: only neighbours along the path matter)."""
    r_out, dt, C_r, C_v = 0.01, 1.0, 3.0, 1.5
    ahead = [[0.2, 0.0, 0.0], [0.5, 0.01, 0.0], [-0.3, 0.0, 0.012]]
    side = [[0.0, 0.3, 0.0], [0.2, 0.0, 0.2], [0.0, -0.02, 0.0]]
    pos = np.array([[0.0, 0.0, 0.0]] + ahead + side)
    vel = np.zeros_like(pos)
    vel[0] = [0.3, 0.0, 0.0]                          # r_nb,0 = 0.01 + 0.9
    mass = np.zeros(len(pos))
    off, idx, ncand = oracle.orbit_neighbours(pos, vel, mass, r_out, dt, C_r, C_v)
    assert ncand[0] == 6
    assert set(idx[off[0]:off[1]].tolist()) == {1, 2, 3}
