"""Seeded synthetic inputs for the P3T long-range force.

This module draws particle sets only; it contains none of the force method's
arithmetic, so the CUDA path and the CPU oracle can both consume its arrays.

The paper generates its star clusters rather than loading a dataset
(Sec. 7.1.1): Plummer spheres in Henon (N-body) units with a Kroupa (2001)
mass function, optionally with every star in a primordial binary.  The
generators here reproduce that structure:

* ``plummer``      -- Plummer positions by the inverse cumulative mass
                      profile (Aarseth, Henon & Wielen 1974), truncated at
                      mass fraction 0.999, isotropic velocities by rejection
                      sampling of q^2 (1 - q^2)^(7/2); a = 3 pi / 16, G = M = 1;
                      centre of mass and mean velocity removed.
* ``kroupa_masses`` -- two-segment power law, slope 1.3 on [0.08, 0.5] and
                      2.3 on [0.5, mmax] solar masses, rescaled to total 1.
* ``plummer_binaries`` -- Plummer centres each carrying a binary with
                      log-uniform semi-major axis in AU (1 AU = 3.726e-6 NB
                      for a 1 pc half-mass radius), thermal eccentricity,
                      uniform mean anomaly and random orientation.
* ``kroupa95_binaries`` -- the paper's own binary population (Sec. 7.1.1,
                      Eq. 39): every star in a binary, periods from the
                      Kroupa (1995) distribution truncated to log10 P in
                      [1, 8.43] days, thermal eccentricities, Kroupa masses
                      0.08-40 Msun, Kepler's third law for the semi-major axes.
* ``cluster_ensemble`` -- many independent clusters with log-uniform sizes.
* ``wide_sparse_groups`` -- an adversarial layout for the mixed-precision
                      near/far decision: two sparse walk groups tens of
                      thousands of r_out wide whose members pair up across
                      the face between them at r_out (1 -+ 1e-4).

Every array is float64; positions are (n, 3) row-major.
"""
from __future__ import annotations

import math

import numpy as np

PLUMMER_A = 3.0 * math.pi / 16.0
"""Plummer scale length in Henon units (G = M = 1, E = -1/4)."""

PLUMMER_XMAX = 0.999
"""Mass-fraction truncation of the Plummer sampler (r_max ~ 22.8)."""

AU_IN_NB = 4.84813681109536e-06 / (1.0 / 0.7686)
"""1 AU in N-body length units when the half-mass radius (0.7686 NB) is 1 pc."""


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    cost = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sint = np.sqrt(1.0 - cost * cost)
    return np.stack([sint * np.cos(phi), sint * np.sin(phi), cost], axis=1)


def kroupa_masses(n: int, rng: np.random.Generator, mmin: float = 0.08,
                  mmax: float = 150.0, mbreak: float = 0.5) -> np.ndarray:
    """Draw n masses (solar units) from the two-segment Kroupa (2001) IMF."""
    a1, a2 = 1.3, 2.3
    # integrals of m^-a over each segment, continuous at mbreak
    i1 = (mbreak ** (1 - a1) - mmin ** (1 - a1)) / (1 - a1)
    c2 = mbreak ** (a2 - a1)            # continuity factor for segment 2
    i2 = c2 * (mmax ** (1 - a2) - mbreak ** (1 - a2)) / (1 - a2)
    u = rng.uniform(0.0, 1.0, n) * (i1 + i2)
    m = np.empty(n)
    lo = u < i1
    m[lo] = (mmin ** (1 - a1) + u[lo] * (1 - a1)) ** (1.0 / (1 - a1))
    hi = ~lo
    m[hi] = (mbreak ** (1 - a2) + (u[hi] - i1) / c2 * (1 - a2)) ** (1.0 / (1 - a2))
    return m


def plummer(n: int, seed: int, masses: str = "equal", mmax: float = 150.0,
            rng: np.random.Generator | None = None) -> dict:
    """Plummer sphere of n particles in Henon units.

    Returns ``{"pos": (n,3), "vel": (n,3), "mass": (n,)}``; masses are
    "equal" (1/n each) or "kroupa" (rescaled to total mass 1).
    """
    if rng is None:
        rng = rng_for(seed)
    a = PLUMMER_A
    x = rng.uniform(0.0, PLUMMER_XMAX, n)
    x = np.maximum(x, 1e-300)
    r = a / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
    pos = _isotropic(rng, n) * r[:, None]
    # speeds: q = v / v_esc with density q^2 (1 - q^2)^(7/2), max 0.0920
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        qq = rng.uniform(0.0, 1.0, todo.size)
        yy = rng.uniform(0.0, 0.1, todo.size)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
    vesc = math.sqrt(2.0) * (1.0 + (r / a) ** 2) ** (-0.25) / math.sqrt(a)
    vel = _isotropic(rng, n) * (q * vesc)[:, None]
    if masses == "equal":
        mass = np.full(n, 1.0 / n)
    elif masses == "kroupa":
        mass = kroupa_masses(n, rng, mmax=mmax)
        mass /= mass.sum()
    else:
        raise ValueError(f"unknown mass model {masses!r}")
    pos -= (mass[:, None] * pos).sum(0) / mass.sum()
    vel -= (mass[:, None] * vel).sum(0) / mass.sum()
    return {"pos": np.ascontiguousarray(pos), "vel": np.ascontiguousarray(vel),
            "mass": np.ascontiguousarray(mass)}


def _kepler_E(M: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Eccentric anomaly from mean anomaly by Newton iteration."""
    E = np.where(e < 0.8, M, np.pi * np.ones_like(M))
    for _ in range(60):
        f = E - e * np.sin(E) - M
        E = E - f / (1.0 - e * np.cos(E))
    return E


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """n uniformly random rotation matrices from unit quaternions."""
    qv = rng.normal(size=(n, 4))
    qv /= np.linalg.norm(qv, axis=1, keepdims=True)
    w, x, y, z = qv.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _orbit_state(a, e, E, mu, R):
    """Relative position and velocity of two-body orbits (semi-major axis a,
    eccentricity e, eccentric anomaly E, mu = G (m1 + m2)), rotated by R."""
    c, s = np.cos(E), np.sin(E)
    q = np.sqrt(1.0 - e * e)
    rel = np.stack([a * (c - e), a * q * s, np.zeros_like(a)], axis=1)
    w = np.sqrt(mu / a) / (1.0 - e * c)              # mean motion * a / (r / a)
    vrel = np.stack([-w * s, w * q * c, np.zeros_like(a)], axis=1)
    return np.einsum("kij,kj->ki", R, rel), np.einsum("kij,kj->ki", R, vrel)


def _members(cen, m1, m2, rel, vrel):
    """Member positions / velocities (2k, 2k+1) about the pair centres."""
    mt = m1 + m2
    n = len(m1)
    pos = np.empty((2 * n, 3))
    vel = np.empty((2 * n, 3))
    pos[0::2] = cen["pos"] - (m2 / mt)[:, None] * rel
    pos[1::2] = cen["pos"] + (m1 / mt)[:, None] * rel
    vel[0::2] = cen["vel"] - (m2 / mt)[:, None] * vrel
    vel[1::2] = cen["vel"] + (m1 / mt)[:, None] * vrel
    return pos, vel


def plummer_binaries(n_pairs: int, seed: int, amin_au: float = 0.005,
                     amax_au: float = 50.0) -> dict:
    """Plummer cluster in which every star is in a binary (2*n_pairs stars).

    Components of pair k are particles 2k and 2k+1; both masses are Kroupa
    draws and the whole set is rescaled to total mass 1.
    """
    rng = rng_for(seed)
    cen = plummer(n_pairs, seed, masses="equal", rng=rng)
    m1 = kroupa_masses(n_pairs, rng)
    m2 = kroupa_masses(n_pairs, rng)
    tot = m1.sum() + m2.sum()
    m1 /= tot
    m2 /= tot
    a = np.exp(rng.uniform(math.log(amin_au), math.log(amax_au), n_pairs)) * AU_IN_NB
    e = np.sqrt(rng.uniform(0.0, 1.0, n_pairs))        # thermal: f(e) = 2e
    Manom = rng.uniform(0.0, 2.0 * math.pi, n_pairs)
    E = _kepler_E(Manom, e)
    rel, vrel = _orbit_state(a, e, E, m1 + m2, _random_rotations(rng, n_pairs))
    pos, vel = _members(cen, m1, m2, rel, vrel)
    mass = np.empty(2 * n_pairs)
    mass[0::2] = m1
    mass[1::2] = m2
    pos -= (mass[:, None] * pos).sum(0)
    vel -= (mass[:, None] * vel).sum(0)
    return {"pos": np.ascontiguousarray(pos), "vel": np.ascontiguousarray(vel), "mass": mass,
            "semi_major": a}


KROUPA95_LOGP_MIN = 1.0      # log10 of the period in days (Sec. 7.1.1)
KROUPA95_LOGP_MAX = 8.43


def kroupa95_log_periods(n: int, rng: np.random.Generator) -> np.ndarray:
    """log10 P [days] from Eq. 39, F(P) = 2.5 (lg P - 1) / (45 + (lg P - 1)^2),
    truncated to [1, 8.43]: with x = lg P - 1 the cumulative distribution is
    ln(1 + x^2/45) / ln(1 + x_max^2/45), inverted in closed form."""
    xmax = KROUPA95_LOGP_MAX - KROUPA95_LOGP_MIN
    u = rng.uniform(0.0, 1.0, n)
    x = np.sqrt(45.0 * ((1.0 + xmax * xmax / 45.0) ** u - 1.0))
    return KROUPA95_LOGP_MIN + x


def kroupa95_binaries(n_pairs: int, seed: int, mmin: float = 0.08, mmax: float = 40.0) -> dict:
    """Plummer cluster with 100% primordial binaries drawn like the paper's
    N1kb..N1mkb models (Sec. 7.1.1): Kroupa IMF 0.08-40 Msun, periods from
    Eq. 39, thermal eccentricity, half-mass radius 1 pc.  The pre-main-sequence
    eigenevolution adjustment of tight orbits that the paper also applies is
    not modelled.  Components of pair k are particles 2k and 2k+1."""
    rng = rng_for(seed)
    cen = plummer(n_pairs, seed, masses="equal", rng=rng)
    m1 = kroupa_masses(n_pairs, rng, mmin=mmin, mmax=mmax)
    m2 = kroupa_masses(n_pairs, rng, mmin=mmin, mmax=mmax)
    lgp = kroupa95_log_periods(n_pairs, rng)
    p_yr = 10.0 ** lgp / 365.25
    a_au = ((m1 + m2) * p_yr * p_yr) ** (1.0 / 3.0)          # Kepler's third law, solar units
    tot = m1.sum() + m2.sum()
    a = a_au * AU_IN_NB
    e = np.sqrt(rng.uniform(0.0, 1.0, n_pairs))
    Manom = rng.uniform(0.0, 2.0 * math.pi, n_pairs)
    E = _kepler_E(Manom, e)
    rel, vrel = _orbit_state(a, e, E, (m1 + m2) / tot, _random_rotations(rng, n_pairs))
    pos, vel = _members(cen, m1, m2, rel, vrel)
    mass = np.empty(2 * n_pairs)
    mass[0::2] = m1 / tot
    mass[1::2] = m2 / tot
    pos -= (mass[:, None] * pos).sum(0)
    vel -= (mass[:, None] * vel).sum(0)
    return {"pos": np.ascontiguousarray(pos), "vel": np.ascontiguousarray(vel), "mass": mass,
            "semi_major": a, "log_period_days": lgp, "ecc": e, "m1_msun": m1, "m2_msun": m2}


def r_out_first_guess(n: int, total_mass: float = 1.0, sigma2: float = 1.0 / 6.0) -> float:
    """Sec. 7.1.1, Eq. 42: r_out = 0.1 G M / (3 N^(1/3) sigma_1D^2)."""
    return 0.1 * total_mass / (3.0 * n ** (1.0 / 3.0) * sigma2)


def cluster_ensemble(n_clusters: int, nmin: int, nmax: int, seed: int,
                     masses: str = "kroupa") -> list[dict]:
    """Independent Plummer clusters with log-uniform particle counts.

    Each cluster also carries its own changeover radii from the first-guess
    recipe (r_out from Eq. 42, r_in = r_out / 10 as in Table 2).
    """
    rng = rng_for(seed)
    sizes = np.exp(rng.uniform(math.log(nmin), math.log(nmax), n_clusters)).astype(np.int64)
    seeds = rng.integers(1, 2 ** 31 - 1, n_clusters)
    out = []
    for n, s in zip(sizes, seeds):
        c = plummer(int(n), int(s), masses=masses)
        c["r_out"] = r_out_first_guess(int(n))
        c["r_in"] = 0.1 * c["r_out"]
        out.append(c)
    return out


def wide_sparse_groups(r_out: float, k_sites: int, n_decoys: int, seed: int) -> np.ndarray:
    """Positions (n, 3) of two sparse groups, each spanning a 32-unit cube
    of a 64-unit box (~2e4 r_out at r_out = 0.0016).

    The box is fixed by particles at (0, 0, 0) and (64, 64, 64); a third at
    (32.5, 0.5, 0.5) is the first particle (lowest key) of the cube
    [32, 64) x [0, 32)^2.  k_sites sites along the face x = 32 each hold a
    particle b just below the face and a partner j = b + rho v just above it,
    v within ~17 degrees of +x, rho = r_out (1 - 1e-4) for three sites in
    four and r_out (1 + 1e-4) for the fourth.  Each of b and j gets n_decoys
    companions 0.01-0.01 n_decoys further from the face (well outside r_out
    of every other particle), so with n_leaf = n_decoys + 1 every leaf near
    the face holds exactly one of b, j and its decoys, and a walk group's PP
    entries that could be neighbours are never next to one another in its
    list.  With n_group >= 1 + k_sites (n_decoys + 1) each cube is one group
    whose members sit up to ~45 units from its first particle."""
    rng = rng_for(seed)
    pts = [(0.0, 0.0, 0.0), (64.0, 64.0, 64.0), (32.5, 0.5, 0.5)]
    for k in range(k_sites):
        y = 8.0 + 22.0 * (k + rng.uniform(0.2, 0.8)) / k_sites
        z = rng.uniform(8.0, 30.0)
        b = np.array([32.0 - rng.uniform(0.1, 0.8) * r_out, y, z])
        v = np.array([1.0, rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3)])
        v /= np.linalg.norm(v)
        j = b + r_out * (1.0 + 1e-4 if k % 4 == 3 else 1.0 - 1e-4) * v
        pts += [tuple(b), tuple(j)]
        for side, base in ((-1.0, b), (1.0, j)):
            for q in range(n_decoys):
                d = base + side * np.array([0.01 + 0.01 * q, rng.uniform(-0.01, 0.01),
                                            rng.uniform(-0.01, 0.01)])
                pts.append(tuple(d))
    return np.array(pts, dtype=np.float64)
