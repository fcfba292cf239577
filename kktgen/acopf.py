"""Seeded ACOPF-shaped KKT sequences (synthetic stand-in for the paper's grids).

The paper measures on TAMU synthetic grids (25k-80k buses, Table 1) that are
not available here; these generators reproduce the shape of its KKT systems
(Sec. 2, Eq. 4): a symmetric, quasi-definite 3x3 block matrix

    K = [[H + D_x, Je^T, Ji^T],
         [Je,     -1e-8 I,  0],
         [Ji,        0, -D_s^-1]]

whose pattern is fixed while its values change every interior-point step, with
about 10 stored entries per row (Table 1 has nnz/N ~ 11).

Recipe (every draw from NumPy PCG64, seed = 1000*cfg + scenario):
  * Grid: nb buses on a ceil(sqrt(nb))-wide snake lattice; ring lines join
    consecutive buses plus (nb-1, 0); nl - nb chords each join a uniform random
    bus to a uniform random bus within lattice offset +-3 (self loops, repeats
    and ring edges rejected).  ``chords="global"`` draws chord ends uniformly
    over all buses (an expander-like stress variant).  ng generators sit on
    uniform random buses (with replacement).
  * Variables x = (|V|_i, theta_i) per bus, then (P_g, Q_g) per generator.
  * H: dense 2x2 blocks on each bus, on both orientations of each line, and on
    each generator; off-diagonal entries N(0,1) + per-step N(0, 0.1^2),
    symmetric; the diagonal is sigma_i + sum_row |off-diagonal| (strictly
    diagonally dominant, so H + D_x is SPD).
  * Je: 2 rows per bus (P and Q balance), dense 2x2 blocks on the bus and its
    neighbours, plus (P_i, P_g) and (Q_i, Q_g) for each generator g on bus i.
  * Ji: 2 rows per line (flow at each end), dense 2x4 on (|V|, theta) of both
    ends.  Je and Ji entries are N(0,1), fixed across steps.
  * D_x = 10^(w_k u), D_s = 10^(w_k v), u, v ~ U(-1, 1) fixed per run,
    w_k = W (k + 1) / K (log-range of D = mu Y^-2 widening one step at a time),
    or w_k = W for late-IPM sequences.
  * Scenario scaling sigma_i ~ U(0.8, 1.2) per bus multiplies the Je rows of
    bus i and the H 2x2 block of bus i.
  * ``asym`` > 0 multiplies every stored off-diagonal entry by an independent
    (1 + asym N(0,1)) so tests can catch a transposed operand.
  * Right-hand side b = K x_true with x_true ~ N(0, 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

# Configurations of the workloads (buses, lines, generators, steps, W, ...).
CONFIGS = {
    0: dict(name="plain FP64, 200-bus sequence", nb=200, nl=260, ng=40, steps=10, W=6.0,
            widen=True, scenarios=1),
    1: dict(name="plain FP64 + adjoint, 2,000-bus sequence", nb=2000, nl=2600, ng=400,
            steps=30, W=8.0, widen=True, scenarios=1),
    2: dict(name="batched FP64, 10,000-bus x 64 scenarios", nb=10000, nl=13000, ng=2000,
            steps=5, W=8.0, widen=True, scenarios=64),
    3: dict(name="FP32 factors + FP64 refinement, 70,000-bus late-IPM", nb=70000, nl=91000,
            ng=14000, steps=4, W=8.0, widen=False, scenarios=1),
}
# Uneven batch: (buses, lines, generators, count)
UNEVEN = [(500, 650, 100, 16), (2000, 2600, 400, 16), (5000, 6500, 1000, 12),
          (20000, 26000, 4000, 4)]


def _rng(*key):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(key))))


@dataclass
class Grid:
    nb: int
    lines: np.ndarray  # (nl, 2) int64 bus pairs
    gen_bus: np.ndarray  # (ng,) int64

    @property
    def nl(self):
        return int(self.lines.shape[0])

    @property
    def ng(self):
        return int(self.gen_bus.shape[0])


def make_grid(nb: int, nl: int, ng: int, seed: int, chords: str = "local") -> Grid:
    """Ring-plus-chords grid on a snake lattice (see module docstring)."""
    if nb < 3 or nl < nb:
        raise ValueError("need nb >= 3 and nl >= nb")
    rng = _rng(seed, 0)
    w = int(math.ceil(math.sqrt(nb)))
    b = np.arange(nb)
    r = b // w
    c = np.where(r % 2 == 0, b % w, w - 1 - b % w)
    at = -np.ones((r.max() + 1, w), dtype=np.int64)
    at[r, c] = b
    ring = np.stack([b, np.roll(b, -1)], axis=1)
    key = lambda u, v: np.minimum(u, v) * nb + np.maximum(u, v)
    used = set(key(ring[:, 0], ring[:, 1]).tolist())
    need = nl - nb
    out = []
    tries = 0
    while need > 0:
        tries += 1
        if tries > 10000:
            raise RuntimeError("could not place chords")
        m = max(64, 2 * need)
        a = rng.integers(0, nb, size=m)
        if chords == "local":
            dr = rng.integers(-3, 4, size=m)
            dc = rng.integers(-3, 4, size=m)
            rr, cc = r[a] + dr, c[a] + dc
            ok = (rr >= 0) & (rr < at.shape[0]) & (cc >= 0) & (cc < w)
            t = np.full(m, -1, dtype=np.int64)
            t[ok] = at[rr[ok], cc[ok]]
        elif chords == "global":
            t = rng.integers(0, nb, size=m)
        else:
            raise ValueError(chords)
        for u, v in zip(a.tolist(), t.tolist()):
            if v < 0 or u == v:
                continue
            k = min(u, v) * nb + max(u, v)
            if k in used:
                continue
            used.add(k)
            out.append((u, v))
            need -= 1
            if need == 0:
                break
    lines = np.concatenate([ring, np.array(out, dtype=np.int64).reshape(-1, 2)], axis=0)
    gen_bus = rng.integers(0, nb, size=ng).astype(np.int64)
    return Grid(nb=nb, lines=lines, gen_bus=gen_bus)


@dataclass
class KKTSequence:
    """A fixed KKT pattern with per-step, per-scenario values.

    ``indptr``/``indices`` are the CSR pattern (int32, sorted, unique).  The
    values of step k for scenario s are ``values(k, s)`` (float64, CSR order).
    """
    grid: Grid
    seed: int
    steps: int
    W: float
    widen: bool
    asym: float = 0.0
    reg: float = 1e-8      # regularization of the equality block (-reg I); 0: a zero
                           # diagonal block, the KKT matrix is then not quasi-definite
    n_x: int = 0
    n: int = 0
    indptr: np.ndarray = field(default=None, repr=False)
    indices: np.ndarray = field(default=None, repr=False)

    def __post_init__(self):
        g = self.grid
        nb, nl, ng = g.nb, g.nl, g.ng
        self.n_x = 2 * nb + 2 * ng
        self.n_eq = 2 * nb
        self.n_in = 2 * nl
        self.n = self.n_x + self.n_eq + self.n_in
        V = 2 * np.arange(nb)          # |V| of bus
        T = V + 1                      # theta of bus
        P = 2 * nb + 2 * np.arange(ng)
        Q = P + 1
        a, bb = g.lines[:, 0], g.lines[:, 1]

        # --- H off-diagonal pairs (p < q not required; stored as (p,q),(q,p))
        hp, hq, hkind, hbus = [], [], [], []
        hp.append(V); hq.append(T); hkind.append(np.zeros(nb, np.int8)); hbus.append(np.arange(nb))
        hp.append(P); hq.append(Q); hkind.append(np.ones(ng, np.int8)); hbus.append(-np.ones(ng, np.int64))
        for ea in (V, T):
            for eb in (V, T):
                hp.append(ea[a]); hq.append(eb[bb]); hkind.append(np.ones(nl, np.int8))
                hbus.append(-np.ones(nl, np.int64))
        self._hp = np.concatenate(hp); self._hq = np.concatenate(hq)
        self._hbus = np.concatenate(hbus)  # bus whose block the pair belongs to, or -1
        # --- Je entries: (row, col) with row in the equality block
        adj_u = np.concatenate([np.arange(nb), a, bb])
        adj_v = np.concatenate([np.arange(nb), bb, a])
        jr, jc, jbus = [], [], []
        for rowoff in (0, 1):
            for var in (V, T):
                jr.append(self.n_x + 2 * adj_u + rowoff); jc.append(var[adj_v]); jbus.append(adj_u)
        jr.append(self.n_x + 2 * g.gen_bus); jc.append(P); jbus.append(g.gen_bus)
        jr.append(self.n_x + 2 * g.gen_bus + 1); jc.append(Q); jbus.append(g.gen_bus)
        self._jr = np.concatenate(jr); self._jc = np.concatenate(jc); self._jbus = np.concatenate(jbus)
        # --- Ji entries
        ir, ic = [], []
        lrow = self.n_x + self.n_eq + 2 * np.arange(nl)
        for rowoff in (0, 1):
            for var in (V[a], T[a], V[bb], T[bb]):
                ir.append(lrow + rowoff); ic.append(var)
        self._ir = np.concatenate(ir); self._ic = np.concatenate(ic)

        diag = np.arange(self.n)
        rows = np.concatenate([self._hp, self._hq, self._jr, self._jc, self._ir, self._ic, diag])
        cols = np.concatenate([self._hq, self._hp, self._jc, self._jr, self._ic, self._ir, diag])
        self._n_off = rows.size - self.n
        key = rows.astype(np.int64) * self.n + cols
        order = np.argsort(key, kind="stable")
        skey = key[order]
        if np.any(skey[1:] == skey[:-1]):
            raise RuntimeError("duplicate KKT entries in generator")
        self._order = order
        srow = rows[order]
        self.indices = cols[order].astype(np.int32)
        self.indptr = np.zeros(self.n + 1, dtype=np.int32)
        np.add.at(self.indptr, srow + 1, 1)
        self.indptr = np.cumsum(self.indptr).astype(np.int32)
        # fixed per-run draws
        rng = _rng(self.seed, 1)
        self._h0 = rng.standard_normal(self._hp.size)
        self._je = rng.standard_normal(self._jr.size)
        self._ji = rng.standard_normal(self._ir.size)
        self._u = rng.uniform(-1.0, 1.0, self.n_x)
        self._v = rng.uniform(-1.0, 1.0, self.n_in)
        self._asym = _rng(self.seed, 2).standard_normal(self._n_off) if self.asym else None

    @property
    def nnz(self):
        return int(self.indices.size)

    def w(self, k):
        return self.W * (k + 1) / self.steps if self.widen else self.W

    def sigma(self, scenario):
        if scenario == 0:
            return np.ones(self.grid.nb)
        return _rng(self.seed + scenario, 3).uniform(0.8, 1.2, self.grid.nb)

    def values(self, k: int, scenario: int = 0) -> np.ndarray:
        """CSR-ordered float64 values of step k, scenario s."""
        sig = self.sigma(scenario)
        h = self._h0 + 0.1 * _rng(self.seed, 100 + k).standard_normal(self._h0.size)
        hs = np.where(self._hbus >= 0, sig[np.maximum(self._hbus, 0)], 1.0)
        h = h * hs
        je = self._je * sig[self._jbus]
        ji = self._ji
        rowabs = np.zeros(self.n_x)
        np.add.at(rowabs, self._hp, np.abs(h))
        np.add.at(rowabs, self._hq, np.abs(h))
        dsig = np.ones(self.n_x)
        dsig[: 2 * self.grid.nb] = np.repeat(sig, 2)
        wk = self.w(k)
        dx = 10.0 ** (wk * self._u)
        ds = 10.0 ** (wk * self._v)
        dvals = np.concatenate([dsig + rowabs + dx, np.full(self.n_eq, -self.reg), -1.0 / ds])
        off = np.concatenate([h, h, je, je, ji, ji])
        if self._asym is not None:
            off = off * (1.0 + self.asym * self._asym)
        data = np.concatenate([off, dvals])
        return np.ascontiguousarray(data[self._order])

    def csr(self, k: int, scenario: int = 0) -> sp.csr_matrix:
        return sp.csr_matrix((self.values(k, scenario), self.indices, self.indptr),
                             shape=(self.n, self.n))

    def x_true(self, k: int, scenario: int = 0) -> np.ndarray:
        return _rng(self.seed + scenario, 200 + k).standard_normal(self.n)

    def rhs(self, k: int, scenario: int = 0) -> np.ndarray:
        """b = K x_true (SciPy sparse product)."""
        return self.csr(k, scenario) @ self.x_true(k, scenario)


def kkt_sequence(nb, nl, ng, seed, steps=10, W=6.0, widen=True, chords="local",
                 asym=0.0, reg=1e-8) -> KKTSequence:
    grid = make_grid(nb, nl, ng, seed, chords=chords)
    return KKTSequence(grid=grid, seed=seed, steps=steps, W=W, widen=widen, asym=asym, reg=reg)


def config_sequence(cfg: int, asym: float = 0.0, chords: str = "local") -> KKTSequence:
    c = CONFIGS[cfg]
    return kkt_sequence(c["nb"], c["nl"], c["ng"], seed=1000 * cfg, steps=c["steps"], W=c["W"],
                        widen=c["widen"], chords=chords, asym=asym)


def uneven_sequences(asym: float = 0.0):
    """The 48 uneven systems: each a different grid (seed 4000 + j)."""
    out = []
    j = 0
    for nb, nl, ng, cnt in UNEVEN:
        for _ in range(cnt):
            out.append(kkt_sequence(nb, nl, ng, seed=4000 + j, steps=1, W=8.0, widen=False,
                                    asym=asym))
            j += 1
    return out


def random_sparse_pattern(n: int, density: float, seed: int, drop_diag: float = 0.0):
    """Random (non-symmetric) CSR pattern, sorted and unique; the diagonal is
    present except for a ``drop_diag`` fraction of rows."""
    rng = _rng(seed, 7)
    m = rng.random((n, n)) < density
    np.fill_diagonal(m, rng.random(n) >= drop_diag)
    rows, cols = np.nonzero(m)
    indptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(indptr, rows + 1, 1)
    return np.cumsum(indptr).astype(np.int32), cols.astype(np.int32)


def random_dd_values(indptr, indices, seed: int, dominance: float = 1.0):
    """Random values on a pattern, diagonal set so that rows and columns are
    diagonally dominant (factorization without pivoting stays stable)."""
    rng = _rng(seed, 8)
    n = indptr.size - 1
    vals = rng.standard_normal(indices.size)
    rows = np.repeat(np.arange(n), np.diff(indptr))
    off = rows != indices
    ra = np.zeros(n)
    ca = np.zeros(n)
    np.add.at(ra, rows[off], np.abs(vals[off]))
    np.add.at(ca, indices[off], np.abs(vals[off]))
    d = ~off
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    vals[d] = sign[rows[d]] * (dominance + np.maximum(ra, ca)[rows[d]])
    return vals
