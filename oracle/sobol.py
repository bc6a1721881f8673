"""Quasi-Monte Carlo normals for the oracle: Sobol points, digital shifts,
inverse normal, Brownian bridge (test infrastructure only).

The paper's Sec. 2.7 introduces Sobol sequences and their Properties A and A';
it reports plain QMC as unsatisfactory for the discretised schemes.  The
variant built here randomises a Sobol sequence with digital shifts and feeds
it through a Brownian bridge, so that the first dimensions carry the coarse
shape of the two Brownian motions.  Definitions (written out here from the
mathematics; the CUDA library's host code implements the same definitions
separately):

* Dimension 0: v_k = 2^(32-k) (van der Corput).  Dimension j >= 1 uses the
  j-th primitive polynomial over GF(2), ordered by degree and then by the
  integer whose bits are its coefficients, starting with x + 1.
* Initial direction numbers m_1..m_s of dimension j (s = degree, m_k odd,
  m_k < 2^k) come from Philox4x32-10 with key (0x50B01, 0): candidate c
  takes m_k = 2 (w mod 2^(k-1)) + 1 from word (k-1) mod 4 of the block with
  counter ((k-1) div 4, j, c, 3).  For j < 32 the first candidate
  c = 0, 1, 2, ... for which the leading (j+1) x (j+1) matrix of first
  binary digits of v_{i,k} (i <= j, k <= j+1) is non-singular over GF(2) is
  kept: that is Property A for the first j+1 dimensions (2^(j+1) points,
  one in each half-split subcube).  With 32-bit direction numbers the
  property cannot extend past 32 dimensions; from j = 32 on, and after 64
  failed candidates, candidate 0 is kept.
* Recurrence (Bratley and Fox): for P = x^s + a_1 x^(s-1) + ... + a_(s-1) x + 1,
  m_k = 2 a_1 m_(k-1) ^ 4 a_2 m_(k-2) ^ ... ^ 2^(s-1) a_(s-1) m_(k-s+1)
        ^ 2^s m_(k-s) ^ m_(k-s);  v_k = m_k 2^(32-k), k = 1..32.
* Point n, dimension d: x_d(n) = XOR of v_{d,b+1} over the set bits b of n.
* Replicate r's digital shift of dimension d: word d mod 4 of Philox block
  (d div 4, r, 0, 2) under key = the run's seed; y = x XOR shift.
* Uniform u = ((y >> 8) + 1/2) 2^-24 (24 bits, never 0 or 1); normal
  z = Phi^-1(u).
* Brownian bridge over the step grid 0..N (unit steps, scaled by sqrt(dt)
  later): node 0 is time N with W_N = sqrt(N) z; the other nodes come from
  bisecting intervals [l, r] (r - l >= 2) in breadth-first order at
  m = l + (r - l) div 2 with W_m = W_l + (m-l)/(r-l) (W_r - W_l)
  + sqrt((m-l)(r-m)/(r-l)) z.  Node j of motion a uses dimension 2j, of
  motion b dimension 2j+1.  The step normals are Za_k = W_a(k+1) - W_a(k)
  (and Zb likewise), i.i.d. N(0, 1) for every randomised point.
"""
from __future__ import annotations

import numpy as np
from scipy.special import ndtri

import oracle

SOBOL_KEY = (0x50B01, 0)
SHIFT_TAG = 2
INIT_TAG = 3
MAX_TRIES = 64


def _gf2_mulmod(a: int, b: int, mod: int, deg: int) -> int:
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a >> deg & 1:
            a ^= mod
    return r


def _gf2_powmod(base: int, e: int, mod: int, deg: int) -> int:
    r = 1
    while e:
        if e & 1:
            r = _gf2_mulmod(r, base, mod, deg)
        base = _gf2_mulmod(base, base, mod, deg)
        e >>= 1
    return r


def _prime_factors(n: int):
    out, p = [], 2
    while p * p <= n:
        if n % p == 0:
            out.append(p)
            while n % p == 0:
                n //= p
        p += 1
    if n > 1:
        out.append(n)
    return out


def is_primitive(poly: int) -> bool:
    """poly: coefficient bits, degree = bit length - 1.  Primitive iff the
    constant term is 1 and x has multiplicative order 2^s - 1 modulo poly."""
    deg = poly.bit_length() - 1
    if deg < 1 or not poly & 1:
        return False
    if deg == 1:
        return poly == 0b11
    order = (1 << deg) - 1
    if _gf2_powmod(0b10, order, poly, deg) != 1:
        return False
    return all(_gf2_powmod(0b10, order // q, poly, deg) != 1 for q in _prime_factors(order))


def primitive_polynomials(count: int):
    """The first `count` primitive polynomials by (degree, integer value)."""
    out, deg = [], 1
    while len(out) < count:
        for poly in range(1 << deg, 1 << (deg + 1)):
            if is_primitive(poly):
                out.append(poly)
                if len(out) == count:
                    break
        deg += 1
    return out


def _directions_from(poly: int, m_init):
    s = poly.bit_length() - 1
    a = [(poly >> (s - i)) & 1 for i in range(1, s)]          # a_1 .. a_(s-1)
    m = list(m_init)
    for k in range(s, 32):                                    # 0-based: m[k] is m_(k+1)
        val = m[k - s] ^ (m[k - s] << s)
        for i in range(1, s):
            if a[i - 1]:
                val ^= m[k - i] << i
        m.append(val)
    return [m[k] << (31 - k) for k in range(32)]              # v_(k+1) = m_(k+1) 2^(32-(k+1))


def _first_digit_row(v, n_cols):
    row = 0
    for k in range(n_cols):
        row |= ((v[k] >> 31) & 1) << k
    return row


def _rank_with(basis, row, n_cols):
    """Insert row into a GF(2) echelon basis {pivot: row}; True if independent."""
    for bit in range(n_cols):
        if not row >> bit & 1:
            continue
        if bit in basis:
            row ^= basis[bit]
        else:
            basis[bit] = row
            return True
    return False


def direction_numbers(n_dims: int) -> np.ndarray:
    """(n_dims, 32) uint32 direction integers v_{d,k} (column k-1 holds v_k)."""
    V = np.zeros((n_dims, 32), dtype=np.uint32)
    V[0] = [1 << (31 - k) for k in range(32)]
    polys = primitive_polynomials(n_dims - 1) if n_dims > 1 else []
    for j in range(1, n_dims):
        poly = polys[j - 1]
        s = poly.bit_length() - 1

        def candidate(c):
            m_init = []
            for k in range(1, s + 1):
                w = oracle.philox4x32_10([(k - 1) // 4, j, c, INIT_TAG], list(SOBOL_KEY))[(k - 1) % 4]
                m_init.append(2 * (w % (1 << (k - 1))) + 1)
            return _directions_from(poly, m_init)

        chosen = candidate(0)
        if j < 32:
            n_cols = j + 1
            # rows of dims 0..j-1 restricted to the first j+1 columns
            basis = {}
            for i in range(j):
                _rank_with(basis, _first_digit_row([int(x) for x in V[i]], n_cols), n_cols)
            for c in range(MAX_TRIES):
                v = candidate(c)
                if _rank_with(dict(basis), _first_digit_row(v, n_cols), n_cols):
                    chosen = v
                    break
        V[j] = chosen
    return V


def points(V: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Sobol integers x_d(n): (len(idx), n_dims) uint32."""
    idx = np.asarray(idx, dtype=np.uint64)
    out = np.zeros((len(idx), V.shape[0]), dtype=np.uint32)
    for b in range(32):
        sel = ((idx >> np.uint64(b)) & np.uint64(1)).astype(bool)
        if sel.any():
            out[sel] ^= V[:, b]
    return out


def shifts(seed: int, replicate: int, n_dims: int) -> np.ndarray:
    key = [seed & 0xFFFFFFFF, seed >> 32]
    out = np.zeros(n_dims, dtype=np.uint32)
    for d in range(n_dims):
        out[d] = oracle.philox4x32_10([d // 4, replicate, 0, SHIFT_TAG], key)[d % 4]
    return out


def uniforms(y: np.ndarray) -> np.ndarray:
    return ((y >> np.uint32(8)).astype(np.float64) + 0.5) * 2.0**-24


class BridgePlan:
    """Breadth-first bisection of the step grid 0..N (see module docstring)."""

    def __init__(self, n_steps: int):
        self.N = n_steps
        nodes = [(n_steps, 0, n_steps)]          # (time, left, right); node 0 = time N
        queue = [(0, n_steps)]
        while queue:
            l, r = queue.pop(0)
            if r - l < 2:
                continue
            m = l + (r - l) // 2
            nodes.append((m, l, r))
            queue.append((l, m))
            queue.append((m, r))
        assert len(nodes) == n_steps
        self.nodes = nodes

    def build(self, z: np.ndarray) -> np.ndarray:
        """z: (paths, N) node normals -> W: (paths, N+1) on the unit grid."""
        W = np.zeros((z.shape[0], self.N + 1))
        W[:, self.N] = np.sqrt(self.N) * z[:, 0]
        for j in range(1, self.N):
            m, l, r = self.nodes[j]
            W[:, m] = (W[:, l] + (m - l) / (r - l) * (W[:, r] - W[:, l])
                       + np.sqrt((m - l) * (r - m) / (r - l)) * z[:, j])
        return W

    def step_normals(self, z: np.ndarray) -> np.ndarray:
        return np.diff(self.build(z), axis=1)


def qmc_normals(V, plan: BridgePlan, seed: int, replicate: int, point_idx):
    """(Za, Zb), each (paths, N), for the given points of one replicate."""
    N = plan.N
    y = points(V, point_idx) ^ shifts(seed, replicate, V.shape[0])[None, :]
    z = ndtri(uniforms(y))
    return plan.step_normals(z[:, 0:2 * N:2]), plan.step_normals(z[:, 1:2 * N:2])


def qmc_price_greeks(params, contracts, n_shifts, points_per_shift, n_steps, seed,
                     trunc=oracle.TRUNC_FULL, batch=4096):
    """Randomised-QMC estimates: mean over replicates of each replicate's
    average, and SE = stdev of the replicate averages / sqrt(n_shifts)."""
    V = direction_numbers(2 * n_steps)
    plan = BridgePlan(n_steps)
    reps = []
    for r in range(n_shifts):
        s = np.zeros((len(contracts), 6))
        for lo in range(0, points_per_shift, batch):
            idx = np.arange(lo, min(points_per_shift, lo + batch))
            za, zb = qmc_normals(V, plan, seed, r, idx)
            est = oracle.paths_from_normals(params, contracts, za, zb, trunc)[1]
            s += est.sum(axis=0)
        reps.append(s / points_per_shift)
    reps = np.array(reps)
    mean = reps.mean(axis=0)
    se = reps.std(axis=0, ddof=1) / np.sqrt(n_shifts) if n_shifts > 1 else np.zeros_like(mean)
    return mean, se, reps
