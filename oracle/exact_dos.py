"""Exact densities of states g(E) of the 2D Ising and q-state Potts models on an
L x L periodic lattice (J = 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  These are the pins the
REWL oracle is checked against; none of them uses Wang-Landau sampling.

- ``ising_bruteforce`` / ``potts_bruteforce``: enumerate every configuration.
- ``ising_transfer`` / ``potts_transfer``: row-to-row transfer matrix with the
  energy kept as a polynomial degree, in float64 (exact while the counts stay
  below 2^53, i.e. q^N <= 2^53).
- ``ising_kaufman``: Kaufman's closed form of the finite periodic lattice's
  partition function (Phys. Rev. 76, 1232 (1949)), as used by Beale
  (Phys. Rev. Lett. 76, 78 (1996)) to obtain exact g(E):
      Z = 1/2 (2 sinh 2K)^{N/2} (Z1 + Z2 + Z3 + Z4),
      Z1 = prod_{k odd} 2 cosh(L g_k/2),  Z2 = prod_{k odd} 2 sinh(L g_k/2),
      Z3 = prod_{k even} 2 cosh(L g_k/2), Z4 = prod_{k even} 2 sinh(L g_k/2),
      cosh g_k = cosh 2K coth 2K - cos(pi k/L), k in [0, 2L), e^{g_0} = e^{2K} tanh K.
  Each factor is rewritten so that no square root or logarithm appears
  (cosh(n g) = T_n(cosh g), sinh(n g) = sinh g U_{n-1}(cosh g); the factors of
  k and 2L-k are equal, so their product holds sinh^2 g = cosh^2 g - 1; and
  sinh g_L = cosh 2K (1 + sinh 2K)/sinh 2K).  Z e^{-2NK} is then a polynomial
  sum_j g_j z^j in z = e^{-4K} (E = -2N + 4j); it is evaluated in multiprecision
  on a circle |z| = rho and its integer coefficients are read off with a DFT.
- ``ising_kaufman_modular``: the same closed form written as a rational function
  of u = e^{-2K} (z = u^2) and evaluated exactly in prime fields GF(p),
  p = 1 mod 2M: cos(pi k / L) = (w^k + w^-k)/2 with w a primitive 2L-th root of
  unity in GF(p), evaluation points z_i = b^2 c^i on the M-th roots of unity c
  (M a power of two > N, b a random scale away from the poles u^2 = 1), the
  coefficients mod p by an inverse number-theoretic transform, and the integers
  g_j by the Chinese remainder theorem over enough primes to exceed 2^N.  No
  floating point anywhere, so it reaches L = 128 in minutes.

Energies are returned as dicts {E: g} of Python integers.
"""
import itertools
import math

import numpy as np


# ---------------------------------------------------------------------------
# brute force
# ---------------------------------------------------------------------------
def ising_bruteforce(L):
    """g(E) for the L x L periodic Ising model by enumerating all 2^N states."""
    N = L * L
    if N > 24:
        raise ValueError("brute force limited to N <= 24")
    idx = np.arange(1 << N, dtype=np.int64)
    s = 1 - 2 * ((idx[:, None] >> np.arange(N)) & 1)          # (2^N, N) spins +-1
    s = s.reshape(-1, L, L)
    E = -(s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)) - (s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    vals, counts = np.unique(E, return_counts=True)
    return {int(e): int(c) for e, c in zip(vals, counts)}


def potts_bruteforce(q, L):
    """g(E) for the L x L periodic q-state Potts model, E = -sum delta(s_i, s_j),
    enumerating all q^N states (first row outermost, the rest vectorised)."""
    N = L * L
    if q ** N > 2 ** 33:
        raise ValueError("brute force limited to q^N <= 2^33")
    rest = np.array(list(itertools.product(range(q), repeat=N - L)), dtype=np.int8)
    counts = {}
    for first in itertools.product(range(q), repeat=L):
        s = np.concatenate([np.broadcast_to(np.array(first, np.int8), (rest.shape[0], L)), rest], axis=1)
        s = s.reshape(-1, L, L)
        E = -(s == np.roll(s, -1, axis=2)).sum(axis=(1, 2)) - (s == np.roll(s, -1, axis=1)).sum(axis=(1, 2))
        vals, c = np.unique(E, return_counts=True)
        for e, n in zip(vals, c):
            counts[int(e)] = counts.get(int(e), 0) + int(n)
    return counts


# ---------------------------------------------------------------------------
# transfer matrix (float64)
# ---------------------------------------------------------------------------
def _transfer(states, bond_equal_count, L):
    """Shared row-transfer driver.  states: (S, L) int array of row values.
    Energy is counted as the number of *unsatisfied* bonds u (horizontal bonds
    inside each row + vertical bonds to the row below); rows are periodic and
    the last row bonds to the first.  Returns counts[u] for u in 0..2N."""
    S = states.shape[0]
    N = L * L
    # unsatisfied horizontal bonds inside a row
    h = L - bond_equal_count(states, np.roll(states, -1, axis=1))
    # unsatisfied vertical bonds between rows r and r'
    v = L - bond_equal_count(states[:, None, :], states[None, :, :])
    umax = 2 * N
    # vec[f, r, u]: first row f, current row r, u unsatisfied bonds so far
    vec = np.zeros((S, S, umax + 1))
    for f in range(S):
        vec[f, f, h[f]] = 1.0
    for _ in range(L - 1):
        new = np.zeros_like(vec)
        for dv in range(L + 1):
            M = (v == dv).astype(np.float64)                  # (r, r')
            if not M.any():
                continue
            t = np.einsum("fru,rs->fsu", vec, M)
            for r2 in range(S):
                shift = dv + h[r2]
                new[:, r2, shift:] += t[:, r2, :umax + 1 - shift]
        vec = new
    out = np.zeros(umax + 1)
    for f in range(S):
        for r in range(S):
            out[v[r, f]:] += vec[f, r, :umax + 1 - v[r, f]]
    return out


def ising_transfer(L):
    """g(E) (float64 counts) of the L x L periodic Ising model; exact for L <= 7."""
    states = 1 - 2 * ((np.arange(1 << L)[:, None] >> np.arange(L)) & 1)
    counts = _transfer(states, lambda a, b: (a == b).sum(axis=-1), L)
    N = L * L
    return {-2 * N + 2 * u: c for u, c in enumerate(counts) if c != 0}


def potts_transfer(q, L):
    """g(E) (float64 counts) of the L x L periodic q-state Potts model."""
    states = np.array(list(itertools.product(range(q), repeat=L)))
    counts = _transfer(states, lambda a, b: (a == b).sum(axis=-1), L)
    N = L * L
    return {-2 * N + u: c for u, c in enumerate(counts) if c != 0}


# ---------------------------------------------------------------------------
# Kaufman / Beale, multiprecision
# ---------------------------------------------------------------------------
def _cheb(n, c, one):
    """(T_n(c), U_{n-1}(c)) by the three-term recurrences."""
    t_prev, t = one, c               # T_0, T_1
    u_prev, u = 0 * one, one         # U_{-1}, U_0
    for _ in range(1, n):
        t_prev, t = t, 2 * c * t - t_prev
        u_prev, u = u, 2 * c * u - u_prev
    if n == 0:
        return one, 0 * one
    return t, u


def kaufman_polynomial_value(L, K, mp):
    """Z(K) e^{-2NK} = sum_j g_j z^j at z = e^{-4K} for complex K (mpmath)."""
    N = L * L
    n = L // 2
    one = mp.mpf(1)
    s2 = mp.sinh(2 * K)
    ch2 = mp.cosh(2 * K)
    C = ch2 * ch2 / s2
    x0 = mp.exp(2 * K) * mp.tanh(K)
    cosk = [mp.cos(mp.pi * k / L) for k in range(2 * L)]
    z1 = z2 = z3 = z4 = one
    for k in range(1, L, 2):                       # odd pairs (k, 2L - k)
        c = C - cosk[k]
        t, u = _cheb(n, c, one)
        z1 *= (2 * t) ** 2
        z2 *= 4 * (c * c - 1) * u * u
    for k in range(2, L, 2):                       # even pairs (k, 2L - k)
        c = C - cosk[k]
        t, u = _cheb(n, c, one)
        z3 *= (2 * t) ** 2
        z4 *= 4 * (c * c - 1) * u * u
    cL = C + 1                                     # k = L pairs with itself
    tL, uL = _cheb(n, cL, one)
    sinh_gL = ch2 * (1 + s2) / s2
    z3 *= 2 * tL
    z4 *= 2 * sinh_gL * uL
    p0 = x0 ** n                                   # k = 0: e^{g_0 L/2}
    z3 *= p0 + 1 / p0
    z4 *= p0 - 1 / p0
    Z = (2 * s2) ** (N // 2) * (z1 + z2 + z3 + z4) / 2
    return Z * mp.exp(-2 * N * K)


def ising_kaufman(L, K0=0.3):
    """Exact g(E) of the L x L periodic Ising model (L even, L >= 4) as a dict of
    Python integers, from Kaufman's closed form read off on |z| = e^{-4 K0}."""
    import mpmath

    if L < 4 or L % 2:
        raise ValueError("even L >= 4 required")
    N = L * L
    rho_log10 = 4 * K0 / math.log(10)               # log10(1/rho)
    dps = int(N * (rho_log10 + math.log10(2)) + 40)
    M = N + 1
    with mpmath.workdps(dps):
        mp = mpmath.mp
        rho = mp.exp(-4 * mp.mpf(K0))
        # P(z) has real coefficients: P(conj z) = conj P(z); evaluate half the circle
        vals = [None] * M
        for k in range(M // 2 + 1):
            z = rho * mp.expjpi(mp.mpf(2 * k) / M)
            K = -mp.log(z) / 4
            vals[k] = kaufman_polynomial_value(L, K, mp)
        for k in range(M // 2 + 1, M):
            vals[k] = mp.conj(vals[M - k])
        roots = [mp.expjpi(mp.mpf(-2 * t) / M) for t in range(M)]
        g = {}
        for j in range(N + 1):
            acc = mp.mpc(0)
            for k in range(M):
                acc += vals[k] * roots[(j * k) % M]
            c = (acc / M).real / rho ** j
            gj = int(mp.nint(c))
            if abs(c - gj) > 1e-6:
                raise ArithmeticError(f"coefficient {j} not integral: {c}")
            if gj:
                g[-2 * N + 4 * j] = gj
    return g


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def log_dos_on_bins(g, e_min, step, B):
    """ln g on the bin grid e_min + b * step (nan where g = 0)."""
    out = np.full(B, np.nan)
    for E, c in g.items():
        b = (E - e_min) // step
        if 0 <= b < B and (E - e_min) % step == 0 and c > 0:
            out[b] = math.log(c) if isinstance(c, int) else float(np.log(c))
    return out


def log_sum(lg):
    """ln sum_b exp(lg[b]) over finite entries."""
    v = lg[np.isfinite(lg)]
    mx = v.max()
    return float(mx + np.log(np.exp(v - mx).sum()))


# ---------------------------------------------------------------------------
# Kaufman / Beale, exact in prime fields
# ---------------------------------------------------------------------------
def _is_prime(n):
    if n < 2:
        return False
    for d in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % d == 0:
            return n == d
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in (2, 3, 5, 7, 11, 13, 17):          # deterministic below 3.4e14
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def _primes_1_mod(m, count, below=1 << 31):
    """The `count` largest primes p < below with p = 1 (mod m)."""
    out = []
    k = (below - 2) // m
    while len(out) < count and k > 0:
        p = k * m + 1
        if _is_prime(p):
            out.append(p)
        k -= 1
    if len(out) < count:
        raise ArithmeticError("not enough primes")
    return out


def _prime_factors(n):
    out, d = set(), 2
    while d * d <= n:
        while n % d == 0:
            out.add(d)
            n //= d
        d += 1
    if n > 1:
        out.add(n)
    return out


def _root_of_unity(p, order):
    """A primitive `order`-th root of unity mod p (order dividing p - 1)."""
    qs = _prime_factors(order)
    for a in range(2, 1000):
        x = pow(a, (p - 1) // order, p)
        if all(pow(x, order // q, p) != 1 for q in qs):
            return x
    raise ArithmeticError("no root found")


def _vinv(x, p):
    """Elementwise inverse mod p of an int64 array (Fermat), all entries nonzero."""
    r = np.ones_like(x)
    b = x % p
    e = p - 2
    while e:
        if e & 1:
            r = r * b % p
        b = b * b % p
        e >>= 1
    return r


def _ntt(a, root, p):
    """In-place iterative radix-2 transform of int64 array a (len a power of 2)
    with the primitive len(a)-th root `root`: A_i = sum_j a_j root^(ij)."""
    n = a.size
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    a = a[rev].copy()
    size = 2
    while size <= n:
        half = size // 2
        w = pow(root, n // size, p)
        tw = np.ones(half, dtype=np.int64)
        for j in range(1, half):
            tw[j] = tw[j - 1] * w % p
        a = a.reshape(-1, size)
        lo = a[:, :half].copy()
        hi = a[:, half:] * tw % p
        a[:, :half] = (lo + hi) % p
        a[:, half:] = (lo - hi) % p
        a = a.reshape(-1)
        size *= 2
    return a


def _cheb_vec(n, c, p):
    """(T_n(c), U_{n-1}(c)) mod p elementwise (n >= 1), by doubling
    (T_2k = 2T_k^2 - 1, U_2k-1 = 2 T_k U_k-1) and increments
    (T_k+1 = c T_k - (1 - c^2) U_k-1, U_k = c U_k-1 + T_k)."""
    t = c % p
    u = np.ones_like(c)
    one_m_c2 = (1 - c * c % p) % p
    for bit in bin(n)[3:]:
        t, u = (2 * (t * t % p) - 1) % p, 2 * (t * u % p) % p
        if bit == "1":
            t, u = (c * t % p - one_m_c2 * u % p) % p, (c * u % p + t) % p
    return t, u


def _kaufman_values_mod(L, p, M):
    """P(z_i) mod p, z_i = b^2 c^i (i < M), P(z) = Z e^{-2NK} = sum_j g_j z^j,
    for the first scale b that keeps every u_i^2 away from 1; returns (values, b^2)."""
    N = L * L
    n = L // 2
    eta = _root_of_unity(p, 2 * M)              # u_i = b eta^i, z_i = b^2 eta^(2i)
    w = _root_of_unity(p, 2 * L)                # cos(pi k/L) = (w^k + w^-k)/2
    inv2 = (p + 1) // 2
    for b in range(3, 200):
        if pow(b * b % p, M, p) != 1:            # b^2 c^i != 1 for every i
            break
    etas = np.ones(M, dtype=np.int64)
    step = eta
    # eta^i by repeated squaring blocks (vectorised): eta^i = eta^(i mod B) * (eta^B)^(i div B)
    B = 1 << ((M.bit_length() - 1) // 2)
    small = np.ones(B, dtype=np.int64)
    for i in range(1, B):
        small[i] = small[i - 1] * step % p
    bigstep = pow(eta, B, p)
    big = np.ones(M // B, dtype=np.int64)
    for i in range(1, M // B):
        big[i] = big[i - 1] * bigstep % p
    etas = (big[:, None] * small[None, :] % p).reshape(-1)
    u = etas * b % p
    iu = _vinv(u, p)
    s2 = (iu - u) % p * inv2 % p                 # sinh 2K
    ch2 = (iu + u) % p * inv2 % p                # cosh 2K
    is2 = _vinv(s2, p)
    C = ch2 * ch2 % p * is2 % p                  # cosh 2K coth 2K
    x0 = iu * ((1 - u) % p) % p * _vinv((1 + u) % p, p) % p   # e^{2K} tanh K
    cosk = [(pow(w, k, p) + pow(w, 2 * L - k, p)) % p * inv2 % p for k in range(2 * L)]
    z1 = np.ones(M, dtype=np.int64)
    z2 = np.ones(M, dtype=np.int64)
    z3 = np.ones(M, dtype=np.int64)
    z4 = np.ones(M, dtype=np.int64)
    for k in range(1, L):                        # pairs (k, 2L - k)
        c = (C - cosk[k]) % p
        t, uu = _cheb_vec(n, c, p)
        a = 2 * t % p
        bb = 4 * ((c * c - 1) % p) % p * (uu * uu % p) % p
        if k % 2:
            z1 = z1 * (a * a % p) % p
            z2 = z2 * bb % p
        else:
            z3 = z3 * (a * a % p) % p
            z4 = z4 * bb % p
    cL = (C + 1) % p                             # k = L pairs with itself
    tL, uL = _cheb_vec(n, cL, p)
    sinh_gL = ch2 * ((1 + s2) % p) % p * is2 % p
    z3 = z3 * (2 * tL % p) % p
    z4 = z4 * (2 * sinh_gL % p) % p * uL % p
    p0 = np.ones(M, dtype=np.int64)              # k = 0: e^{g_0 L/2} = x0^n
    for _ in range(n):
        p0 = p0 * x0 % p
    ip0 = _vinv(p0, p)
    z3 = z3 * ((p0 + ip0) % p) % p
    z4 = z4 * ((p0 - ip0) % p) % p
    pre = np.ones(M, dtype=np.int64)             # (2 sinh 2K)^{N/2} e^{-2NK} = (2 s2)^{N/2} u^N
    base = 2 * s2 % p * (u * u % p) % p
    e = N // 2
    bpow = base.copy()
    while e:
        if e & 1:
            pre = pre * bpow % p
        bpow = bpow * bpow % p
        e >>= 1
    tot = (z1 + z2 + z3 + z4) % p * inv2 % p
    return pre * tot % p, b * b % p


def ising_kaufman_modular(L):
    """Exact g(E) of the L x L periodic Ising model (L even, L >= 4) as a dict of
    Python integers, from Kaufman's closed form evaluated in prime fields."""
    if L < 4 or L % 2:
        raise ValueError("even L >= 4 required")
    N = L * L
    M = 1 << N.bit_length()                      # power of two > N
    n_primes = (N + 8) // 30 + 2                 # primes > 2^30 each; product > 2^(N+2)
    primes = _primes_1_mod(2 * M * (2 * L) // math.gcd(2 * M, 2 * L), n_primes)
    res = []
    for p in primes:
        vals, b2 = _kaufman_values_mod(L, p, M)
        c = _root_of_unity(p, M)
        coef = _ntt(vals, pow(c, p - 2, p), p) * pow(M, p - 2, p) % p    # h_j = g_j b^(2j)
        ib2 = pow(b2, p - 2, p)
        scale = np.ones(M, dtype=np.int64)
        s = 1
        for j in range(1, N + 1):                # b^(-2j)
            s = s * ib2 % p
            scale[j] = s
        res.append((p, coef * scale % p))
    # Chinese remainder theorem (Garner), coefficient by coefficient
    g = {}
    mod = 1
    acc = [0] * (N + 1)
    for p, r in res:
        inv = pow(mod % p, p - 2, p)
        rl = r.tolist()
        for j in range(N + 1):
            t = (rl[j] - acc[j]) % p * inv % p
            acc[j] += mod * t
        mod *= p
    half = mod // 2
    for j in range(N + 1):
        v = acc[j] if acc[j] <= half else acc[j] - mod
        if v < 0:
            raise ArithmeticError(f"negative coefficient {j}")
        if v:
            g[-2 * N + 4 * j] = v
    return g
