"""Integer lattice algebra of the nonseparable DGT (oracle side; test infrastructure only).

Everything here is exact integer arithmetic on Python ints.

Notation (Section 2.1): L signal length, a time step, M channels, b = L/M,
N = L/a, lattice normal form [[a, 0], [s, b]] with s = b*lam1/lam2,
gcd(lam1, lam2) = 1, 0 <= lam1 < lam2.
"""
from __future__ import annotations

from dataclasses import dataclass
from math import gcd


def lcm(x: int, y: int) -> int:
    return x * y // gcd(x, y)


def ext_gcd(x: int, y: int) -> tuple[int, int, int]:
    """Return (g, u, v) with u*x + v*y = g = gcd(x, y) >= 0."""
    old_r, r = x, y
    old_u, u = 1, 0
    old_v, v = 0, 1
    while r != 0:
        qq = old_r // r
        old_r, r = r, old_r - qq * r
        old_u, u = u, old_u - qq * u
        old_v, v = v, old_v - qq * v
    if old_r < 0:
        old_r, old_u, old_v = -old_r, -old_u, -old_v
    return old_r, old_u, old_v


def min_length(a: int, M: int, lam2: int) -> int:
    """Minimal feasible signal length L_min = lam2 * lcm(a, M) (Prop. minsig)."""
    return lam2 * lcm(a, M)


def feasible(L: int, a: int, M: int, lam1: int, lam2: int) -> bool:
    """The lattice parameters define a lattice on Z_L iff L is a multiple of L_min (Prop. minsig)."""
    if a <= 0 or M <= 0 or lam2 <= 0 or not (0 <= lam1 < lam2) or gcd(lam1, lam2) != 1:
        return False
    return L % min_length(a, M, lam2) == 0


@dataclass(frozen=True)
class Lattice:
    L: int
    a: int
    M: int
    lam1: int
    lam2: int

    def __post_init__(self):
        if not feasible(self.L, self.a, self.M, self.lam1, self.lam2):
            raise ValueError("infeasible lattice (L must be a multiple of lam2*lcm(a,M))")

    @property
    def b(self) -> int:
        return self.L // self.M

    @property
    def N(self) -> int:
        return self.L // self.a

    @property
    def s(self) -> int:
        """Shear parameter of the normal form, s = b*lam1/lam2 (Section 2.1)."""
        return self.b * self.lam1 // self.lam2

    def freq_offset_num(self, n: int) -> int:
        """Numerator of w(n) = ((n*lam1) mod lam2) / lam2 (eq. DGT)."""
        return (n * self.lam1) % self.lam2

    def points(self) -> set[tuple[int, int]]:
        """The lattice A Z_L^2 as a set of (x, omega) pairs, generated from the
        normal-form matrix [[a,0],[s,b]] (Prop. lattNF).  Small L only."""
        pts = set()
        for n in range(self.N):
            for k in range(self.M):
                pts.add(((self.a * n) % self.L, (self.s * n + self.b * k) % self.L))
        return pts


def sep_constants(L: int, a: int, M: int) -> dict:
    """c = gcd(a, M), d = gcd(b, N), p = a/c = b/d, q = M/c = N/d (eqs. cd, pq)."""
    b, N = L // M, L // a
    c = gcd(a, M)
    d = gcd(b, N)
    p, q = a // c, M // c
    assert p == b // d and q == N // d and L == c * d * p * q
    return dict(c=c, d=d, p=p, q=q, b=b, N=N)


def coset_params(lat: Lattice) -> list[tuple[int, int]]:
    """Coset decomposition (Prop. mwindec): Lambda is the union over j < lam2 of
    (j*a, j*s mod b) + tilde-Lambda, tilde-Lambda separable with time step lam2*a
    and frequency step b.  Returns [(time shift j*a, frequency shift sigma_j)]."""
    return [(j * lat.a, (j * lat.s) % lat.b) for j in range(lat.lam2)]


@dataclass(frozen=True)
class Shear:
    s0: int          # frequency-side shear
    s1: int          # time-side shear
    b_r: int         # frequency step of the separable lattice reached by the shear
    L: int

    @property
    def freq_shear(self) -> bool:
        return self.s0 % self.L != 0


def _solve_linear_congruence(A: int, B: int, m: int):
    """Smallest x >= 0 with A*x = B (mod m), or None."""
    g = gcd(A, m)
    if B % g:
        return None
    m2 = m // g
    if m2 == 1:
        return 0
    inv = pow((A // g) % m2, -1, m2)
    return ((B // g) * inv) % m2


def shearfind(L: int, a: int, M: int, lam1: int, lam2: int) -> Shear:
    """Shear parameters (s0, s1, b_r) with U_{s0,s1}^{-1} A separable.

    Theorem shearform reduces A = [[a,0],[s,b]] with U^{-1} = [[s0 s1 + 1, s0],
    [s1, 1]].  Following the proof: with X = gcd(s1*a + s, b) and Bezout
    k1*(s1*a + s) + k2*b = X, the sheared lattice is separable iff eq. (modcond)
    s0*X + a*k1 = 0 (mod a*b/X) holds; it is then generated by diag(a*b/X, X).

    Choice (performance only; every valid pair gives the same coefficients):
    first try s0 = 0, which is possible iff a | s + k*b for some k < M (proof of
    Prop. noshearlength), giving s1 = -(s + k*b)/a and b_r = b; otherwise take the
    smallest s1 >= 0 for which eq. (modcond) is solvable in s0.
    """
    lat = Lattice(L, a, M, lam1, lam2)
    b, s = lat.b, lat.s
    if s == 0:
        return Shear(0, 0, b, L)
    for k in range(M):
        if (s + k * b) % a == 0:
            return Shear(0, (-(s + k * b) // a) % L, b, L)
    for s1 in range(L):
        v = s1 * a + s
        X, k1, _ = ext_gcd(v, b)
        mod = a * b // X
        s0 = _solve_linear_congruence(X, (-a * k1) % mod, mod)
        if s0 is not None:
            return Shear(s0 % L, s1, X, L)
    raise AssertionError("no shear found (contradicts Theorem shearform)")


def sheared_is_separable(L: int, a: int, M: int, lam1: int, lam2: int, sh: Shear) -> bool:
    """Integer check, independent of the search: the image of the lattice under
    U^{-1} = [[s0 s1 + 1, s0], [s1, 1]] equals the product lattice
    (a_r Z_L) x (b_r Z_L) with a_r = a b / b_r.  Enumerates points (small L only)."""
    lat = Lattice(L, a, M, lam1, lam2)
    s0, s1 = sh.s0, sh.s1
    img = set()
    for (x, w) in lat.points():
        img.add((((s0 * s1 + 1) * x + s0 * w) % L, (s1 * x + w) % L))
    ar = a * lat.b // sh.b_r
    if L % ar or L % sh.b_r:
        return False
    prod = {((i * ar) % L, (j * sh.b_r) % L) for i in range(L // ar) for j in range(L // sh.b_r)}
    return img == prod


def noshear_length_factor(a: int, M: int, lam1: int, lam2: int) -> int:
    """The factor c/c1 of eq. (noshearlength): lengths L = n * L_min * c / c1
    need no frequency shear; c1 collects the prime powers of c = gcd(a, M)
    whose prime does not divide lam2 (Prop. noshearlength).  Reading: the
    condition printed as gcd(lam2, p_j) = 0 means gcd(lam2, p_j) = 1."""
    c = gcd(a, M)
    c1 = 1
    x = c
    pfac = 2
    while x > 1:
        if x % pfac == 0:
            e = 1
            while x % pfac == 0:
                x //= pfac
                e *= pfac
            if gcd(lam2, pfac) == 1:
                c1 *= e
        pfac += 1
    return c // c1


def alg1_constants(L: int, a: int, M: int, sh: Shear) -> dict:
    """Constants of Algorithm 1 (both branches) as integers."""
    b, N = L // M, L // a
    if not sh.freq_shear:
        return dict(C1=(sh.s1 * a * (L + 1)) % (2 * N))
    br = sh.b_r
    ar = a * b // br
    Mr, Nr = L // br, L // ar
    assert (ar % a) == 0 and (sh.s0 * br) % a == 0
    C1 = ar // a
    C2 = -sh.s0 * br // a
    C3 = a * sh.s1 * (L + 1)
    C4 = C2 * br * (L + 1)
    C5 = 2 * C1 * br
    C6 = (sh.s0 * sh.s1 + 1) * br
    return dict(ar=ar, Mr=Mr, Nr=Nr, C1=C1, C2=C2, C3=C3, C4=C4, C5=C5, C6=C6)
