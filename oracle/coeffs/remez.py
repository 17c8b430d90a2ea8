"""Minimax (Remez exchange) fitter for the polynomial coefficients.

Design tool, not part of any runtime path.  Section 5 (the overview before
5.1) describes the coefficient tool of the method: it minimises the maximum
*relative* error, and the lowest-degree coefficients are either split into a
double-double pair or restricted to a short mantissa so that those terms can
be evaluated in DD arithmetic.  This module does the same with mpmath:

    remez(...)      one exchange fit of free coefficients (weighted max error)
    fit_rounded(...) fit, then round the coefficients one at a time (lowest
                    degree first) into their storage format and refit the rest.

The coefficients it prints are design constants: they are written out as
hex-float literals in the oracle's C sources and, separately, in the CUDA
sources, in the same way the paper prints the tan coefficients in its
Appendix A listing.  Neither the oracle nor the CUDA build runs this file.
"""
import mpmath as mp


def _round_to_bits(x, bits):
    with mp.workprec(bits):
        return +x


def to_double(x):
    return float(_round_to_bits(mp.mpf(x), 53))


def to_float(x):
    import struct
    v = float(_round_to_bits(mp.mpf(x), 24))
    return struct.unpack("f", struct.pack("f", v))[0]


def split_dd(x):
    hi = to_double(x)
    lo = to_double(mp.mpf(x) - hi)
    return hi, lo


def split_ff(x):
    hi = to_float(x)
    lo = to_float(mp.mpf(x) - hi)
    return hi, lo


def _cheb_grid(a, b, n):
    a = mp.mpf(a)
    b = mp.mpf(b)
    return [(a + b) / 2 - (b - a) / 2 * mp.cos(mp.pi * k / (n - 1)) for k in range(n)]


def _poly(cs, exps, t):
    s = mp.mpf(0)
    for c, e in zip(cs, exps):
        s += c * t ** e
    return s


def _alternating_extrema(err, n_need):
    n = len(err)
    idx = []
    for k in range(n):
        left = abs(err[k - 1]) if k > 0 else -1
        right = abs(err[k + 1]) if k < n - 1 else -1
        if abs(err[k]) >= left and abs(err[k]) >= right and err[k] != 0:
            idx.append(k)
    # merge same-sign neighbours, keep the larger
    merged = []
    for k in idx:
        if merged and (err[merged[-1]] > 0) == (err[k] > 0):
            if abs(err[k]) > abs(err[merged[-1]]):
                merged[-1] = k
        else:
            merged.append(k)
    while len(merged) > n_need:
        if abs(err[merged[0]]) < abs(err[merged[-1]]):
            merged.pop(0)
        else:
            merged.pop()
    return merged


def _single_exchange(ref, err):
    """Classic one-point exchange: bring the global maximum of |err| into the
    reference while keeping the signs alternating."""
    k = max(range(len(err)), key=lambda i: abs(err[i]))
    if k in ref:
        return ref
    ref = list(ref)
    sg = lambda i: err[i] > 0
    if k < ref[0]:
        if sg(k) == sg(ref[0]):
            ref[0] = k
        else:
            ref = [k] + ref[:-1]
    elif k > ref[-1]:
        if sg(k) == sg(ref[-1]):
            ref[-1] = k
        else:
            ref = ref[1:] + [k]
    else:
        for i in range(len(ref) - 1):
            if ref[i] < k < ref[i + 1]:
                if sg(k) == sg(ref[i]):
                    ref[i] = k
                else:
                    ref[i + 1] = k
                break
    return ref


def remez(f, w, exps, a, b, fixed=(), n_grid=3000, max_iter=60, tol=1e-6,
          dps=50, verbose=False):
    """Fit c_j in P(t) = sum_j c_j t^exps[j] minimising
    max_{t in [a,b]} |w(t) * (P(t) + F(t) - f(t))|, F = sum of fixed terms
    given as (exponent, value) pairs.  Returns (coeffs, max_error)."""
    with mp.workdps(dps):
        grid = [t for t in _cheb_grid(a, b, n_grid) if w(t) != 0]
        n_grid = len(grid)
        fv = [f(t) for t in grid]
        wv = [w(t) for t in grid]
        gv = [fv[k] - _poly([c for _, c in fixed], [e for e, _ in fixed], grid[k])
              for k in range(n_grid)]
        n = len(exps)
        # initial reference: evenly spaced grid indices (the grid itself is
        # Chebyshev-distributed, so these are Chebyshev-like points)
        ref = [int(round((n_grid - 1) * i / n)) for i in range(n + 1)]
        ref = sorted(set(ref))
        while len(ref) < n + 1:
            ref.append(min(n_grid - 1, ref[-1] + 1))
        cs = None
        best = None
        for it in range(max_iter):
            A = mp.matrix(n + 1, n + 1)
            rhs = mp.matrix(n + 1, 1)
            for i, k in enumerate(ref):
                t = grid[k]
                for j, e in enumerate(exps):
                    A[i, j] = t ** e
                A[i, n] = (-1) ** i / wv[k]
                rhs[i] = gv[k]
            sol = mp.lu_solve(A, rhs)
            cs = [sol[j] for j in range(n)]
            E = abs(sol[n])
            err = [wv[k] * (_poly(cs, exps, grid[k]) - gv[k]) for k in range(n_grid)]
            emax = max(abs(e) for e in err)
            best = (cs, emax)
            if verbose:
                print(f"  iter {it}: |E|={mp.nstr(E, 5)} max={mp.nstr(emax, 5)}")
            if E > 0 and (emax - E) / E < tol:
                break
            new_ref = _alternating_extrema(err, n + 1)
            if len(new_ref) < n + 1:
                new_ref = _single_exchange(ref, err)
            if new_ref == ref:
                break
            ref = new_ref
        return best


def max_error(f, w, terms, a, b, n=20000, dps=50):
    """max |w*(P-f)| on a dense grid for a list of (exponent, value) terms."""
    with mp.workdps(dps):
        grid = [t for t in _cheb_grid(a, b, n) if w(t) != 0]
        m = mp.mpf(0)
        for t in grid:
            p = _poly([c for _, c in terms], [e for e, _ in terms], t)
            m = max(m, abs(w(t) * (p - f(t))))
        return m


def _store(c, fmt):
    """(stored value(s), exact value of what is stored) for one coefficient"""
    if fmt == "d":
        v = to_double(c)
        return v, mp.mpf(v)
    if fmt == "f":
        v = to_float(c)
        return v, mp.mpf(v)
    if fmt == "dd":
        hi, lo = split_dd(c)
        return (hi, lo), mp.mpf(hi) + mp.mpf(lo)
    if fmt == "ff":
        hi, lo = split_ff(c)
        return (hi, lo), mp.mpf(hi) + mp.mpf(lo)
    v = float(_round_to_bits(c, fmt[1]))
    return v, mp.mpf(v)


def fit_rounded(f, w, exps, formats, a, b, fixed=(), **kw):
    """Fit, then store the coefficients in formats[j]: 'd' double, 'dd'
    double-double (hi, lo), 'f' float, 'ff' float-float, ('bits', k) k-bit
    mantissa.  Two candidates: (1) round coefficient j (lowest degree first)
    and refit the rest after each rounding; (2) round the free minimax fit
    directly.  Returns the one with the smaller max weighted error as
    (list of (exponent, stored value(s)), max weighted error)."""
    try:
        seq = _fit_sequential(f, w, exps, formats, a, b, fixed, **kw)
    except ZeroDivisionError:          # a degenerate reference late in the refits
        seq = None
    cs, _ = remez(f, w, list(exps), a, b, fixed=list(fixed), **kw)
    stored, terms = [], list(fixed)
    for e, c, fmt in zip(exps, cs, formats):
        v, exact = _store(c, fmt)
        stored.append((e, v))
        terms.append((e, exact))
    naive = (stored, max_error(f, w, terms, a, b))
    return seq if seq is not None and seq[1] <= naive[1] else naive


def _fit_sequential(f, w, exps, formats, a, b, fixed=(), **kw):
    fixed = list(fixed)
    stored = []
    exps = list(exps)
    formats = list(formats)
    while exps:
        cs, _ = remez(f, w, exps, a, b, fixed=fixed, **kw)
        e0, c0, fmt = exps[0], cs[0], formats[0]
        if fmt == "d":
            v = to_double(c0)
            fixed.append((e0, mp.mpf(v)))
            stored.append((e0, v))
        elif fmt == "f":
            v = to_float(c0)
            fixed.append((e0, mp.mpf(v)))
            stored.append((e0, v))
        elif fmt == "dd":
            hi, lo = split_dd(c0)
            fixed.append((e0, mp.mpf(hi) + mp.mpf(lo)))
            stored.append((e0, (hi, lo)))
        elif fmt == "ff":
            hi, lo = split_ff(c0)
            fixed.append((e0, mp.mpf(hi) + mp.mpf(lo)))
            stored.append((e0, (hi, lo)))
        else:
            _, bits = fmt
            v = float(_round_to_bits(c0, bits))
            fixed.append((e0, mp.mpf(v)))
            stored.append((e0, v))
        exps.pop(0)
        formats.pop(0)
    err = max_error(f, w, fixed, a, b)
    return stored, err


def hexf(v):
    if isinstance(v, tuple):
        return tuple(float(x).hex() for x in v)
    return float(v).hex()
