"""Exact integrals over [0,1]^d of the test families (for quadrature-error
checks, not parity).  Returned as mpmath numbers so that products over
d = 1000 factors neither underflow nor overflow."""
import mpmath as mp

mp.mp.dps = 40


def exact(fam, params, d):
    a = [mp.mpf(float(v)) for v in params[:d]]
    u = [mp.mpf(float(v)) for v in params[d:2 * d]]
    if fam == 0:      # exp(sum a_i x_i)
        return mp.fprod((mp.expm1(ai) / ai) if ai != 0 else mp.mpf(1) for ai in a)
    if fam == 1:      # cos(2 pi u_0 + sum a_i x_i)
        z = mp.expj(2 * mp.pi * u[0])
        for ai in a:
            z *= (mp.expj(ai) - 1) / (1j * ai)
        return mp.re(z)
    if fam == 2:      # prod 1/(a^-2 + (x-u)^2)
        return mp.fprod(ai * (mp.atan(ai * (1 - ui)) + mp.atan(ai * ui)) for ai, ui in zip(a, u))
    if fam == 3:      # exp(-sum a^2 (x-u)^2)
        return mp.fprod(mp.sqrt(mp.pi) / (2 * ai) * (mp.erf(ai * (1 - ui)) + mp.erf(ai * ui))
                        for ai, ui in zip(a, u))
    if fam == 4:      # exp(-sum a (x-u)^2)
        return mp.fprod(mp.sqrt(mp.pi) / (2 * mp.sqrt(ai)) *
                        (mp.erf(mp.sqrt(ai) * (1 - ui)) + mp.erf(mp.sqrt(ai) * ui))
                        for ai, ui in zip(a, u))
    raise ValueError(fam)


def as_mp(mant, exp2):
    return mp.ldexp(mp.mpf(mant), int(exp2))
