"""Critical Reynolds number and grid extrapolation -- oracle.

TEST INFRASTRUCTURE ONLY.

Section 3: the steady flow becomes unstable at Re_cr where the real part of
the leading eigenvalue Lambda crosses zero; the critical circular frequency
is omega_cr ~ Im(Lambda).  The paper does not say how Re_cr is bracketed;
this project uses the secant iteration on sigma(Re) = Re(Lambda(Re)).

Section 5 / Table 3: Richardson extrapolation to zero grid size from two
consecutive grids N1 < N2 of a second-order method,
  X_inf = (N2^2 X2 - N1^2 X1) / (N2^2 - N1^2).

Pinned by: the printed Richardson values of Table 3 (tests/golden/table3.json)
and, for the secant, a closed-form test function.
"""


def richardson(n1, x1, n2, x2, order=2):
    a, b = float(n1) ** order, float(n2) ** order
    return (b * x2 - a * x1) / (b - a)


def secant(sigma, re0, re1, rtol=1e-6, max_iter=30):
    """Root of sigma(Re) by the secant method.  ``sigma`` returns
    (real part, extra) for a Re; returns (Re_cr, extra at Re_cr, history)."""
    s0, _ = sigma(re0)
    s1, extra = sigma(re1)
    hist = [(re0, s0), (re1, s1)]
    for _ in range(max_iter):
        if s1 == s0:
            break
        re2 = re1 - s1 * (re1 - re0) / (s1 - s0)
        re0, s0 = re1, s1
        re1 = re2
        s1, extra = sigma(re1)
        hist.append((re1, s1))
        if abs(re1 - re0) <= rtol * abs(re1):
            return re1, extra, hist
    raise RuntimeError(f"secant did not converge: {hist[-3:]}")
