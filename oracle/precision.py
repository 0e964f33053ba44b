"""Oracle for the a-priori precision rule (test infrastructure only).

Section 5.4: the accumulated rounding error of g gate applications on N = 2^n
amplitudes is bounded by eps_round <= g N eps_mach (Eq. 11); complex64 is chosen iff
g 2^n 1.19e-7 <= eps_tol (Eq. 12), otherwise complex128.  The paper prints the value of
the left-hand side for n = 20, g = 200 as about 2.5e1.
"""

EPS_MACH_F32 = 1.19e-7     # the constant Eq. 12 uses
EPS_MACH_F64 = 2.22e-16    # Section 5.4


def eps_round(n: int, g: int, eps_mach: float = EPS_MACH_F32) -> float:
    """Right-hand side of Eq. 11 (= left-hand side of Eq. 12 for float32)."""
    return g * (2 ** n) * eps_mach


def choose_c64(n: int, g: int, eps_tol: float) -> bool:
    """Eq. 12: complex64 iff g 2^n 1.19e-7 <= eps_tol."""
    return eps_round(n, g) <= eps_tol
