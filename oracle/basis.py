"""Reference-element basis of the nodal spectral element method, FP64 numpy.

Test infrastructure only (see ``oracle/__init__``).

Paper passages followed:
  * orthonormal Legendre polynomials by the three-term recurrence, with
    P~0 = 1/sqrt(2), P~1 = sqrt(3/2) x and a_k = sqrt(k^2/((2k+1)(2k-1)))      (Sec. 4.3)
  * Legendre-Gauss-Lobatto (LGL) nodal distribution                          (Sec. 4.3)
  * generalized Vandermonde V_ij = psi_j(r_i), V_r = d/dr psi_j(r_i),
    exact mass M = (V V^T)^-1, derivative D_r = V_r V^-1                      (Sec. 4.3)
  * p-transfer I_Pp = Phi^p V^-1 with Phi^p_ij = psi_j(x^p_i)                 (Sec. 5.2)

Pins (tests/test_oracle_basis.py): closed-form LGL nodes and weights for p <= 4,
orthonormality by an independent Gauss-Legendre rule, row sums of M equal the LGL
weights, D exact on polynomials of degree <= p, transfers exact on degree-p data.
"""
import numpy as np


def recurrence_coeff(k):
    """a_k of the orthonormal Legendre recurrence (Sec. 4.3)."""
    return np.sqrt(k * k / ((2.0 * k + 1.0) * (2.0 * k - 1.0)))


def legendre_orthonormal(x, n):
    """Columns P~_0..P~_n evaluated at the points x (Sec. 4.3 recurrence).

    a_k P~_k(x) = x P~_{k-1}(x) - a_{k-1} P~_{k-2}(x).
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.zeros((x.size, n + 1))
    out[:, 0] = 1.0 / np.sqrt(2.0)
    if n >= 1:
        out[:, 1] = np.sqrt(1.5) * x
    for k in range(2, n + 1):
        prev2 = recurrence_coeff(k - 1) * out[:, k - 2] if k >= 2 else 0.0
        out[:, k] = (x * out[:, k - 1] - prev2) / recurrence_coeff(k)
    return out


def legendre_orthonormal_deriv(x, n):
    """d/dx of P~_0..P~_n: the recurrence differentiated term by term.

    a_k P~'_k = P~_{k-1} + x P~'_{k-1} - a_{k-1} P~'_{k-2}.
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    p = legendre_orthonormal(x, n)
    out = np.zeros((x.size, n + 1))
    if n >= 1:
        out[:, 1] = np.sqrt(1.5)
    for k in range(2, n + 1):
        out[:, k] = (p[:, k - 1] + x * out[:, k - 1]
                     - recurrence_coeff(k - 1) * out[:, k - 2]) / recurrence_coeff(k)
    return out


def _legendre_std(x, p):
    """Standard-normalised Legendre L_p and L_p' (L_p(1) = 1), from the orthonormal ones.

    P~_p = sqrt((2p+1)/2) L_p.
    """
    c = np.sqrt((2.0 * p + 1.0) / 2.0)
    return legendre_orthonormal(x, p)[:, p] / c, legendre_orthonormal_deriv(x, p)[:, p] / c


def lgl_nodes_weights(p):
    """LGL nodes (ascending) and weights of order p >= 1.

    Nodes: -1, +1 and the p-1 roots of L_p'.  The roots are found by Newton's method
    on L_p' with L_p'' taken from Legendre's equation,
    (1 - x^2) L'' = 2 x L' - p(p+1) L, starting from the Chebyshev-Gauss-Lobatto
    points -cos(pi i / p).  Weights: w_i = 2 / (p (p+1) L_p(x_i)^2).
    """
    if p < 1:
        raise ValueError("order must be >= 1")
    x = -np.cos(np.pi * np.arange(p + 1) / p)
    interior = x[1:-1].copy()
    for _ in range(100):
        if interior.size == 0:
            break
        L, dL = _legendre_std(interior, p)
        ddL = (2.0 * interior * dL - p * (p + 1.0) * L) / (1.0 - interior ** 2)
        step = dL / ddL
        interior -= step
        if np.max(np.abs(step)) < 1e-16:
            break
    x = np.concatenate(([-1.0], np.sort(interior), [1.0]))
    L, _ = _legendre_std(x, p)
    w = 2.0 / (p * (p + 1.0) * L ** 2)
    return x, w


def vandermonde(p):
    """(V, V_r) of order p at its own LGL nodes (Sec. 4.3)."""
    r, _ = lgl_nodes_weights(p)
    return legendre_orthonormal(r, p), legendre_orthonormal_deriv(r, p)


def diff_matrix(p):
    """D_r = V_r V^{-1}: nodal derivative on [-1, 1] (Sec. 4.3)."""
    V, Vr = vandermonde(p)
    return Vr @ np.linalg.inv(V)


def exact_mass_1d(p):
    """Exact 1D mass matrix M = (V V^T)^{-1} (Sec. 4.3)."""
    V, _ = vandermonde(p)
    return np.linalg.inv(V @ V.T)


def transfer_1d(p_from, p_to):
    """I = Phi V^{-1}: maps nodal values of order p_from to nodal values at the LGL
    nodes of order p_to by evaluating the order-p_from modal expansion there (Sec. 5.2).

    With p_to > p_from this is the 1D factor of the prolongation (interpolation of the
    coarse polynomial at the fine nodes); shape (p_to + 1, p_from + 1).
    """
    V_from, _ = vandermonde(p_from)
    r_to, _ = lgl_nodes_weights(p_to)
    Phi = legendre_orthonormal(r_to, p_from)
    return Phi @ np.linalg.inv(V_from)


def coarsening_sequence(P):
    """Level orders P_N > ... > P_1 from P_{n-1} = ceil((P_n + 1) / 2) (Sec. 5.1).

    The rule has the fixed point 2 (ceil(3/2) = 2) and does not name the coarsest
    order; the sequence is iterated down to 2 and the order-1 level appended.
    """
    seq = [int(P)]
    while seq[-1] > 2:
        seq.append(int(np.ceil((seq[-1] + 1) / 2.0)))
    if seq[-1] != 1:
        seq.append(1)
    return seq


def semi_coarsening_sequence(P, Pz):
    """Level order pairs (p_x, p_z) for different horizontal and vertical orders (Sec. 5.1:
    semi-coarsening reduces the higher order until the two match).  Reading: while they
    differ, only the higher order takes a step of the rule P_{n-1} = ceil((P_n + 1) / 2),
    clamped so as not to fall below the other; once equal, both follow
    `coarsening_sequence`."""
    px, pz = int(P), int(Pz)
    seq = [(px, pz)]
    while px != pz:
        if px > pz:
            px = max(pz, int(np.ceil((px + 1) / 2.0)))
        else:
            pz = max(px, int(np.ceil((pz + 1) / 2.0)))
        seq.append((px, pz))
    seq += [(p, p) for p in coarsening_sequence(px)[1:]]
    return seq
