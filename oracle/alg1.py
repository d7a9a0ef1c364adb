"""Algorithm 1 and Algorithm 2 restated step by step on exact integers.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Small sizes only:
every matrix is a numpy object array of Python integers, and every product is
a plain ``@`` on those, so nothing rounds or overflows.

``alg1_low_aat`` takes the steps of Algorithm 1 (Sec. 3) in the paper's order
and notation: four additions with two multiplications by the skew-unitary Y,
three recursive products P1, P2, P5 and two general products P3, P4, then the
additions that form U1..U5.  The recursion stops after ``levels`` levels,
where Low(A A^T) is taken from its definition.  It returns the intermediate
blocks as well, so that tests can check the proof identities of Theorem 3.1.

``syrk_table4`` takes the steps of the SYRK schedule of Table 4 (Sec. 7),
one level, on the locations the table names.

``quat_6m`` takes the steps of the 6-multiplication quaternion algorithm of
Sec. 6.2 over F_p.

``two_m`` takes the steps of Algorithm 2 (Sec. 6.1) with K = R, E = C.

``winograd_gemm`` takes the steps of one level of Winograd's variant of
Strassen's algorithm (7 block products, 15 block additions; the MM_omega of
Theorem 3.1 and Table 1 with omega = log2 7) for a general product X Y^T mod
p; ``alg1_low_aat`` can use it for its two general products P3 and P4.
"""
from __future__ import annotations

import numpy as np


def _obj(A):
    return np.asarray(A, dtype=object)


def low(M):
    """Low(M): entries with i >= j kept, the others set to 0 (Sec. 2)."""
    M = _obj(M).copy()
    n, m = M.shape
    for i in range(n):
        for j in range(i + 1, m):
            M[i, j] = 0
    return M


def dense_y(ykind, ya, yb, p, kappa):
    """Y as a dense kappa x kappa matrix of Python integers mod p.

    ykind 1: Y = i I (Sec. 4.2).  ykind 2: Y = [[a, b], [-b, a]] (x) I_{kappa/2}
    (Prop. 4.2)."""
    Y = np.zeros((kappa, kappa), dtype=object)
    if ykind == 1:
        for j in range(kappa):
            Y[j, j] = ya % p
        return Y
    if ykind == 2:
        if kappa % 2:
            raise ValueError("kappa must be even for the 2x2 (x) I form")
        h = kappa // 2
        for j in range(h):
            Y[j, j] = ya % p
            Y[j, j + h] = yb % p
            Y[j + h, j] = (-yb) % p
            Y[j + h, j + h] = ya % p
        return Y
    raise ValueError("unknown ykind")


def alg1_low_aat(A, p, ykind, ya, yb, levels, trace=None, gemm=None):
    """Low(A A^T) mod p by Algorithm 1 applied ``levels`` times.

    ``trace`` (a list) receives, for the top level, a dict with S1..S4,
    P1..P5, U1..U5 (all mod p) when given.  ``gemm(X, Y, p)`` (X Y^T mod p)
    computes the general products P3 and P4 of every level when given;
    otherwise they are plain products."""
    A = _obj(A) % p
    n, k = A.shape
    need = 4 if ykind == 2 else 2
    if levels == 0 or n % 2 or k % need or n == 0 or k == 0:
        return low((A @ A.T) % p)
    h, kap = n // 2, k // 2
    A11, A12 = A[:h, :kap], A[:h, kap:]
    A21, A22 = A[h:, :kap], A[h:, kap:]
    Y = dense_y(ykind, ya, yb, p, kap)
    # 4 additions and 2 multiplications by Y
    S1 = ((A21 - A11) @ Y) % p
    S2 = (A22 - A21 @ Y) % p
    S3 = (S1 - A22) % p
    S4 = (S3 + A12) % p
    # 3 recursive and 2 general products
    P1 = alg1_low_aat(A11, p, ykind, ya, yb, levels - 1, gemm=gemm)
    P2 = alg1_low_aat(A12, p, ykind, ya, yb, levels - 1, gemm=gemm)
    if gemm is None:
        P3 = (A22 @ S4.T) % p
        P4 = (S1 @ S2.T) % p
    else:
        P3 = _obj(gemm(A22, S4, p)) % p
        P4 = _obj(gemm(S1, S2, p)) % p
    P5 = alg1_low_aat(S3, p, ykind, ya, yb, levels - 1, gemm=gemm)
    # 3 half additions and 2 complete additions
    U1_low = (P1 + P5) % p
    U3_low = (P1 + P2) % p
    U1 = U1_low.copy()
    for i in range(h):            # Up(U1) <- Low(U1)^T forms the full U1
        for j in range(i + 1, h):
            U1[i, j] = U1_low[j, i]
    U2 = (U1 + P4) % p
    U4 = (U2 + P3) % p
    U5_low = low((U2 + P4.T) % p)
    C = np.zeros((n, n), dtype=object)
    C[:h, :h] = low(U3_low)
    C[h:, :h] = U4
    C[h:, h:] = U5_low
    if trace is not None:
        trace.append(dict(S1=S1, S2=S2, S3=S3, S4=S4, P1=P1, P2=P2, P3=P3,
                          P4=P4, P5=P5, U1=U1, U2=U2, U3=U3_low, U4=U4,
                          U5=U5_low, Y=Y))
    return C


def syrk_table4(alpha, A, beta, C, p, ykind, ya, yb, save_diagonal=True):
    """Low(alpha A A^T + beta C) mod p by the schedule of Table 4 (Sec. 7),
    one level of Algorithm 1 with the leaves from their definitions.

    The locations of Table 4 are modelled as blocks of one n x n array M
    (initially C) plus an h x h array tmp, and each step reads and writes only
    the locations the table names, in its order.  Reading: Up(C11) includes
    the diagonal (Sec. 2), which C11 still needs for P2 = alpha A12 A12^T +
    beta C11, so the diagonal of Low(C22) is kept in a separate h-vector
    (``save_diagonal``); with ``save_diagonal=False`` the schedule is taken
    literally (Up(C11) <- Low(C22)^T over the diagonal), which loses C11's
    diagonal (tests show that it does)."""
    A = _obj(A) % p
    n, k = A.shape
    h, kap = n // 2, k // 2
    al, be = alpha % p, beta % p
    M = _obj(C) % p
    A11, A12 = A[:h, :kap], A[:h, kap:]
    A21, A22 = A[h:, :kap], A[h:, kap:]
    Y = dense_y(ykind, ya, yb, p, kap)
    C11 = lambda: M[:h, :h]          # noqa: E731  views of the locations
    C12 = lambda: M[:h, h:]          # noqa: E731
    C21 = lambda: M[h:, :h]          # noqa: E731
    C22 = lambda: M[h:, h:]          # noqa: E731
    tmp = np.zeros((h, kap if kap > h else h), dtype=object)
    # left column of Table 4
    S1 = ((A21 - A11) @ Y) % p                       # S1 -> tmp
    tmp[:, :kap] = S1
    C12()[:, :kap] = (A22 - A21 @ Y) % p              # S2 -> C12
    S2 = C12()[:, :kap].copy()
    dg = [C22()[i, i] for i in range(h)]
    for i in range(h):                                # Up(C11) <- Low(C22)^T
        for j in range(i, h):
            if i == j and save_diagonal:
                continue
            C11()[i, j] = C22()[j, i]
    C22()[:, :] = (al * (S2 @ S1.T)) % p             # P4^T = alpha S2 S1^T -> C22
    tmp[:, :kap] = (tmp[:, :kap] - A22) % p           # S3 = S1 - A22 -> tmp
    S3 = tmp[:, :kap].copy()
    C12()[:, :] = low((al * (S3 @ S3.T)) % p)         # P5 = alpha S3 S3^T -> C12
    tmp[:, :kap] = (tmp[:, :kap] + A12) % p           # S4 = S3 + A12 -> tmp
    S4 = tmp[:, :kap].copy()
    C21()[:, :] = (al * (A22 @ S4.T) + be * C21()) % p  # P3 -> C21
    # right column of Table 4
    tmp = np.zeros((h, h), dtype=object)
    tmp[:, :] = low((al * (A11 @ A11.T)) % p)         # P1 -> tmp
    U1 = low((tmp + C12()) % p)                       # U1 = P1 + P5 -> C12
    for i in range(h):                                # Up(U1) <- Low(U1)^T
        for j in range(i + 1, h):
            U1[i, j] = U1[j, i]
    C12()[:, :] = U1
    P4T = C22().copy()
    C12()[:, :] = (C12() + P4T.T) % p                 # U2 = U1 + P4 -> C12
    U2 = C12().copy()
    C21()[:, :] = (U2 + C21()) % p                    # U4 = U2 + P3 -> C21
    old22 = np.zeros((h, h), dtype=object)            # beta Up(C11)^T (+ saved diagonal)
    for i in range(h):
        for j in range(i + 1):
            old22[i, j] = (dg[i] if (i == j and save_diagonal) else C11()[j, i])
    C22()[:, :] = low((U2 + P4T + be * old22) % p)    # U5 -> C22
    C11()[:, :] = low((al * (A12 @ A12.T) + be * C11()) % p)  # P2 -> C11
    C11()[:, :] = low((tmp + C11()) % p)              # U3 = P1 + P2 -> C11
    return low(M)


def quat_6m(A, B, C, D, p):
    """The 6-multiplication algorithm of Sec. 6.2 for M M^H, M = A + B i +
    C j + D k a quaternion matrix (Q6 a product by its own transpose), in the
    paper's order and notation (U1, U2, Q1..Q6, T1..T3, H1..H4), on exact
    integers mod p.
    Returns Low(H1), Low(H2), Low(H3), Low(H4)."""
    A, B, C, D = (_obj(X) % p for X in (A, B, C, D))
    U1 = (A + B) % p
    U2 = (C + D) % p
    Q1 = (C @ A.T) % p
    Q2 = (D @ B.T) % p
    Q3 = (U2 @ U1.T) % p
    Q4 = (A @ B.T) % p
    Q5 = (C @ D.T) % p
    Q6 = ((U1 + U2) @ (U1 + U2).T) % p
    T1 = (Q1 - Q2) % p
    T2 = (Q4 + Q5) % p
    T3 = ((Q1 + Q2) - Q3) % p
    H1 = low((Q6 - (Q3.T + Q3) - (T2.T + T2)) % p)
    H2 = low((T2.T - T2) % p)
    H3 = low((T1 - T1.T) % p)
    H4 = low((T3.T - T3) % p)
    return H1, H2, H3, H4


def two_m(Are, Aim, conj=True):
    """Algorithm 2 with K = R, E = C, A + iB the complex input.

    phi is the transposition on real matrices; on C it is the conjugate
    transposition (eps = i phi(i) = 1) or the transposition (eps = i i = -1).
    Returns (Re, Im) of (A + iB) phi(A + iB)."""
    A = np.asarray(Are, dtype=np.float64)
    B = np.asarray(Aim, dtype=np.float64)
    eps = 1.0 if conj else -1.0
    H = A @ B.T
    G = (A + B) @ (A + eps * B).T
    # (G - eps H - H^T) + H phi(i) + i H^T, with phi(i) = -i (conj) or i
    re = G - eps * H - H.T
    if conj:
        im = H.T - H          # H (-i) + i H^T
    else:
        im = H + H.T          # H i + i H^T
    return re, im


def winograd_gemm(X, Y, p, trace=None):
    """X Y^T mod p by one level of Winograd's form of Strassen's algorithm.

    With A = X (M x K) and B = Y^T (K x N), both cut into 2 x 2 blocks (M, N,
    K even), Winograd's form takes 8 additions before the products
        S1 = A21 + A22, S2 = S1 - A11, S3 = A11 - A21, S4 = A12 - S2,
        T1 = B12 - B11, T2 = B22 - T1, T3 = B22 - B12, T4 = T2 - B21,
    7 block products
        P1 = A11 B11, P2 = A12 B21, P3 = S4 B22, P4 = A22 T4,
        P5 = S1 T1,   P6 = S2 T2,   P7 = S3 T3,
    and 7 additions after them
        U1 = P1 + P2, U2 = P1 + P6, U3 = U2 + P7, U4 = U2 + P5,
        U5 = U4 + P3, U6 = U3 - P4, U7 = U3 + P5,
    giving C11 = U1, C12 = U5, C21 = U6, C22 = U7.  Every block sum is taken
    mod p.  ``trace`` receives the blocks when given."""
    X = _obj(X) % p
    Y = _obj(Y) % p
    M, K = X.shape
    N = Y.shape[0]
    if M % 2 or N % 2 or K % 2:
        raise ValueError("M, N and K must be even")
    m, n, k = M // 2, N // 2, K // 2
    B = Y.T
    A11, A12, A21, A22 = X[:m, :k], X[:m, k:], X[m:, :k], X[m:, k:]
    B11, B12, B21, B22 = B[:k, :n], B[:k, n:], B[k:, :n], B[k:, n:]
    S1 = (A21 + A22) % p
    S2 = (S1 - A11) % p
    S3 = (A11 - A21) % p
    S4 = (A12 - S2) % p
    T1 = (B12 - B11) % p
    T2 = (B22 - T1) % p
    T3 = (B22 - B12) % p
    T4 = (T2 - B21) % p
    P1 = (A11 @ B11) % p
    P2 = (A12 @ B21) % p
    P3 = (S4 @ B22) % p
    P4 = (A22 @ T4) % p
    P5 = (S1 @ T1) % p
    P6 = (S2 @ T2) % p
    P7 = (S3 @ T3) % p
    U1 = (P1 + P2) % p
    U2 = (P1 + P6) % p
    U3 = (U2 + P7) % p
    U4 = (U2 + P5) % p
    U5 = (U4 + P3) % p
    U6 = (U3 - P4) % p
    U7 = (U3 + P5) % p
    C = np.zeros((M, N), dtype=object)
    C[:m, :n] = U1
    C[:m, n:] = U5
    C[m:, :n] = U6
    C[m:, n:] = U7
    if trace is not None:
        trace.append(dict(S=(S1, S2, S3, S4), T=(T1, T2, T3, T4),
                          P=(P1, P2, P3, P4, P5, P6, P7)))
    return C
