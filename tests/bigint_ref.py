"""Big-integer restatement of BFV ring operations, for pinning the oracle.

Works on Python integers modulo the full composite moduli Q and QP (no RNS
limbs, no NTT): negacyclic products by the schoolbook definition, key
switching as the rounded division round(u / P), decryption by the integer
formula of Sec. 2.  It is a different formulation from the oracle's RNS code,
so agreement pins the oracle's limb-wise arithmetic.  Small N only.
"""
from __future__ import annotations


def crt(residues, moduli) -> int:
    M = 1
    for m in moduli:
        M *= m
    x = 0
    for r, m in zip(residues, moduli):
        Mi = M // m
        x += int(r) * Mi * pow(Mi % m, -1, m)
    return x % M


def poly_crt(limbs, moduli) -> list[int]:
    """limbs[j][n] residues mod moduli[j] -> list of integers mod prod(moduli)."""
    N = len(limbs[0])
    return [crt([limbs[j][n] for j in range(len(moduli))], moduli) for n in range(N)]


def negacyclic_mul(a, b, M: int) -> list[int]:
    N = len(a)
    out = [0] * N
    for x in range(N):
        ax = int(a[x])
        if ax == 0:
            continue
        for y in range(N):
            k = x + y
            if k < N:
                out[k] += ax * int(b[y])
            else:
                out[k - N] -= ax * int(b[y])
    return [v % M for v in out]


def automorphism(a, k: int, M: int) -> list[int]:
    N = len(a)
    out = [0] * N
    for n in range(N):
        e = (n * k) % (2 * N)
        if e < N:
            out[e] = int(a[n]) % M
        else:
            out[e - N] = (-int(a[n])) % M
    return out


def rotate(prm, k: int, key, ct) -> list[list[int]]:
    """Rot_k with hybrid key switching stated over Z_QP:
    d_i = [sigma(c1)]_{q_i} (an integer in [0, q_i)),
    u = sum_i d_i * key_i  (key_i CRT-composed over q_0..q_{L-1}, P),
    u' = round(u / P) mod Q, result (sigma(c0) + u0', u1')."""
    L, q, P = prm.L, prm.q, prm.P
    Q = prm.Q
    QP = Q * P
    mods = list(q) + [P]
    c0 = poly_crt(ct[0], q)
    c1 = poly_crt(ct[1], q)
    s0 = automorphism(c0, k, Q)
    s1 = automorphism(c1, k, Q)
    N = len(s0)
    u = [[0] * N, [0] * N]
    for i in range(L):
        d_i = [v % q[i] for v in s1]
        for comp in range(2):
            kp = poly_crt(key[i][comp], mods)
            prod = negacyclic_mul(d_i, kp, QP)
            u[comp] = [(x + y) % QP for x, y in zip(u[comp], prod)]
    # nearest integer to u/P (P odd: no ties), for u in [0, QP)
    down = [[((2 * v + P) // (2 * P)) % Q for v in u[c]] for c in range(2)]
    r0 = [(x + y) % Q for x, y in zip(s0, down[0])]
    r1 = down[1]
    return [[[v % qi for v in r0] for qi in q], [[v % qi for v in r1] for qi in q]]


def ptct_sum(prm, ptxts, cts):
    """sum_b P_b * ct_b over Z_Q (P_b given as residues [L][N])."""
    q, Q = prm.q, prm.Q
    N = prm.N
    acc = [[0] * N, [0] * N]
    for pt, ct in zip(ptxts, cts):
        pz = poly_crt(pt, q)
        for comp in range(2):
            cz = poly_crt(ct[comp], q)
            prod = negacyclic_mul(pz, cz, Q)
            acc[comp] = [(x + y) % Q for x, y in zip(acc[comp], prod)]
    return [[[v % qi for v in acc[c]] for qi in q] for c in range(2)]


def add(prm, a, b):
    return [[[(int(x) + int(y)) % prm.q[l] for x, y in zip(a[c][l], b[c][l])] for l in range(prm.L)]
            for c in range(2)]


def eval_query(prm, ptxt, ct, keys):
    """Alg. "Server Computation" with the readings of the oracle (chained Rot_1
    baby steps, Horner with Rot_g), every operation in big integers."""
    g, h = prm.g, prm.h
    ctp = [ct]
    for _ in range(1, g):
        ctp.append(rotate(prm, prm.k1, keys[0], ctp[-1]))
    outs = []
    for k in range(len(ptxt)):
        T = [ptct_sum(prm, [ptxt[k][i][b] for b in range(g)], ctp) for i in range(h)]
        S = T[h - 1]
        for i in range(h - 2, -1, -1):
            S = add(prm, rotate(prm, prm.kg, keys[1], S), T[i])
        outs.append(S)
    return outs
