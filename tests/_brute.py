"""A second, loop-only restatement of the propagation (pin P-14 of the oracle).

Plain Python loops over matrix elements and lists of complex numbers; no numpy
linear algebra, written independently of ``oracle/``.  Only practical for a
handful of orbitals and one k-point (Gamma), where every phase is 1.
"""
C = 137.035999084


def _zeros(n):
    return [[0j] * n for _ in range(n)]


def _mul(a, b):
    n = len(a)
    out = _zeros(n)
    for i in range(n):
        ai = a[i]
        oi = out[i]
        for k in range(n):
            x = ai[k]
            if x == 0:
                continue
            bk = b[k]
            for j in range(n):
                oi[j] += x * bk[j]
    return out


def _inv(a):
    """Gauss-Jordan inverse with partial pivoting."""
    n = len(a)
    m = [list(a[i]) + [1.0 + 0j if j == i else 0j for j in range(n)] for i in range(n)]
    for c in range(n):
        p = max(range(c, n), key=lambda r: abs(m[r][c]))
        m[c], m[p] = m[p], m[c]
        piv = m[c][c]
        m[c] = [x / piv for x in m[c]]
        for r in range(n):
            if r != c and m[r][c] != 0:
                f = m[r][c]
                m[r] = [x - f * y for x, y in zip(m[r], m[c])]
    return [row[n:] for row in m]


def propagate_gamma(sysd, A_table, nsteps, D0):
    """Return (J list, D final) for a Gamma-only system, loop by loop."""
    off = [int(x) for x in sysd["orb_offset"]]
    nat = len(off) - 1
    n = off[-1]
    kx = [float(x) for x in sysd["kpt"][0]]
    assert kx == [0.0, 0.0, 0.0]
    lat = [[float(x) for x in r] for r in sysd["lattice"]]
    omega = abs(lat[0][0] * (lat[1][1] * lat[2][2] - lat[1][2] * lat[2][1])
                - lat[0][1] * (lat[1][0] * lat[2][2] - lat[1][2] * lat[2][0])
                + lat[0][2] * (lat[1][0] * lat[2][1] - lat[1][1] * lat[2][0]))
    S, H0 = _zeros(n), _zeros(n)
    P = [_zeros(n) for _ in range(3)]
    pos = 0
    for row in sysd["blk_ijl"]:
        I, J = int(row[0]), int(row[1])
        ni, nj = off[I + 1] - off[I], off[J + 1] - off[J]
        for a in range(ni):
            for b in range(nj):
                e = pos + a * nj + b
                S[off[I] + a][off[J] + b] += float(sysd["s"][e])
                H0[off[I] + a][off[J] + b] += float(sysd["h0"][e])
                for c in range(3):
                    P[c][off[I] + a][off[J] + b] += 1j * float(sysd["ds"][c][e])
        pos += ni * nj
    Si = _inv(S)
    atom = [I for I in range(nat) for _ in range(off[I + 1] - off[I])]
    gam = [[float(x) for x in r] for r in sysd["gamma"]]
    z = [float(x) for x in sysd["z_ref"]]
    dt = float(sysd["dt"])
    D = [[complex(D0[i][j]) for j in range(n)] for i in range(n)]
    Dp = None
    Js = []
    for step in range(nsteps + 1):
        A = [float(x) for x in A_table[step]]
        a2 = sum(x * x for x in A)
        q = [0.0] * nat
        for mu in range(n):
            q[atom[mu]] += sum(D[mu][nu] * S[nu][mu] for nu in range(n)).real
        dq = [q[I] - z[I] for I in range(nat)]
        eps = [sum(gam[I][K] * dq[K] for K in range(nat)) for I in range(nat)]
        J = []
        for c in range(3):
            tr = 0j
            for mu in range(n):
                for nu in range(n):
                    tr += D[mu][nu] * (P[c][nu][mu] + A[c] / C * S[nu][mu])
            J.append(-tr.real / omega)
        Js.append(J)
        if step == nsteps:
            break
        H = _zeros(n)
        for mu in range(n):
            for nu in range(n):
                H[mu][nu] = (H0[mu][nu] + 0.5 * (eps[atom[mu]] + eps[atom[nu]]) * S[mu][nu]
                             + sum(A[c] * P[c][mu][nu] for c in range(3)) / C
                             + a2 / (2 * C * C) * S[mu][nu])
        X = _mul(_mul(Si, H), D)
        Y = _mul(_mul(D, H), Si)
        Dd = [[-1j * (X[i][j] - Y[i][j]) for j in range(n)] for i in range(n)]
        if Dp is None:
            Dn = [[D[i][j] + dt * Dd[i][j] for j in range(n)] for i in range(n)]
        else:
            Dn = [[Dp[i][j] + 2 * dt * Dd[i][j] for j in range(n)] for i in range(n)]
        Dp, D = D, Dn
    return Js, D
