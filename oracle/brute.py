"""Scalar pure-Python restatement of the modal heat current for tiny systems.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Written with per-atom
3-vectors and 3x3 tensors exactly as the paper writes the equations, so that
it is structurally different from the flattened loops in mhc_oracle.c:

  Eq. 10  J = sum_i W_i . v_i
  Eq. 13  Xdot_n = sum_i sqrt(m_i) e_{i,n} . v_i
  Eq. 16  J_n = (sum_i m_i^{-1/2} W_i . e_{i,n}) Xdot_n
  Eq. 17  C_b^{mu nu}(l) = < J_b^mu(t) J^nu(t - l) >  (average over origins)
  Eq. 19  <J_b^mu>
Intended for N <= 8 atoms and a few dozen steps.
"""
from __future__ import annotations

import math


def matvec(Wi, e):
    """(W e)^a = sum_b W^{ab} e^b for a 3x3 nested list W and a 3-vector e."""
    return [Wi[a][0] * e[0] + Wi[a][1] * e[1] + Wi[a][2] * e[2] for a in range(3)]


def dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def step(e, mass, v, W):
    """One time step.  e[i][n] is the 3-vector e_{i,n}; v[i] a 3-vector;
    W[i] a 3x3 nested list.  Returns (Xdot[n], Jn[n][3], J[3])."""
    N = len(mass)
    M = len(e[0])
    J = [0.0, 0.0, 0.0]
    for i in range(N):
        wv = matvec(W[i], v[i])
        for a in range(3):
            J[a] += wv[a]
    Xdot = []
    Jn = []
    for n in range(M):
        x = 0.0
        y = [0.0, 0.0, 0.0]
        for i in range(N):
            x += math.sqrt(mass[i]) * dot(e[i][n], v[i])
            we = matvec(W[i], e[i][n])
            for a in range(3):
                y[a] += we[a] / math.sqrt(mass[i])
        Xdot.append(x)
        Jn.append([y[a] * x for a in range(3)])
    return Xdot, Jn, J


def run(E, mass, v, W, bin_of_mode, B, L=0):
    """E: dof-major nested list/array [3N][M]; v [T][N][3]; W [T][N][9].
    Returns dict with Jb [T][B][3], J [T][3], Xdot, Jn, and C [B][3][3][L]
    (averaged over origins) when L > 0, and meanJb [B][3]."""
    N = len(mass)
    M = len(E[0])
    e = [[[float(E[3 * i + b][n]) for b in range(3)] for n in range(M)] for i in range(N)]
    T = len(v)
    Jb_t, J_t, X_t, Jn_t = [], [], [], []
    for t in range(T):
        vt = [[float(v[t][i][b]) for b in range(3)] for i in range(N)]
        Wt = [[[float(W[t][i][3 * a + b]) for b in range(3)] for a in range(3)] for i in range(N)]
        Xdot, Jn, J = step(e, [float(m) for m in mass], vt, Wt)
        Jb = [[0.0, 0.0, 0.0] for _ in range(B)]
        for n in range(M):
            b = int(bin_of_mode[n])
            if 0 <= b < B:
                for a in range(3):
                    Jb[b][a] += Jn[n][a]
        Jb_t.append(Jb)
        J_t.append(J)
        X_t.append(Xdot)
        Jn_t.append(Jn)
    out = {"Jb": Jb_t, "J": J_t, "xdot": X_t, "Jn": Jn_t}
    mean = [[sum(Jb_t[t][b][a] for t in range(T)) / T for a in range(3)] for b in range(B)]
    out["meanJb"] = mean
    if L > 0:
        C = [[[[0.0] * L for _ in range(3)] for _ in range(3)] for _ in range(B)]
        for b in range(B):
            for mu in range(3):
                for nu in range(3):
                    for l in range(L):
                        pairs = [Jb_t[t][b][mu] * J_t[t - l][nu] for t in range(l, T)]
                        C[b][mu][nu][l] = sum(pairs) / len(pairs) if pairs else 0.0
        out["C"] = C
    return out


def step_dir(e, mass, v, W):
    """Direction-resolved step: J_n^{ab} = Xdot_n sum_i W_i^{ab} e^b_{i,n} / sqrt(m_i), i.e. the
    heat current of the modal atomic velocities v_{i,n} = Xdot_n e_{i,n}/sqrt(m_i) (Eq. 14)
    restricted to their b-th component.  Returns Jn[n][b][a]."""
    N = len(mass)
    M = len(e[0])
    out = []
    for n in range(M):
        x = sum(math.sqrt(mass[i]) * dot(e[i][n], v[i]) for i in range(N))
        jn = [[0.0, 0.0, 0.0] for _ in range(3)]
        for i in range(N):
            # modal velocity of atom i, component b only
            for b in range(3):
                vb = x * e[i][n][b] / math.sqrt(mass[i])
                for a in range(3):
                    jn[b][a] += W[i][a][b] * vb
        out.append(jn)
    return out


def run_dir(E, mass, v, W, bin_of_mode, B):
    """Binned direction-resolved current Jbd[t][b][bin][a]."""
    N = len(mass)
    M = len(E[0])
    e = [[[float(E[3 * i + b][n]) for b in range(3)] for n in range(M)] for i in range(N)]
    out = []
    for t in range(len(v)):
        vt = [[float(v[t][i][b]) for b in range(3)] for i in range(N)]
        Wt = [[[float(W[t][i][3 * a + b]) for b in range(3)] for a in range(3)] for i in range(N)]
        jn = step_dir(e, [float(m) for m in mass], vt, Wt)
        jb = [[[0.0, 0.0, 0.0] for _ in range(B)] for _ in range(3)]
        for n in range(M):
            bn = int(bin_of_mode[n])
            if 0 <= bn < B:
                for b in range(3):
                    for a in range(3):
                        jb[b][bn][a] += jn[n][b][a]
        out.append(jb)
    return out


def shc(v, W, nc):
    """Eq. 21 with per-atom tensors: K^{ab}(l) = < sum_i W_i^{ab}(t - l) v_i^b(t) > over the
    origins t - l >= 0 (not summed over b; summing over b gives K^a)."""
    T = len(v)
    N = len(v[0])
    out = [[0.0] * nc for _ in range(9)]
    for l in range(nc):
        n = 0
        acc = [0.0] * 9
        for t in range(l, T):
            n += 1
            for i in range(N):
                Wi = [[float(W[t - l][i][3 * a + b]) for b in range(3)] for a in range(3)]
                vi = [float(v[t][i][b]) for b in range(3)]
                for a in range(3):
                    for b in range(3):
                        acc[3 * a + b] += Wi[a][b] * vi[b]
        for c in range(9):
            out[c][l] = acc[c] / n if n else 0.0
    return out
