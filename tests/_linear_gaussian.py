"""Closed form of the linear-Gaussian test model (test helper, no oracle code).

For dx/dt = K x + (p0, I) the RK4 map is exactly x -> T x + h S (p0, I) with
T = I + Z + Z^2/2 + Z^3/6 + Z^4/24 and S = I + Z/2 + Z^2/6 + Z^3/24, Z = h K.
Every residual of the action (delta_n, eps_{n+1}) is then affine in
z = (X, p): e = L z - r, and A(z) = 1/2 e^T W e.  The posterior exp(-A) is
Gaussian with precision Q = L^T W L and mean Q^{-1} L^T W r (the Kalman-smoother
solution, which the paper notes is exact for linear Gaussian models).
"""
import numpy as np

K_LG = np.array([[-0.5, -2.0], [2.0, -0.5]])


def rk4_polys(Z):
    I2 = np.eye(Z.shape[0])
    Z2 = Z @ Z
    Z3 = Z2 @ Z
    Z4 = Z3 @ Z
    return I2 + Z + Z2 / 2 + Z3 / 6 + Z4 / 24, I2 + Z / 2 + Z2 / 6 + Z3 / 24


def system(M, dt, Rm, Rf, y, I, p_free=True, p_value=0.0, beta=1.0, scheme=0):
    """Return (L, r, w) with A(z) = 1/2 sum_k w_k (L z - r)_k^2.  z is the SoA
    path X[a*(M+1)+n] followed by p0 when the parameter is free.  scheme 1 is
    the trapezoid rule eps_{n+1} = x_{n+1} - x_n - dt/2 (F_{n+1} + F_n) with
    F_n = K x_n + (p0, I_n) (I_M := I_{M-1})."""
    if scheme == 1:
        return _trapezoid_system(M, dt, Rm, Rf, y, I, p_free, p_value, beta)
    D = 2
    T, S = rk4_polys(dt * K_LG)
    nx = D * (M + 1)
    nz = nx + (1 if p_free else 0)
    rows, rhs, wts = [], [], []
    for n in range(1, M + 1):
        row = np.zeros(nz)
        row[n] = 1.0
        rows.append(row); rhs.append(y[n]); wts.append(Rm)
    for n in range(M):
        for a in range(D):
            row = np.zeros(nz)
            row[a * (M + 1) + n + 1] += 1.0
            for b in range(D):
                row[b * (M + 1) + n] -= T[a, b]
            c = dt * S[a, 1] * I[n]
            if p_free:
                row[nx] -= dt * S[a, 0]
            else:
                c += dt * S[a, 0] * p_value
            rows.append(row); rhs.append(c); wts.append(beta * Rf[a])
    return np.array(rows), np.array(rhs), np.array(wts)


def action(L, r, w, z):
    e = L @ z - r
    return 0.5 * np.sum(w * e * e)


def posterior(L, r, w):
    Q = L.T @ (w[:, None] * L)
    cov = np.linalg.inv(Q)
    mean = cov @ (L.T @ (w * r))
    return mean, cov


def _trapezoid_system(M, dt, Rm, Rf, y, I, p_free, p_value, beta):
    D = 2
    K = K_LG
    nx = D * (M + 1)
    nz = nx + (1 if p_free else 0)
    drive = lambda n: I[n] if n < M else I[M - 1]
    rows, rhs, wts = [], [], []
    for n in range(1, M + 1):
        row = np.zeros(nz)
        row[n] = 1.0
        rows.append(row); rhs.append(y[n]); wts.append(Rm)
    for n in range(M):
        for a in range(D):
            row = np.zeros(nz)
            row[a * (M + 1) + n + 1] += 1.0
            row[a * (M + 1) + n] -= 1.0
            for b in range(D):
                row[b * (M + 1) + n + 1] -= 0.5 * dt * K[a, b]
                row[b * (M + 1) + n] -= 0.5 * dt * K[a, b]
            c = 0.0
            if a == 0:
                if p_free:
                    row[nx] -= dt          # dt/2 (p0 + p0)
                else:
                    c += dt * p_value
            else:
                c += 0.5 * dt * (drive(n + 1) + drive(n))
            rows.append(row); rhs.append(c); wts.append(beta * Rf[a])
    return np.array(rows), np.array(rhs), np.array(wts)
