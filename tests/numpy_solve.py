"""A second FP64 statement of one MPPI solve, in NumPy, for tiny inputs.

TEST INFRASTRUCTURE ONLY: it exists to cross-check the C oracle
(oracle/mppi_oracle.c) on small cases (K <= 64, N <= 10).  It is written
independently from the same definitions -- the paper's equations and the
readings recorded for the places the paper leaves open -- and vectorised
over the samples instead of looping over them, so that a slip in either
implementation shows up as a disagreement:

  Eq. 3   samples U^m = clamp(U* + sigma z^m), z from Philox4x32-10
          (Salmon et al., SC'11) and Box-Muller, counter (m, k, iteration,
          block), key (seed, drone); the 5th (progress) normals of steps
          4j .. 4j+3 are the four outputs of block 1 at step 4j
  Eq. 2   quadrotor with collective thrust and body-rate command: p' = v,
          v' = (c/m) R(q) e_z - g e_z, q' = q (x) (0, w) / 2,
          w' = k_w (w_cmd - w) - J^-1 (w x J w); classical RK4, the input
          held over the step, q normalised after each step
  Eq. 6/7 gate progress with per-state gate switching, the temporal rule
          (time-aligned pass counts of the previous nominal) and the
          near-gate term on p_k
  Eq. 9   contouring with the progress state (theta, v_theta)
  Eq. 8   full-state tracking against x_ref(t0 + k dt)
  Eq. 4/5 exponential weights and the weighted update; warm start by a
          one-step shift.
Only the collective-thrust model without drag is covered.
"""
from __future__ import annotations

import numpy as np

M32 = np.uint64(0xFFFFFFFF)


# ---------------------------------------------------------------------------
# noise (Eq. 3)
# ---------------------------------------------------------------------------

def philox(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 on arrays of counters; returns the four output words."""
    c = [np.asarray(v, np.uint64) & M32 for v in (c0, c1, c2, c3)]
    k0, k1 = np.uint64(k0) & M32, np.uint64(k1) & M32
    for rnd in range(10):
        if rnd:
            k0 = (k0 + np.uint64(0x9E3779B9)) & M32
            k1 = (k1 + np.uint64(0xBB67AE85)) & M32
        p0 = np.uint64(0xD2511F53) * c[0]
        p1 = np.uint64(0xCD9E8D57) * c[2]
        c = [((p1 >> np.uint64(32)) ^ c[1] ^ k0) & M32, p1 & M32, ((p0 >> np.uint64(32)) ^ c[3] ^ k1) & M32,
             p0 & M32]
    return c


def unit(x):
    """24 random bits to a uniform in (0, 1]."""
    return ((x >> np.uint64(8)).astype(np.float64) + 1.0) / 16777216.0


def normals(seed, drone, m, k, it, blk):
    """[len(m)][4] standard normals of samples m at step k."""
    m = np.asarray(m, np.uint64)
    x = philox(m, np.full_like(m, k), np.full_like(m, it), np.full_like(m, blk), seed, drone)
    out = []
    for a, b in ((x[0], x[1]), (x[2], x[3])):
        r = np.sqrt(-2.0 * np.log(unit(a)))
        ang = 2.0 * np.pi * unit(b)
        out += [r * np.cos(ang), r * np.sin(ang)]
    return np.stack(out, axis=1)


# ---------------------------------------------------------------------------
# model (Eq. 2)
# ---------------------------------------------------------------------------

def deriv(mc, x, u):
    """State derivative for rows of x [B][13] and inputs u [B][4]."""
    p, v, q, w = x[:, 0:3], x[:, 3:6], x[:, 6:10], x[:, 10:13]
    qw, qx, qy, qz = q.T
    bz = np.stack([2 * (qx * qz + qw * qy), 2 * (qy * qz - qw * qx), 1 - 2 * (qx * qx + qy * qy)], axis=1)
    acc = (u[:, 0] / mc.mass)[:, None] * bz
    acc[:, 2] -= mc.gravity
    wx, wy, wz = w.T
    dq = 0.5 * np.stack([-(qx * wx + qy * wy + qz * wz), qw * wx + qy * wz - qz * wy, qw * wy + qz * wx - qx * wz,
                         qw * wz + qx * wy - qy * wx], axis=1)
    Jd = np.asarray(mc.inertia, np.float64)
    Jw = w * Jd
    gyro = np.cross(w, Jw)
    dw = mc.k_omega * (u[:, 1:4] - w) - gyro / Jd
    return np.concatenate([v, acc, dq, dw], axis=1)


def rk4(mc, x, u, h):
    k1 = deriv(mc, x, u)
    k2 = deriv(mc, x + 0.5 * h * k1, u)
    k3 = deriv(mc, x + 0.5 * h * k2, u)
    k4 = deriv(mc, x + h * k3, u)
    xn = x + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    xn[:, 6:10] /= np.linalg.norm(xn[:, 6:10], axis=1, keepdims=True)
    return xn


def penalty(mc, sc, x):
    over = np.maximum(np.abs(x[:, 10:13]) - mc.omega_max, 0.0)
    low = np.maximum(mc.z_floor - x[:, 2], 0.0)
    return sc.w_limit * (np.sum(over * over, axis=1) + low * low)


# ---------------------------------------------------------------------------
# track lookups (inputs of Algorithm 1)
# ---------------------------------------------------------------------------

def gate_rows(track, idx):
    n = track.gates.shape[0]
    idx = np.asarray(idx)
    i = np.mod(idx, n) if track.closed else np.minimum(idx, n - 1)
    return np.asarray(track.gates, np.float64)[i]


def path_at(track, theta):
    """Position and unit tangent at arc length theta [B] (closed path)."""
    S, L = track.path.shape[0], track.L
    ds = L / S
    th = np.mod(theta, L)
    s = th / ds
    j = np.floor(s).astype(np.int64)
    f = s - j
    over = j >= S
    j[over], f[over] = S - 1, 1.0
    a = np.asarray(track.path, np.float64)[j]
    b = np.asarray(track.path, np.float64)[(j + 1) % S]
    P = a[:, 0:3] + f[:, None] * (b[:, 0:3] - a[:, 0:3])
    T = a[:, 3:6] + f[:, None] * (b[:, 3:6] - a[:, 3:6])
    return P, T / np.linalg.norm(T, axis=1, keepdims=True)


def project(track, p, jlo, jhi):
    """Arc length of the closest point of the node segments jlo..jhi."""
    S, L = track.path.shape[0], track.L
    ds = L / S
    best, best_th = np.inf, 0.0
    path = np.asarray(track.path, np.float64)
    for jj in range(jlo, jhi + 1):
        j = jj % S
        a, b = path[j, 0:3], path[(j + 1) % S, 0:3]
        d = b - a
        t = min(max(np.dot(p - a, d) / np.dot(d, d), 0.0), 1.0)
        dist = np.sum((p - a - t * d) ** 2)
        if dist < best:
            best, best_th = dist, (j + t) * ds
    return best_th


def ref_at(track, t):
    ref = np.asarray(track.ref, np.float64)
    T = ref.shape[0]
    s = np.mod(t, T * track.dt_ref) / track.dt_ref
    i = int(np.floor(s))
    f = s - i
    if i >= T:
        i, f = T - 1, 1.0
    a, b = ref[i], ref[(i + 1) % T]
    x = a + f * (b - a)
    sg = -1.0 if np.dot(a[6:10], b[6:10]) < 0 else 1.0
    q = (1 - f) * a[6:10] + f * sg * b[6:10]
    x[6:10] = q / np.linalg.norm(q)
    return x


# ---------------------------------------------------------------------------
# one solve
# ---------------------------------------------------------------------------

class NumpyController:
    """Controller state carried between solves, as the oracle carries it."""

    def __init__(self, mc, sc, track):
        self.mc, self.sc, self.track = mc, sc, track
        self.U = None          # nominal [N][5] (None: hover)
        self.it = 0
        self.gate = 0
        self.prev = None       # pass counts of the previous nominal, aligned to this solve
        self.prev_x0 = None
        self.theta = None
        self.v_theta = 0.0
        self.c_last = mc.mass * mc.gravity

    def _crossing(self, g, pa, pb):
        """Rows of pass tests of segments pa -> pb through gates g."""
        n = np.stack([np.cos(g[:, 3]), np.sin(g[:, 3]), np.zeros(len(g))], axis=1)
        lat_dir = np.stack([-np.sin(g[:, 3]), np.cos(g[:, 3]), np.zeros(len(g))], axis=1)
        sa = np.sum(n * (pa - g[:, 0:3]), axis=1)
        sb = np.sum(n * (pb - g[:, 0:3]), axis=1)
        front_to_back = (sa < 0) & (sb >= 0)
        a = np.where(front_to_back, sa / np.where(front_to_back, sa - sb, 1.0), 0.0)
        e = pa + a[:, None] * (pb - pa) - g[:, 0:3]
        lat = np.sum(lat_dir * e, axis=1)
        return front_to_back & (np.abs(lat) <= g[:, 4]) & (np.abs(e[:, 2]) <= g[:, 5])

    def _rollout(self, x0, Us, xref, theta0, vth0):
        """Costs, term magnitudes and pass bookkeeping of sequences Us [B][N][5]."""
        mc, sc, tr = self.mc, self.sc, self.track
        B, N = Us.shape[0], sc.N
        x = np.tile(x0, (B, 1))
        J, Jabs = np.zeros(B), np.zeros(B)
        gi = np.full(B, self.gate)
        passed, first = np.zeros(B, np.int64), np.full(B, -1)
        pc = np.zeros((B, N + 1), np.int64)
        g0 = gate_rows(tr, np.array([self.gate]))[0]
        theta, vth, cprev = np.full(B, theta0), np.full(B, vth0), np.full(B, self.c_last)
        hover = mc.mass * mc.gravity
        for k in range(N):
            u = Us[:, k, :]
            xn = rk4(mc, x, u[:, 0:4], sc.dt)
            pen = penalty(mc, sc, xn)
            if sc.objective == 0:
                g = gate_rows(tr, gi)
                dn = np.sum((xn[:, 0:3] - g[:, 0:3]) ** 2, axis=1)
                dp = np.sum((x[:, 0:3] - g[:, 0:3]) ** 2, axis=1)
                d0 = np.sum((x[:, 0:3] - g0[0:3]) ** 2, axis=1)
                near = np.where(np.sqrt(d0) < sc.r_near, sc.q_near * d0, 0.0)
                stage = dn - dp + near
                Jabs += dn + dp + np.abs(near)
                prev_k = 0 if self.prev is None else self.prev[min(k, len(self.prev) - 1)]
                ok_time = (sc.temporal_rule == 0) | (prev_k <= passed)
                done = (not tr.closed) & (gi >= tr.gates.shape[0])
                acc = self._crossing(g, x[:, 0:3], xn[:, 0:3]) & ok_time & ~done
                first = np.where(acc & (first < 0), k, first)
                passed += acc
                gi += acc
            elif sc.objective == 1:
                a = u[:, 4]
                v1 = np.clip(vth + a * sc.dt, 0.0, sc.v_theta_max)
                th1 = theta + 0.5 * (vth + v1) * sc.dt
                P, T = path_at(tr, th1)
                e = xn[:, 0:3] - P
                el = np.sum(e * T, axis=1)[:, None] * T
                ec = e - el
                lag = sc.q_lag * np.sum(el * el, axis=1)
                con = sc.q_cont * np.sum(ec * ec, axis=1)
                om = np.sum(np.asarray(sc.q_omega) * xn[:, 10:13] ** 2, axis=1)
                dv = sc.r_dv * a * a
                dT = sc.r_dthrust * (u[:, 0] - cprev) ** 2
                prog = sc.mu * v1
                stage = lag + con + om + dv + dT - prog
                Jabs += lag + con + om + dv + dT + np.abs(prog)
                cprev, theta, vth = u[:, 0], th1, v1
            else:
                stage = self._track_err(x, xref[k], sc.Q)
                du = u[:, 0:4].copy()
                du[:, 0] -= hover
                stage = stage + np.sum(np.asarray(sc.R) * du * du, axis=1)
                if k == N - 1:
                    stage = stage + self._track_err(xn, xref[N], sc.QN)
                Jabs += stage
            J += stage + pen
            Jabs += pen
            x = xn
            pc[:, k + 1] = passed
        return J, Jabs, passed, first, pc

    @staticmethod
    def _track_err(x, xr, W):
        sg = np.where(np.sum(x[:, 6:10] * xr[6:10], axis=1) < 0, -1.0, 1.0)
        r = np.tile(xr, (x.shape[0], 1))
        r[:, 6:10] *= sg[:, None]
        return np.sum(np.asarray(W) * (x - r) ** 2, axis=1)

    def solve(self, x0, t0):
        mc, sc, tr = self.mc, self.sc, self.track
        K, N = sc.K, sc.N
        x0 = np.asarray(x0, np.float64)
        nu = 5 if sc.objective == 1 else 4
        # the plant's own pass of the current gate since the last solve
        if sc.objective == 0 and self.prev_x0 is not None:
            g = gate_rows(tr, np.array([self.gate]))
            open_done = (not tr.closed) and self.gate >= tr.gates.shape[0]
            if not open_done and self._crossing(g, self.prev_x0[None, 0:3], x0[None, 0:3])[0]:
                self.gate += 1
                if self.prev is not None:
                    self.prev = np.maximum(self.prev - 1, 0)
        U = self.U if self.U is not None else np.tile([mc.mass * mc.gravity, 0, 0, 0, 0], (N, 1)).astype(float)
        # Eq. 3
        Z = np.zeros((K, N, 5))
        for k in range(N):
            Z[:, k, 0:4] = normals(sc.seed, sc.drone_id, np.arange(K), k, self.it, 0)
            if nu == 5:
                Z[:, k, 4] = normals(sc.seed, sc.drone_id, np.arange(K), k - k % 4, self.it, 1)[:, k % 4]
        Us = np.clip(U[None] + np.asarray(sc.sigma) * Z, np.asarray(mc.u_min), np.asarray(mc.u_max))
        Us[:, :, nu:] = 0.0
        theta0, vth0, xref = 0.0, 0.0, None
        if sc.objective == 1:
            S, ds = tr.path.shape[0], tr.L / tr.path.shape[0]
            if self.theta is None:
                theta0 = project(tr, x0[0:3], 0, S - 1)
            else:
                theta0 = project(tr, x0[0:3], int(np.floor((self.theta - sc.theta_back) / ds)),
                                 int(np.floor((self.theta + sc.theta_ahead) / ds)))
                vth0 = self.v_theta
        elif sc.objective == 2:
            xref = np.stack([ref_at(tr, t0 + k * sc.dt) for k in range(N + 1)])
        J, Jabs, npass, first, _ = self._rollout(x0, Us, xref, theta0, vth0)
        # Eq. 4 and Eq. 5
        w = np.exp(-(J - J.min()) / sc.lam)
        w /= w.sum()
        Unew = np.einsum("m,mkj->kj", w, Us)
        # pass counts along the new nominal (for the next solve's temporal rule)
        _, _, _, _, pc = self._rollout(x0, Unew[None], xref, theta0, vth0)
        # warm start and controller state
        self.U = np.vstack([Unew[1:], Unew[-1:]])
        self.prev = pc[0, 0:N].copy() if sc.temporal_rule == 2 else pc[0, 1:N + 1].copy()
        if sc.objective == 1:
            self.theta = theta0
            self.v_theta = float(np.clip(vth0 + Unew[0, 4] * sc.dt, 0.0, sc.v_theta_max))
        self.c_last = Unew[0, 0]
        self.prev_x0 = x0.copy()
        self.it += 1
        return {"J": J, "Jabs": Jabs, "w": w, "Unew": Unew, "u0": Unew[0], "npass": npass, "first_pass": first,
                "Us": Us}
