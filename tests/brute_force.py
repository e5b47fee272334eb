"""A second, independent restatement of the method for tiny bodies: plain
Python floats, node by node and link by link, written from the paper's
equations and the readings listed in the oracle's header (not from the
oracle's code).  It pins the C oracle on 3 x 3 .. 6 x 5 bodies, where every
node is a boundary node or next to one, so the boundary rules of Sec. 6,
the ghost values of the differences and the corner links are all exercised.
A rectangular hole (removed nodes, faces with a constant traction each)
follows reading R16: a removed neighbour takes the linear ghost, a link
into the hole the anti-bounce-back rule with the crossed face's normal (a
link through the hole's corner: both faces, as at the body's corners).

Notation: direction k has integer offset E[k] and lattice velocity
C_k = c E[k]; weights 4/9, 1/9, 1/36; Cs^2 = mu / rho0 = c^2 / 3.
"""
import math

E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
W = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
OPPOSITE = [E.index((-a, -b)) for a, b in E]
PER, DIR, NEU = 0, 1, 2


class BruteForce:
    def __init__(self, prob, scheme):
        self.nx, self.ny = prob.nx, prob.ny
        self.lam, self.mu, self.rho0, self.omega = prob.lam, prob.mu, prob.rho0, prob.omega
        self.dX = prob.dX
        self.b = tuple(prob.body)
        self.edges = prob.edges
        # 0: source of time t in the moment; 1: predicted source; 2: source of
        # the u that j extrapolated to t + dt gives (reading R17)
        self.scheme = scheme
        self.Cs2 = self.mu / self.rho0
        self.dt = self.dX / math.sqrt(3.0 * self.Cs2)  # Sec. 7's time step
        self.c = self.dX / self.dt
        self.n = 0
        u0, v0 = prob.initial() if hasattr(prob, "initial") else (prob.u0, prob.v0)
        self.hole = getattr(prob, "hole", None)
        self.hole_T = getattr(prob, "hole_traction", None) or [(0.0, 0.0)] * 4
        nodes = [(x, y) for y in range(self.ny) for x in range(self.nx) if not self.removed((x, y))]
        self.nodes = nodes
        self.u = {p: [float(u0[p[1], p[0], 0]), float(u0[p[1], p[0], 1])] for p in nodes}
        self.j = {p: [self.rho0 * float(v0[p[1], p[0], 0]), self.rho0 * float(v0[p[1], p[0], 1])]
                  for p in nodes}
        # initialisation of Algorithm 1
        self.Q = {}
        H = {p: self.grad(self.u, p, 0.0) for p in nodes}
        self.Pstore = {}
        for p in nodes:
            self.Pstore[p] = (self.piola(H[p]), self.pbar(H[p]))
        self.r = {p: -self.rho0 * (H[p][0][0] + H[p][1][1]) for p in nodes}
        self.f = {p: self.feq(self.r[p], self.j[p], self.pbar(H[p])) for p in nodes}
        self.j_before = {p: list(self.j[p]) for p in nodes}  # j one step back (none yet: j(0))
        self.S = {p: self.source(p) for p in nodes}

    # ---------------------------------------------------------------- pieces
    def removed(self, p):
        if self.hole is None:
            return False
        x0, x1, y0, y1 = self.hole
        return x0 <= p[0] < x1 and y0 <= p[1] < y1

    def periodic(self, axis):
        return self.edges[2 * axis].kind == PER

    def C(self, k):
        return (self.c * E[k][0], self.c * E[k][1])

    def feq(self, r, j, Pb):
        out = []
        for k in range(9):
            ck = self.C(k)
            s = 0.0
            for a in range(2):
                for b in range(2):
                    delta = 1.0 if a == b else 0.0
                    s += (Pb[a][b] - r * self.Cs2 * delta) * (ck[a] * ck[b] - self.Cs2 * delta)
            out.append(W[k] * (r + (ck[0] * j[0] + ck[1] * j[1]) / self.Cs2 + s / (2 * self.Cs2 ** 2)))
        return out

    def piola(self, H):
        F = [[1 + H[0][0], H[0][1]], [H[1][0], 1 + H[1][1]]]
        J = F[0][0] * F[1][1] - F[0][1] * F[1][0]
        FinvT = [[F[1][1] / J, -F[1][0] / J], [-F[0][1] / J, F[0][0] / J]]
        return [[self.mu * (F[a][b] - FinvT[a][b]) + 0.5 * self.lam * (J * J - 1) * FinvT[a][b] for b in range(2)]
                for a in range(2)]

    def pbar(self, H):
        tr = H[0][0] + H[1][1]
        return [[-self.mu * (H[a][b] + H[b][a] + (tr if a == b else 0.0)) for b in range(2)] for a in range(2)]

    def ustar(self, e, t):
        E_ = self.edges[e]
        return [E_.value[a] + E_.rate[a] * t for a in range(2)]

    def tstar(self, e, t):
        E_ = self.edges[e]
        t_on, t_ramp, t_off = E_.times
        if t < t_on or t >= t_off:
            s = 0.0
        elif t_ramp > 0:
            s = min(1.0, (t - t_on) / t_ramp)
        else:
            s = 1.0
        return [E_.value[a] + (E_.rate[a] - E_.value[a]) * s for a in range(2)]

    def neighbour(self, field, p, axis, side, t, extrapolate_only):
        """field at p + side along axis; beyond a bounded edge the ghost value
        (Dirichlet: 2 u*(t) - u_edge for u; otherwise the linear extrapolation
        2 v0 - v1 from the edge node and the node behind it)."""
        x, y = p
        step = (side, 0) if axis == 0 else (0, side)
        if self.removed((x + step[0], y + step[1])):
            # across a face of the hole: the linear ghost from p and the node
            # behind it
            vals = [field[(x - m * step[0], y - m * step[1])] for m in range(2)]
            if isinstance(vals[0], float):
                return 2 * vals[0] - vals[1]
            return [2 * vals[0][a] - vals[1][a] for a in range(len(vals[0]))]
        n = self.nx if axis == 0 else self.ny
        k = (x if axis == 0 else y) + side
        if 0 <= k < n or self.periodic(axis):
            k %= n
            q = (k, y) if axis == 0 else (x, k)
            return list(field[q]) if not isinstance(field[q], float) else field[q]
        edge = 2 * axis + (0 if side < 0 else 1)
        k0 = 0 if side < 0 else n - 1
        inward = 1 if side < 0 else -1
        pts = [(k0 + m * inward) for m in range(2)]
        vals = [field[(kk, y) if axis == 0 else (x, kk)] for kk in pts]
        if not extrapolate_only and self.edges[edge].kind == DIR:
            us = self.ustar(edge, t)
            return [2 * us[a] - vals[0][a] for a in range(2)]
        if isinstance(vals[0], float):
            return 2 * vals[0] - vals[1]
        return [2 * vals[0][a] - vals[1][a] for a in range(len(vals[0]))]

    def grad(self, U, p, t):
        H = [[0.0, 0.0], [0.0, 0.0]]
        for axis in range(2):
            hi = self.neighbour(U, p, axis, +1, t, False)
            lo = self.neighbour(U, p, axis, -1, t, False)
            for a in range(2):
                H[a][axis] = (hi[a] - lo[a]) / (2 * self.dX)
        return H

    def source(self, p):
        """1S = rho0 b + Div(P + Pbar), central differences, linear ghosts."""
        Qf = {q: [self.Pstore[q][0][a][b] + self.Pstore[q][1][a][b] for a in range(2) for b in range(2)]
              for q in self.nodes}
        out = []
        for a in range(2):
            d = 0.0
            for axis in range(2):
                hi = self.neighbour(Qf, p, axis, +1, 0.0, True)
                lo = self.neighbour(Qf, p, axis, -1, 0.0, True)
                d += (hi[2 * a + axis] - lo[2 * a + axis]) / (2 * self.dX)
            out.append(self.rho0 * self.b[a] + d)
        return out

    def wall_rule(self, p, k, crossed, fcol, t):
        """f_opp(k) at p after a link k that leaves the body through the
        bounded edges in `crossed` (Eqs. bbcon, abbcon of Sec. 6)."""
        ck = self.C(k)
        dirs = [e for e in crossed if self.edges[e].kind == DIR]
        if dirs:
            js = [sum(self.rho0 * self.edges[e].rate[a] for e in dirs) / len(dirs) for a in range(2)]
            return fcol[k] - 2 * W[k] * (ck[0] * js[0] + ck[1] * js[1]) / self.Cs2
        sx = sy = 0
        for e in crossed:
            if e in (0, 1):
                sx = -1 if e == 0 else 1
            else:
                sy = -1 if e == 2 else 1
        norm = math.hypot(sx, sy)
        N = (sx / norm, sy / norm)
        T = [sum(self.tstar(e, t)[a] for e in crossed) / norm for a in range(2)]
        return self.anti_bounce(p, k, N, T, fcol)

    def hole_rule(self, p, k, fcol):
        """f_opp(k) at p after a link k that enters the hole: anti-bounce-back
        across the face(s) it crosses (the hole's corner: both faces)."""
        ex, ey = E[k]
        faces = []
        if ex and self.removed((p[0] + ex, p[1])):
            faces.append((0, ex))
        if ey and self.removed((p[0], p[1] + ey)):
            faces.append((1, ey))
        if not faces:
            faces = [(0, ex), (1, ey)]
        s = [0, 0]
        T = [0.0, 0.0]
        for axis, sign in faces:
            s[axis] = sign
            face = 2 * axis + (0 if sign > 0 else 1)  # faces at x0, x1, y0, y1
            T = [T[a] + self.hole_T[face][a] for a in range(2)]
        norm = math.hypot(s[0], s[1])
        return self.anti_bounce(p, k, (s[0] / norm, s[1] / norm), [T[a] / norm for a in range(2)], fcol)

    def anti_bounce(self, p, k, N, T, fcol):
        ck = self.C(k)
        fw = self.f[p]  # wall values: the edge node at time t
        rw = sum(fw)
        Pf = [[sum(self.C(i)[a] * self.C(i)[b] * fw[i] for i in range(9)) for b in range(2)] for a in range(2)]
        P, Pb = self.Pstore[p]
        g = [-T[a] + sum((P[a][b] + Pb[a][b]) * N[b] for b in range(2)) for a in range(2)]
        tv = (-N[1], N[0])
        pnn = N[0] * g[0] + N[1] * g[1]
        pnt = tv[0] * g[0] + tv[1] * g[1]
        ptt = sum(tv[a] * Pf[a][b] * tv[b] for a in range(2) for b in range(2))
        Ps = [[pnn * N[a] * N[b] + pnt * (N[a] * tv[b] + tv[a] * N[b]) + ptt * tv[a] * tv[b] for b in range(2)]
              for a in range(2)]
        s = 0.0
        for a in range(2):
            for b in range(2):
                delta = 1.0 if a == b else 0.0
                s += (Ps[a][b] - rw * self.Cs2 * delta) * (ck[a] * ck[b] - self.Cs2 * delta)
        return -fcol[k] + 2 * W[k] * (rw + s / (2 * self.Cs2 ** 2))

    # ---------------------------------------------------------------- step
    def step(self):
        t, t1, dt = self.n * self.dt, (self.n + 1) * self.dt, self.dt
        fcol = {}
        for p in self.nodes:
            fp = self.f[p]
            Pf = [[sum(self.C(i)[a] * self.C(i)[b] * fp[i] for i in range(9)) for b in range(2)] for a in range(2)]
            fe = self.feq(self.r[p], self.j[p], Pf)
            S = self.S[p]
            fcol[p] = [fp[k] - self.omega * (fp[k] - fe[k])
                       + dt * (1 - 0.5 * self.omega) * W[k] * (self.C(k)[0] * S[0] + self.C(k)[1] * S[1]) / self.Cs2
                       for k in range(9)]
        new = {p: [None] * 9 for p in self.nodes}
        for p in self.nodes:
            for k in range(9):
                x, y = p[0] + E[k][0], p[1] + E[k][1]
                crossed = []
                if not 0 <= x < self.nx:
                    if self.periodic(0):
                        x %= self.nx
                    else:
                        crossed.append(0 if x < 0 else 1)
                if not 0 <= y < self.ny:
                    if self.periodic(1):
                        y %= self.ny
                    else:
                        crossed.append(2 if y < 0 else 3)
                if self.removed((x, y)):
                    new[p][OPPOSITE[k]] = self.hole_rule(p, k, fcol[p])
                elif crossed:
                    new[p][OPPOSITE[k]] = self.wall_rule(p, k, crossed, fcol[p], t)
                else:
                    new[(x, y)][k] = fcol[p][k]
        self.f = new
        m = {}
        for p in self.nodes:
            fp = self.f[p]
            self.r[p] = sum(fp)
            m[p] = [sum(self.C(k)[a] * fp[k] for k in range(9)) for a in range(2)]

        def stresses(U, tt):
            for p in self.nodes:
                H = self.grad(U, p, tt)
                self.Pstore[p] = (self.piola(H), self.pbar(H))

        def trapezoid(jn):
            return {p: [self.u[p][a] + 0.5 * dt * (jn[p][a] + self.j[p][a]) / self.rho0 for a in range(2)]
                    for p in self.nodes}

        def moment(S):
            return {p: [m[p][a] + 0.5 * dt * S[p][a] for a in range(2)] for p in self.nodes}

        scheme = self.scheme
        if scheme == 0:
            jn = moment(self.S)
            self.u = trapezoid(jn)
            stresses(self.u, t1)
            self.S = {p: self.source(p) for p in self.nodes}
        elif scheme == 3:
            # not a scheme of the library: the fully implicit moment the
            # paper's Sec. 5 names as the ideal (the source of u(t + dt)
            # itself), by fixed-point iteration
            S = self.S
            for _ in range(60):
                jn = moment(S)
                stresses(trapezoid(jn), t1)
                S_next = {p: self.source(p) for p in self.nodes}
                change = max(abs(S_next[p][a] - S[p][a]) for p in self.nodes for a in range(2))
                S = S_next
                if change == 0.0:
                    break
            self.S = S
            jn = moment(S)
            self.u = trapezoid(jn)
        else:
            if scheme == 2:
                # j at t + dt on the line through j(t - dt) and j(t); u(t + dt)
                # by the trapezoid over [t, t + dt]
                ahead = {p: [2 * self.j[p][a] - self.j_before[p][a] for a in range(2)] for p in self.nodes}
            else:  # 1: the explicit j of this step
                ahead = moment(self.S)
            stresses(trapezoid(ahead), t1)
            self.S = {p: self.source(p) for p in self.nodes}
            jn = moment(self.S)
            self.u = trapezoid(jn)
        self.j_before = self.j
        self.j = jn
        self.n += 1

    def fields(self):
        import numpy as np

        u = np.zeros((self.ny, self.nx, 2))
        v = np.zeros((self.ny, self.nx, 2))
        r = np.zeros((self.ny, self.nx))
        for (x, y) in self.nodes:
            u[y, x] = self.u[(x, y)]
            v[y, x] = [self.j[(x, y)][a] / self.rho0 for a in range(2)]
            r[y, x] = self.r[(x, y)]
        return {"u": u, "v": v, "r": r}
