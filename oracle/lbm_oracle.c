/*
 * lbm_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the large-deformation Lagrangian
 * lattice Boltzmann method of Faust, Schlueter, Mueller & Mueller,
 * "A Lattice Boltzmann Method for nonlinear solid mechanics in the reference
 * configuration" (arXiv 2208.13769).  It is the reference the CUDA library is
 * checked against; only the test-suite, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * constant table with the CUDA library.
 *
 * Every per-node phase of Algorithm 1 is its own loop over materialised
 * arrays (f, f^col, r, j, u, P, Pbar, S), in the algorithm's order, with no
 * fusion.  Compile with -ffp-contract=off -fno-fast-math so that each reading
 * of the paper has exactly one result.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes of the repository):
 *   R1  C_s = sqrt(mu/rho0) equals the lattice sound speed c/sqrt(3), so
 *       dt = dX / (sqrt(3) C_s)  (Sec. 7 prints dt = 1.443e-2 at dX = 0.025 and
 *       7.217e-3 at dX = 0.0125 with C_s = 1).  Lower-case c_s in Sec. 5 = C_s.
 *   R2  The trapezoidal displacement update of Sec. 5 carries a factor dt:
 *       u += dt/(2 rho0) (j_new + j_old).
 *   R3  omega = dt/tau is an input (the paper never fixes tau).  With the
 *       other readings, the three runs of Sec. 7 complete at the paper's loads
 *       only for omega in about [1.92, 1.99] (at omega = 1 each blows up before
 *       t = 2.1); the workloads take omega = 1.95.
 *   R4  The Pbar that enters f^eq in the collision is the second moment of the
 *       streamed populations, sum_i C_i C_i f_i (Eq. moment with N = 2 and no
 *       second-order source, Sec. 3: the moments computed after streaming feed
 *       the next equilibrium).  Pbar(H) of Eq. (Plin) is used where the paper
 *       needs the constitutive part: in 1S (Eq. source1) and in the wall values
 *       of Sec. 6.  (Taking Pbar(H) in f^eq as well amplifies diagonal grid
 *       modes by ~1.4 per step for every material; the paper's own runs of
 *       several hundred steps rule that reading out.)
 *   R5  Nodes of a bounded axis sit at (k+1/2) dX; walls are half-way between
 *       the edge node and the missing ghost node.  Periodic axes wrap.
 *   R6  Central differences everywhere (Sec. 5), with ghost values at bounded
 *       edges: Dirichlet u_g = 2 u*(t) - u_0, Neumann u_g = 2 u_0 - u_1 (linear
 *       extrapolation); for Div(P + Pbar) the linear ghost 2 Q_0 - Q_1 on every
 *       bounded edge.  Both are exact for affine u (the patch tests).  With the
 *       quadratic extrapolation 3 v_0 - 3 v_1 + v_2 instead, the shear and
 *       tension blocks of Sec. 7 blow up at every omega.
 *   R7  "Extrapolated to the boundary" (Sec. 6) is taken at zeroth order: the
 *       wall values are those of the edge node at time t (the level of f^col):
 *       r^bd = sum_i f_i, the tangential entry of Pbar* from the populations'
 *       second moment sum_i C_i C_i f_i, and (P + Pbar)(H) of the node in the
 *       quasi-traction.  j* and T* are evaluated at t as well.  (Linear
 *       extrapolation from the inner neighbour, or Pbar(H) in the tangential
 *       entry, makes the rule amplify along-wall grid modes even at
 *       lambda = mu; with this choice the scheme is neutrally stable at
 *       lambda = mu for every boundary set.)
 *   R8  Pbar* of Sec. 6: in the frame (N, t) of the wall normal the first row
 *       and column hold the quasi-traction g = -T* + (P + Pbar)_w N, the
 *       tangential diagonal holds t.Pbar_w.t (Pbar_w from the populations,
 *       R7); rotated back to (x, y).
 *   R9  Eq. (abbcon)'s r^bd is used in both places (the algorithm's listing
 *       prints a plain r in the second one).
 *   R10 A diagonal link that leaves through two bounded edges at a corner:
 *       Dirichlet if either edge is Dirichlet (j* averaged when both are);
 *       otherwise anti-bounce-back with N = (N1 + N2)/sqrt(2), the node's wall
 *       values (R7), and T* = (T1 + T2)/sqrt(2), which is
 *       the traction a homogeneous stress with P N1 = T1, P N2 = T2 exerts on N.
 *   R11 "for i from 0 to 9" in the listing means the nine directions 0..8.
 *   R12 P = dW/dF = mu (F - F^-T) + (lambda/2)(J^2 - 1) F^-T for the plane-strain
 *       neo-Hooke energy of Sec. 7, with J - 1 formed from H without
 *       cancellation.
 *   R13 The loop runs exactly the requested number of steps; t_n = n dt.
 *   R14 Time level of 1S (Sec. 5).  Scheme 0 (EXPLICIT) is Algorithm 1: the
 *       time-t source enters both the collision and the moment.  Scheme 1
 *       (PREDICTOR) is the predictor-corrector the paper's footnote to Sec. 5
 *       offers: the explicit update gives a predicted u*(t+dt); the source
 *       evaluated from it, 1S(t+dt), replaces the time-t source in the moment
 *       (corrected j and u) and is the source of the next collision; stresses
 *       and wall values of the step are those of u*.  For Lame constants with
 *       lambda > mu the explicit scheme grows without bound; the predictor form
 *       is neutrally stable up to lambda = 4 mu (Poisson ratio 0.4).
 *   R15 Read-out stresses (P, Pbar, sigma, J) are evaluated from the read-out
 *       displacement u(t_n) by the same central differences and ghost rules.
 *   R16 A rectangular hole (the plate with a square hole of Sec. 7) removes the
 *       nodes x0 <= x < x1, y0 <= y < y1; its four faces lie half-way between
 *       the last node of the body and the first removed one (R5) and carry a
 *       constant traction each (zero: traction-free).  A face is a Neumann
 *       boundary: the linear ghost of R6 for Grad u and Div Q, and
 *       anti-bounce-back (R7, R8) with the face's outward normal for a link
 *       that enters the hole through it; a diagonal link that enters the hole
 *       through its corner takes N = (N1 + N2)/sqrt(2) and
 *       T* = (T1 + T2)/sqrt(2), as at the body's corners (R10).
 *   R17 Scheme 2 (EXTRAPOLATED) is the variant Sec. 5 gives for an O(dt^3)
 *       error: j(t+dt) is extrapolated linearly from j(t) and j(t-dt), the
 *       trapezoidal rule turns it into u(t+dt), and 1S(t+dt) from that u
 *       enters the moment; as in R14, that source is also the next
 *       collision's, and the step's stresses and wall values are those of the
 *       extrapolated u.  The first step has no j(-dt): it takes j(-dt) = j(0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PERIODIC 0
#define ORC_DIRICHLET 1
#define ORC_NEUMANN 2
#define ORC_EXPLICIT 0
#define ORC_PREDICTOR 1
#define ORC_EXTRAPOLATED 2

/* Problem statement (Sec. 4 moment chain, Sec. 6 boundary conditions,
 * Sec. 7 material).  Edge order: 0 = x-, 1 = x+, 2 = y-, 3 = y+.
 * Dirichlet edge: value = u* at t = 0, rate = v*  (u*(t) = value + rate t,
 *                 j* = rho0 v*); times unused.
 * Neumann edge:   value = T0, rate = T1, times = {t_on, t_ramp, t_off}:
 *                 T*(t) = T0 before t_on and from t_off on; in between it
 *                 rises linearly from T0 to T1 over t_ramp (t_ramp = 0: a step).
 */
typedef struct {
    int32_t nx, ny;
    double dX, lambda, mu, rho0, omega;
    double body[2];
    int32_t kind[4];
    double value[4][2];
    double rate[4][2];
    double times[4][3];
    int32_t scheme; /* 0 = EXPLICIT (Algorithm 1), 1 = PREDICTOR (R14), 2 = EXTRAPOLATED (R17) */
    int32_t hole[4];   /* x0, x1, y0, y1 of a removed rectangle (R16); x0 >= x1: none */
    double hole_T[4][2]; /* traction on the hole's faces: x0 face, x1 face, y0 face, y1 face */
    /* Alternative readings of the open points above (zero everywhere selects
     * the readings R4, R6, R7 as listed), kept switchable so that the runs of
     * Sec. 7 can be repeated under each of them. */
    int32_t alt_feq_pbar; /* 1: f^eq takes Pbar(H) of Eq. (Plin), as the listing of Algorithm 1 prints it (R4) */
    int32_t alt_wall;     /* 1: wall values extrapolated linearly, (3 v_0 - v_1)/2, from the edge node
                             and its inner neighbour along the wall normal (R7) */
    int32_t alt_ghost_u;  /* 1: Neumann ghost of u quadratic, 3 u_0 - 3 u_1 + u_2 (R6) */
    int32_t alt_ghost_q;  /* 1: ghost of Q = P + Pbar quadratic; 2: constant, Q_0 (R6) */
    double mu_bar;        /* split stiffness: Pbar and C_s = sqrt(mu_bar/rho0) built with mu_bar,
                             the remainder of P in 1S (0: mu_bar = mu, the paper's split) */
} orc_problem;

typedef struct {
    orc_problem p;
    long n;
    double dt, c, Cs2;
    double C[9][2], w[9];
    int e[9][2];
    int opp[9];
    double *f[9], *fnew[9], *fcol[9];
    double *r, *j[2], *jnew[2], *jp[2], *m[2], *u[2], *us[2], *P[4], *Pb[4], *S[2];
    long step;
} orc_state;

/* ------------------------------------------------------------------ */
/* D2Q9 lattice (Sec. 3): e_0 = 0, four axis links, four diagonal links. */
static const int E9[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                             {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
static const int OPP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

static void lattice(double c, double C[9][2], double w[9], int e[9][2], int opp[9]) {
    for (int i = 0; i < 9; i++) {
        e[i][0] = E9[i][0];
        e[i][1] = E9[i][1];
        C[i][0] = c * E9[i][0];
        C[i][1] = c * E9[i][1];
        opp[i] = OPP9[i];
        int len2 = E9[i][0] * E9[i][0] + E9[i][1] * E9[i][1];
        w[i] = (len2 == 0) ? 4.0 / 9.0 : (len2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
}

/* Reading R1: C_s = sqrt(mu/rho0); dt = dX/(sqrt(3) C_s); c = dX/dt. */
void orc_time_step(double dX, double mu, double rho0, double* dt, double* c, double* Cs2) {
    double Cs = sqrt(mu / rho0);
    *dt = dX / (sqrt(3.0) * Cs);
    *c = dX / *dt;
    *Cs2 = Cs * Cs;
}

/* Equilibrium of Sec. 5 (Murthy et al. form):
 * f_i^eq = w_i ( r + C_i.j / C_s^2
 *               + (Pbar - r C_s^2 I) : (C_i C_i - C_s^2 I) / (2 C_s^4) ).
 * Pbar is a full 2x2 (row-major) array. */
static void feq_lat(const double C[9][2], const double w[9], double Cs2, double r,
                    const double j[2], const double Pb[4], double out[9]) {
    for (int i = 0; i < 9; i++) {
        double cj = C[i][0] * j[0] + C[i][1] * j[1];
        double contr = 0.0;
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                double d = (a == b) ? 1.0 : 0.0;
                contr += (Pb[2 * a + b] - r * Cs2 * d) * (C[i][a] * C[i][b] - Cs2 * d);
            }
        out[i] = w[i] * (r + cj / Cs2 + contr / (2.0 * Cs2 * Cs2));
    }
}

/* Source populations, Eq. (source): psi_i = w_i C_i . S / C_s^2. */
static void psi_lat(const double C[9][2], const double w[9], double Cs2, const double S[2],
                    double out[9]) {
    for (int i = 0; i < 9; i++) out[i] = w[i] * (C[i][0] * S[0] + C[i][1] * S[1]) / Cs2;
}

/* Poisson stress, Eq. (Plin): Pbar = -mu (H + H^T + tr(H) I). */
void orc_poisson_stress(const double H[4], double mu, double Pb[4]) {
    double tr = H[0] + H[3];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            Pb[2 * a + b] = -mu * (H[2 * a + b] + H[2 * b + a] + (a == b ? tr : 0.0));
}

/* Reading R12: first Piola-Kirchhoff stress of the plane-strain neo-Hooke
 * energy W of Sec. 7.  F = I + H, J - 1 = H11 + H22 + H11 H22 - H12 H21,
 * F^-T = (1/J) [[F22, -F21], [-F12, F11]].  Returns J. */
double orc_piola(const double H[4], double lambda, double mu, double P[4]) {
    double F[4] = {1.0 + H[0], H[1], H[2], 1.0 + H[3]};
    double Jm1 = H[0] + H[3] + H[0] * H[3] - H[1] * H[2];
    double J = 1.0 + Jm1;
    double FiT[4] = {F[3] / J, -F[2] / J, -F[1] / J, F[0] / J};
    double J2m1 = Jm1 * (2.0 + Jm1);
    for (int k = 0; k < 4; k++) P[k] = mu * (F[k] - FiT[k]) + 0.5 * lambda * J2m1 * FiT[k];
    return J;
}

/* Strain energy density of Sec. 7:
 * W = mu/2 (I_C - 2) + lambda/4 (J^2 - 1) - lambda/2 ln J - mu ln J,
 * I_C = tr(F^T F). */
double orc_strain_energy(const double H[4], double lambda, double mu) {
    double F[4] = {1.0 + H[0], H[1], H[2], 1.0 + H[3]};
    double IC = F[0] * F[0] + F[1] * F[1] + F[2] * F[2] + F[3] * F[3];
    double Jm1 = H[0] + H[3] + H[0] * H[3] - H[1] * H[2];
    double J = 1.0 + Jm1;
    double lnJ = log1p(Jm1);
    return 0.5 * mu * (IC - 2.0) + 0.25 * lambda * (J * J - 1.0) - 0.5 * lambda * lnJ - mu * lnJ;
}

/* Single-node helpers exported for the unit pins. */
void orc_feq(double c, double Cs2, double r, const double j[2], const double Pb[4], double out[9]) {
    double C[9][2], w[9];
    int e[9][2], opp[9];
    lattice(c, C, w, e, opp);
    feq_lat(C, w, Cs2, r, j, Pb, out);
}

void orc_psi(double c, double Cs2, const double S[2], double out[9]) {
    double C[9][2], w[9];
    int e[9][2], opp[9];
    lattice(c, C, w, e, opp);
    psi_lat(C, w, Cs2, S, out);
}

void orc_lattice(double c, double C[18], double w[9], int32_t opp[9]) {
    double CC[9][2];
    int e[9][2], o[9];
    lattice(c, CC, w, e, o);
    for (int i = 0; i < 9; i++) {
        C[2 * i] = CC[i][0];
        C[2 * i + 1] = CC[i][1];
        opp[i] = o[i];
    }
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Boundary data as functions of time (Sec. 6 and the problem statement). */

static void ustar(const orc_problem* p, int edge, double t, double out[2]) {
    for (int a = 0; a < 2; a++) out[a] = p->value[edge][a] + p->rate[edge][a] * t;
}

static void jstar(const orc_problem* p, int edge, double out[2]) {
    for (int a = 0; a < 2; a++) out[a] = p->rho0 * p->rate[edge][a];
}

static void tstar(const orc_problem* p, int edge, double t, double out[2]) {
    double t_on = p->times[edge][0], t_ramp = p->times[edge][1], t_off = p->times[edge][2];
    double s;
    if (t < t_on || t >= t_off)
        s = 0.0;
    else if (t_ramp > 0.0)
        s = fmin(1.0, (t - t_on) / t_ramp);
    else
        s = 1.0;
    for (int a = 0; a < 2; a++) out[a] = p->value[edge][a] + (p->rate[edge][a] - p->value[edge][a]) * s;
}

static inline long IDX(const orc_state* s, int x, int y) { return (long)y * s->p.nx + x; }

static int axis_periodic(const orc_state* s, int axis) { return s->p.kind[2 * axis] == ORC_PERIODIC; }

static int wrap(int k, int n) { return ((k % n) + n) % n; }

static int has_hole(const orc_problem* p) { return p->hole[0] < p->hole[1] && p->hole[2] < p->hole[3]; }

/* The modulus of the linear split Pbar (Eq. Plin) and of C_s: mu, or mu_bar
 * for the split-stiffness variant. */
static double split_mu(const orc_problem* p) { return p->mu_bar > 0.0 ? p->mu_bar : p->mu; }

/* Ghost value one node outside a traction-free or loaded edge from the edge
 * node v0 and its inner neighbours v1, v2 (R6): linear extrapolation, or the
 * quadratic / constant alternatives. */
static double ghost_extrap(int alt, double v0, double v1, double v2) {
    if (alt == 1) return 3.0 * v0 - 3.0 * v1 + v2;
    if (alt == 2) return v0;
    return 2.0 * v0 - v1;
}

/* (x, y) is a removed node of the hole (R16). */
static int in_hole(const orc_state* s, int x, int y) {
    const int32_t* h = s->p.hole;
    return h[0] < h[1] && x >= h[0] && x < h[1] && y >= h[2] && y < h[3];
}

/* Displacement at (x, y), which may lie one node outside along one axis
 * (reading R6). */
static double u_at(const orc_state* s, double* const U[2], int x, int y, int a, double t) {
    int nx = s->p.nx, ny = s->p.ny;
    if (x >= 0 && x < nx && y >= 0 && y < ny) return U[a][IDX(s, x, y)];
    int axis = (x < 0 || x >= nx) ? 0 : 1;
    int k = axis == 0 ? x : y, n = axis == 0 ? nx : ny;
    if (axis_periodic(s, axis)) {
        int kw = wrap(k, n);
        return axis == 0 ? U[a][IDX(s, kw, y)] : U[a][IDX(s, x, kw)];
    }
    int edge = 2 * axis + (k < 0 ? 0 : 1);
    int k0 = k < 0 ? 0 : n - 1, step = k < 0 ? 1 : -1;
    double v0, v1, v2;
    if (axis == 0) {
        v0 = U[a][IDX(s, k0, y)];
        v1 = U[a][IDX(s, k0 + step, y)];
        v2 = U[a][IDX(s, k0 + 2 * step, y)];
    } else {
        v0 = U[a][IDX(s, x, k0)];
        v1 = U[a][IDX(s, x, k0 + step)];
        v2 = U[a][IDX(s, x, k0 + 2 * step)];
    }
    if (s->p.kind[edge] == ORC_DIRICHLET) {
        double ub[2];
        ustar(&s->p, edge, t, ub);
        return 2.0 * ub[a] - v0;
    }
    return ghost_extrap(s->p.alt_ghost_u, v0, v1, v2);
}

/* Q = P + Pbar component k at (x, y), possibly one node outside along one
 * axis: periodic wrap or the ghost of reading R6. */
static double q_at(const orc_state* s, int x, int y, int k) {
    int nx = s->p.nx, ny = s->p.ny;
    if (x >= 0 && x < nx && y >= 0 && y < ny) {
        long id = IDX(s, x, y);
        return s->P[k][id] + s->Pb[k][id];
    }
    int axis = (x < 0 || x >= nx) ? 0 : 1;
    int kk = axis == 0 ? x : y, n = axis == 0 ? nx : ny;
    if (axis_periodic(s, axis)) {
        int kw = wrap(kk, n);
        return axis == 0 ? q_at(s, kw, y, k) : q_at(s, x, kw, k);
    }
    int k0 = kk < 0 ? 0 : n - 1, step = kk < 0 ? 1 : -1;
    double v0, v1, v2;
    if (axis == 0) {
        v0 = q_at(s, k0, y, k);
        v1 = q_at(s, k0 + step, y, k);
        v2 = q_at(s, k0 + 2 * step, y, k);
    } else {
        v0 = q_at(s, x, k0, k);
        v1 = q_at(s, x, k0 + step, k);
        v2 = q_at(s, x, k0 + 2 * step, k);
    }
    return ghost_extrap(s->p.alt_ghost_q, v0, v1, v2);
}

/* Eq. (defgrad) with central differences: H_ab = d_b u_a. */
/* Displacement at the neighbour (x + dx, y + dy) of the body node (x, y):
 * across a hole face the hole's ghost (R16), else u_at. */
static double u_nb(const orc_state* s, double* const U[2], int x, int y, int dx, int dy, int a, double t) {
    if (in_hole(s, x + dx, y + dy)) /* the hole's ghost (R16): as at a traction-free edge */
        return ghost_extrap(s->p.alt_ghost_u, U[a][IDX(s, x, y)], U[a][IDX(s, x - dx, y - dy)],
                            U[a][IDX(s, x - 2 * dx, y - 2 * dy)]);
    return u_at(s, U, x + dx, y + dy, a, t);
}

static void grad_u(const orc_state* s, double* const U[2], int x, int y, double t, double H[4]) {
    double h2 = 2.0 * s->p.dX;
    for (int a = 0; a < 2; a++) {
        H[2 * a + 0] = (u_nb(s, U, x, y, 1, 0, a, t) - u_nb(s, U, x, y, -1, 0, a, t)) / h2;
        H[2 * a + 1] = (u_nb(s, U, x, y, 0, 1, a, t) - u_nb(s, U, x, y, 0, -1, a, t)) / h2;
    }
}

/* H, P and Pbar at every node from the displacement field U (Alg. 1,
 * update step): U = u for the explicit scheme, U = u* for the predictor. */
static void update_stress(orc_state* s, double* const U[2], double t) {
    int nx = s->p.nx, ny = s->p.ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            if (in_hole(s, x, y)) continue; /* removed nodes keep zero stresses */
            double H[4], P[4], Pb[4];
            grad_u(s, U, x, y, t, H);
            orc_piola(H, s->p.lambda, s->p.mu, P);
            orc_poisson_stress(H, split_mu(&s->p), Pb);
            long id = IDX(s, x, y);
            for (int k = 0; k < 4; k++) {
                s->P[k][id] = P[k];
                s->Pb[k][id] = Pb[k];
            }
        }
}

/* Q component k at the neighbour (x + dx, y + dy) of the body node (x, y):
 * across a hole face the hole's ghost (R16), else q_at. */
static double q_nb(const orc_state* s, int x, int y, int dx, int dy, int k) {
    if (in_hole(s, x + dx, y + dy))
        return ghost_extrap(s->p.alt_ghost_q, q_at(s, x, y, k), q_at(s, x - dx, y - dy, k),
                            q_at(s, x - 2 * dx, y - 2 * dy, k));
    return q_at(s, x + dx, y + dy, k);
}

/* Eq. (source1): 1S = rho0 b + Div(P + Pbar), central differences. */
static void compute_source(orc_state* s) {
    int nx = s->p.nx, ny = s->p.ny;
    double h2 = 2.0 * s->p.dX;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            long id = IDX(s, x, y);
            if (in_hole(s, x, y)) continue;
            for (int a = 0; a < 2; a++) {
                double d1 = (q_nb(s, x, y, 1, 0, 2 * a + 0) - q_nb(s, x, y, -1, 0, 2 * a + 0)) / h2;
                double d2 = (q_nb(s, x, y, 0, 1, 2 * a + 1) - q_nb(s, x, y, 0, -1, 2 * a + 1)) / h2;
                s->S[a][id] = s->p.rho0 * s->p.body[a] + (d1 + d2);
            }
        }
}

/* ------------------------------------------------------------------ */
static double abb_rule(const orc_state* s, int x, int y, int i, const double N[2], const double T[2], int ox,
                       int oy);

/* Boundary rules of Sec. 6 for the link i of node (x, y) that leaves the body.
 * Returns the value of f_{opp(i)}(X, t + dt).  ex/ey: the bounded edges the
 * link crosses (-1 if none).  Time-t data: f (streamed), f^col, P, Pbar. */
static double boundary_rule(const orc_state* s, int x, int y, int i, int ex, int ey, double t) {
    const orc_problem* p = &s->p;
    long id = IDX(s, x, y);
    double fc = s->fcol[i][id];
    int dirichlet = 0;
    double js[2] = {0.0, 0.0};
    int nd = 0;
    int edges[2] = {ex, ey};
    for (int k = 0; k < 2; k++) {
        if (edges[k] >= 0 && p->kind[edges[k]] == ORC_DIRICHLET) {
            double jj[2];
            jstar(p, edges[k], jj);
            js[0] += jj[0];
            js[1] += jj[1];
            nd++;
            dirichlet = 1;
        }
    }
    if (dirichlet) {
        /* Eq. (bbcon): bounce-back with the wall momentum j*. */
        js[0] /= nd;
        js[1] /= nd;
        double cj = s->C[i][0] * js[0] + s->C[i][1] * js[1];
        return fc - 2.0 / s->Cs2 * s->w[i] * cj;
    }
    /* Eq. (abbcon): anti-bounce-back with Pbar* from the traction T*. */
    int dx = 0, dy = 0; /* outward integer offset of the wall normal */
    double N[2], T[2] = {0.0, 0.0};
    if (ex >= 0) dx = (ex == 0) ? -1 : 1;
    if (ey >= 0) dy = (ey == 2) ? -1 : 1;
    double nlen = sqrt((double)(dx * dx + dy * dy));
    N[0] = dx / nlen;
    N[1] = dy / nlen;
    for (int k = 0; k < 2; k++) {
        if (edges[k] < 0) continue;
        double tt[2];
        tstar(p, edges[k], t, tt);
        T[0] += tt[0];
        T[1] += tt[1];
    }
    /* one edge: T = T*; corner: T = (T1 + T2)/sqrt(2) (reading R10) */
    T[0] /= nlen;
    T[1] /= nlen;
    return abb_rule(s, x, y, i, N, T, dx, dy);
}

/* Time-t values at node id that the anti-bounce-back rule needs at the wall:
 * r = sum_i f_i, Pf = sum_i C_i C_i f_i, and the stresses P, Pbar. */
static void wall_data(const orc_state* s, long id, double* rw, double Pfw[4], double Pw[4], double Pbw[4]) {
    *rw = 0.0;
    for (int k = 0; k < 4; k++) Pfw[k] = 0.0;
    for (int k = 0; k < 9; k++) {
        *rw += s->f[k][id];
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) Pfw[2 * a + b] += s->C[k][a] * s->C[k][b] * s->f[k][id];
    }
    for (int k = 0; k < 4; k++) {
        Pw[k] = s->P[k][id];
        Pbw[k] = s->Pb[k][id];
    }
}

/* Eq. (abbcon): anti-bounce-back for the link i of node (x, y) across a wall
 * of outward unit normal N carrying the traction T (time-t data); (ox, oy) is
 * the outward integer offset of the normal, (x - ox, y - oy) the node's inner
 * neighbour. */
static double abb_rule(const orc_state* s, int x, int y, int i, const double N[2], const double T[2], int ox,
                       int oy) {
    long id = IDX(s, x, y);
    double fc = s->fcol[i][id];
    /* wall values at time t: those of the edge node (reading R7), or the
     * linear extrapolation to the wall from it and its inner neighbour */
    double rw, Pfw[4], Pw[4], Pbw[4];
    wall_data(s, id, &rw, Pfw, Pw, Pbw);
    if (s->p.alt_wall == 1) {
        double r1, Pf1[4], P1[4], Pb1[4];
        wall_data(s, IDX(s, x - ox, y - oy), &r1, Pf1, P1, Pb1);
        rw = 0.5 * (3.0 * rw - r1);
        for (int k = 0; k < 4; k++) {
            Pfw[k] = 0.5 * (3.0 * Pfw[k] - Pf1[k]);
            Pw[k] = 0.5 * (3.0 * Pw[k] - P1[k]);
            Pbw[k] = 0.5 * (3.0 * Pbw[k] - Pb1[k]);
        }
    }
    /* quasi-traction g = -T* + (P + Pbar)_w N (Sec. 6) */
    double g[2];
    for (int a = 0; a < 2; a++)
        g[a] = -T[a] + (Pw[2 * a] + Pbw[2 * a]) * N[0] + (Pw[2 * a + 1] + Pbw[2 * a + 1]) * N[1];
    double tv[2] = {-N[1], N[0]};
    double Pnn = N[0] * g[0] + N[1] * g[1];
    double Pnt = tv[0] * g[0] + tv[1] * g[1];
    double Ptt = 0.0;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) Ptt += tv[a] * Pfw[2 * a + b] * tv[b];
    double Ps[4];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            Ps[2 * a + b] = Pnn * N[a] * N[b] + Pnt * (N[a] * tv[b] + tv[a] * N[b]) + Ptt * tv[a] * tv[b];
    double contr = 0.0;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
            double d = (a == b) ? 1.0 : 0.0;
            contr += (Ps[2 * a + b] - rw * s->Cs2 * d) * (s->C[i][a] * s->C[i][b] - s->Cs2 * d);
        }
    return -fc + 2.0 * s->w[i] * (rw + contr / (2.0 * s->Cs2 * s->Cs2));
}

/* ------------------------------------------------------------------ */

/* The link i of body node (x, y) enters the hole (R16): anti-bounce-back with
 * the normal and traction of the face it crosses, or of the hole's corner. */
static double hole_rule(const orc_state* s, int x, int y, int i) {
    int ex = s->e[i][0], ey = s->e[i][1];
    int cx = ex != 0 && in_hole(s, x + ex, y); /* crosses the face normal to x */
    int cy = ey != 0 && in_hole(s, x, y + ey); /* crosses the face normal to y */
    if (!cx && !cy) cx = cy = 1;              /* through the hole's corner */
    double N[2] = {cx ? (double)ex : 0.0, cy ? (double)ey : 0.0};
    double T[2] = {0.0, 0.0};
    /* faces: 0 at x0 (normal +x from the body), 1 at x1 (-x), 2 at y0 (+y), 3 at y1 (-y) */
    if (cx) {
        const double* tf = s->p.hole_T[ex > 0 ? 0 : 1];
        T[0] += tf[0];
        T[1] += tf[1];
    }
    if (cy) {
        const double* tf = s->p.hole_T[ey > 0 ? 2 : 3];
        T[0] += tf[0];
        T[1] += tf[1];
    }
    double nlen = sqrt(N[0] * N[0] + N[1] * N[1]);
    int ox = (int)N[0], oy = (int)N[1];
    N[0] /= nlen;
    N[1] /= nlen;
    T[0] /= nlen;
    T[1] /= nlen;
    return abb_rule(s, x, y, i, N, T, ox, oy);
}

static double* zalloc(long n) { return (double*)calloc((size_t)n, sizeof(double)); }

void orc_destroy(orc_state* s);

/* Validates the problem; returns 0 if usable. */
int orc_check(const orc_problem* p) {
    if (p->nx < 3 || p->ny < 3) return 1;
    if (!(p->dX > 0) || !(p->mu > 0) || !(p->rho0 > 0)) return 2;
    if (!(p->omega > 0) || !(p->omega < 2)) return 3;
    for (int axis = 0; axis < 2; axis++) {
        int a = p->kind[2 * axis], b = p->kind[2 * axis + 1];
        if (a < 0 || a > 2 || b < 0 || b > 2) return 5;
        if ((a == ORC_PERIODIC) != (b == ORC_PERIODIC)) return 4;
    }
    if (p->scheme != ORC_EXPLICIT && p->scheme != ORC_PREDICTOR && p->scheme != ORC_EXTRAPOLATED) return 6;
    if (p->alt_feq_pbar < 0 || p->alt_feq_pbar > 1 || p->alt_wall < 0 || p->alt_wall > 1 || p->alt_ghost_u < 0 ||
        p->alt_ghost_u > 1 || p->alt_ghost_q < 0 || p->alt_ghost_q > 2 || !(p->mu_bar >= 0.0))
        return 8;
    if (has_hole(p)) {
        /* at least 3 body nodes between the hole and each edge or seam */
        if (p->hole[0] < 3 || p->hole[1] > p->nx - 3 || p->hole[2] < 3 || p->hole[3] > p->ny - 3) return 7;
    }
    return 0;
}

/* Initialisation of Alg. 1: u = u0, H = Grad u0, P, Pbar, r = -rho0 Div u0,
 * j = rho0 v0, f_i = f_i^eq(r, j, Pbar(H)), and the source of the first
 * collision 1S(0).  u0, v0: [ny][nx][2]. */
orc_state* orc_create(const orc_problem* p, const double* u0, const double* v0) {
    if (orc_check(p) != 0) return NULL;
    orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
    s->p = *p;
    s->n = (long)p->nx * p->ny;
    orc_time_step(p->dX, split_mu(p), p->rho0, &s->dt, &s->c, &s->Cs2);
    lattice(s->c, s->C, s->w, s->e, s->opp);
    for (int i = 0; i < 9; i++) {
        s->f[i] = zalloc(s->n);
        s->fnew[i] = zalloc(s->n);
        s->fcol[i] = zalloc(s->n);
    }
    s->r = zalloc(s->n);
    for (int a = 0; a < 2; a++) {
        s->j[a] = zalloc(s->n);
        s->jnew[a] = zalloc(s->n);
        s->jp[a] = zalloc(s->n);
        s->m[a] = zalloc(s->n);
        s->u[a] = zalloc(s->n);
        s->us[a] = zalloc(s->n);
        s->S[a] = zalloc(s->n);
    }
    for (int k = 0; k < 4; k++) {
        s->P[k] = zalloc(s->n);
        s->Pb[k] = zalloc(s->n);
    }
    for (long id = 0; id < s->n; id++)
        for (int a = 0; a < 2; a++) {
            const int removed = in_hole(s, (int)(id % p->nx), (int)(id / p->nx));
            s->u[a][id] = u0 && !removed ? u0[2 * id + a] : 0.0;
            s->j[a][id] = p->rho0 * (v0 && !removed ? v0[2 * id + a] : 0.0);
            s->jp[a][id] = s->j[a][id]; /* R17: j(-dt) = j(0) */
        }
    update_stress(s, s->u, 0.0);
    int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            if (in_hole(s, x, y)) continue; /* removed nodes hold nothing */
            double H[4];
            grad_u(s, s->u, x, y, 0.0, H);
            long id = IDX(s, x, y);
            s->r[id] = -p->rho0 * (H[0] + H[3]);
            double jj[2] = {s->j[0][id], s->j[1][id]};
            double Pb[4] = {s->Pb[0][id], s->Pb[1][id], s->Pb[2][id], s->Pb[3][id]};
            double fe[9];
            feq_lat(s->C, s->w, s->Cs2, s->r[id], jj, Pb, fe);
            for (int i = 0; i < 9; i++) s->f[i][id] = fe[i];
        }
    compute_source(s);
    s->step = 0;
    return s;
}

/* One iteration of Alg. 1 from t = step*dt to t + dt.  On entry: f(t),
 * r(t), j(t), u(t), the stresses P, Pbar of the step's displacement and the
 * collision source S = 1S(t). */
static void step_once(orc_state* s) {
    const orc_problem* p = &s->p;
    int nx = p->nx, ny = p->ny;
    double t = s->step * s->dt;
    double t1 = (s->step + 1) * s->dt;
    double omega = p->omega, dt = s->dt;

    /* equilibrium (reading R4), source populations and collision (Eq. col) */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            long id = IDX(s, x, y);
            double jj[2] = {s->j[0][id], s->j[1][id]};
            double Pb[4] = {0.0, 0.0, 0.0, 0.0};
            if (p->alt_feq_pbar == 1) {
                for (int k = 0; k < 4; k++) Pb[k] = s->Pb[k][id];
            } else {
                for (int i = 0; i < 9; i++)
                    for (int a = 0; a < 2; a++)
                        for (int b = 0; b < 2; b++) Pb[2 * a + b] += s->C[i][a] * s->C[i][b] * s->f[i][id];
            }
            double Sv[2] = {s->S[0][id], s->S[1][id]};
            double fe[9], ps[9];
            feq_lat(s->C, s->w, s->Cs2, s->r[id], jj, Pb, fe);
            psi_lat(s->C, s->w, s->Cs2, Sv, ps);
            for (int i = 0; i < 9; i++) {
                double fi = s->f[i][id];
                s->fcol[i][id] = fi - omega * (fi - fe[i]) + dt * (1.0 - 0.5 * omega) * ps[i];
            }
        }

    /* streaming (Eq. stream) for links that stay inside the body, and the
     * boundary rules (Eq. bbcon, abbcon) for the links that leave it */
    int px = axis_periodic(s, 0), py = axis_periodic(s, 1);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            long id = IDX(s, x, y);
            if (in_hole(s, x, y)) continue;
            for (int i = 0; i < 9; i++) {
                int dx = x + s->e[i][0], dy = y + s->e[i][1];
                if (in_hole(s, dx, dy)) {
                    s->fnew[s->opp[i]][id] = hole_rule(s, x, y, i);
                    continue;
                }
                int ex = -1, ey = -1;
                if (dx < 0 || dx >= nx) {
                    if (px)
                        dx = wrap(dx, nx);
                    else
                        ex = dx < 0 ? 0 : 1;
                }
                if (dy < 0 || dy >= ny) {
                    if (py)
                        dy = wrap(dy, ny);
                    else
                        ey = dy < 0 ? 2 : 3;
                }
                if (ex < 0 && ey < 0) {
                    s->fnew[i][IDX(s, dx, dy)] = s->fcol[i][id];
                } else {
                    s->fnew[s->opp[i]][id] = boundary_rule(s, x, y, i, ex, ey, t);
                }
            }
        }
    for (int i = 0; i < 9; i++) {
        double* tmp = s->f[i];
        s->f[i] = s->fnew[i];
        s->fnew[i] = tmp;
    }

    /* moments (Eq. moment): r and the first-order sum without its source */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            long id = IDX(s, x, y);
            double r = 0.0, m0 = 0.0, m1 = 0.0;
            for (int i = 0; i < 9; i++) {
                r += s->f[i][id];
                m0 += s->C[i][0] * s->f[i][id];
                m1 += s->C[i][1] * s->f[i][id];
            }
            s->r[id] = r;
            s->m[0][id] = m0;
            s->m[1][id] = m1;
        }

    if (p->scheme == ORC_EXPLICIT) {
        /* Alg. 1: j(t+dt) with the time-t source, trapezoidal u (R2),
         * then H, P, Pbar and the next source from u(t+dt) */
#pragma omp parallel for schedule(static)
        for (long id = 0; id < s->n; id++)
            for (int a = 0; a < 2; a++) {
                double jn = s->m[a][id] + 0.5 * dt * s->S[a][id];
                s->u[a][id] = s->u[a][id] + dt / (2.0 * p->rho0) * (jn + s->j[a][id]);
                s->j[a][id] = jn;
            }
        update_stress(s, s->u, t1);
        compute_source(s);
    } else if (p->scheme == ORC_EXTRAPOLATED) {
        /* R17: j(t+dt) extrapolated linearly from j(t) and j(t-dt), the
         * trapezoidal u from it, and 1S(t+dt) from that u */
#pragma omp parallel for schedule(static)
        for (long id = 0; id < s->n; id++)
            for (int a = 0; a < 2; a++) {
                double je = 2.0 * s->j[a][id] - s->jp[a][id];
                s->us[a][id] = s->u[a][id] + dt / (2.0 * p->rho0) * (je + s->j[a][id]);
            }
        update_stress(s, s->us, t1);
        compute_source(s);
        /* j(t+dt) with 1S(t+dt), trapezoidal u (R2) */
#pragma omp parallel for schedule(static)
        for (long id = 0; id < s->n; id++)
            for (int a = 0; a < 2; a++) {
                double jn = s->m[a][id] + 0.5 * dt * s->S[a][id];
                s->u[a][id] = s->u[a][id] + dt / (2.0 * p->rho0) * (jn + s->j[a][id]);
                s->jp[a][id] = s->j[a][id];
                s->j[a][id] = jn;
            }
    } else {
        /* predictor (R14): explicit j* and u*(t+dt) */
#pragma omp parallel for schedule(static)
        for (long id = 0; id < s->n; id++)
            for (int a = 0; a < 2; a++) {
                double jp = s->m[a][id] + 0.5 * dt * s->S[a][id];
                s->us[a][id] = s->u[a][id] + dt / (2.0 * p->rho0) * (jp + s->j[a][id]);
            }
        /* H, P, Pbar of u*, and 1S(t+dt) from them */
        update_stress(s, s->us, t1);
        compute_source(s);
        /* corrector: j(t+dt) with 1S(t+dt), trapezoidal u (R2) */
#pragma omp parallel for schedule(static)
        for (long id = 0; id < s->n; id++)
            for (int a = 0; a < 2; a++) {
                double jn = s->m[a][id] + 0.5 * dt * s->S[a][id];
                s->u[a][id] = s->u[a][id] + dt / (2.0 * p->rho0) * (jn + s->j[a][id]);
                s->j[a][id] = jn;
            }
    }
    s->step++;
}

int orc_step(orc_state* s, long nsteps) {
    for (long k = 0; k < nsteps; k++) step_once(s);
    return 0;
}

double orc_time(const orc_state* s) { return s->step * s->dt; }
long orc_step_count(const orc_state* s) { return s->step; }
double orc_dt(const orc_state* s) { return s->dt; }

/* Read-out in row-major [ny][nx][ncomp]; any pointer may be NULL.
 * u (2), v = j/rho0 (2), P (4, row-major 2x2), Pbar (3: 11, 12, 22), r (1),
 * J (1), sigma = J^-1 P F^T (3: 11, 12, 22).  Stresses from u(t) (R15). */
void orc_read(const orc_state* s, double* u, double* v, double* P, double* Pb, double* r,
              double* J, double* sigma) {
    double t = s->step * s->dt;
    int nx = s->p.nx, ny = s->p.ny;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            long id = IDX(s, x, y);
            if (u)
                for (int a = 0; a < 2; a++) u[2 * id + a] = s->u[a][id];
            if (v)
                for (int a = 0; a < 2; a++) v[2 * id + a] = s->j[a][id] / s->p.rho0;
            if (r) r[id] = s->r[id];
            double H[4] = {0.0, 0.0, 0.0, 0.0}, PP[4], PB[4];
            if (!in_hole(s, x, y)) grad_u(s, s->u, x, y, t, H); /* removed nodes read as undeformed */
            double Jv = orc_piola(H, s->p.lambda, s->p.mu, PP);
            orc_poisson_stress(H, split_mu(&s->p), PB);
            if (P)
                for (int k = 0; k < 4; k++) P[4 * id + k] = PP[k];
            if (Pb) {
                Pb[3 * id + 0] = PB[0];
                Pb[3 * id + 1] = PB[1];
                Pb[3 * id + 2] = PB[3];
            }
            if (J) J[id] = Jv;
            if (sigma) {
                double F[4] = {1.0 + H[0], H[1], H[2], 1.0 + H[3]};
                double sg[4];
                for (int a = 0; a < 2; a++)
                    for (int b = 0; b < 2; b++)
                        sg[2 * a + b] = (PP[2 * a] * F[2 * b] + PP[2 * a + 1] * F[2 * b + 1]) / Jv;
                sigma[3 * id + 0] = sg[0];
                sigma[3 * id + 1] = sg[1];
                sigma[3 * id + 2] = sg[3];
            }
        }
}

/* Displacement gradient H = Grad u(t) (R15), [ny][nx][4] row-major 2x2. */
void orc_read_grad(const orc_state* s, double* H) {
    double t = s->step * s->dt;
    for (int y = 0; y < s->p.ny; y++)
        for (int x = 0; x < s->p.nx; x++) {
            double* h = H + 4 * IDX(s, x, y);
            if (in_hole(s, x, y))
                h[0] = h[1] = h[2] = h[3] = 0.0;
            else
                grad_u(s, s->u, x, y, t, h);
        }
}

/* Raw populations f_i(X, t) (after streaming), [9][ny][nx]. */
void orc_read_populations(const orc_state* s, double* out) {
    for (int i = 0; i < 9; i++) memcpy(out + (long)i * s->n, s->f[i], sizeof(double) * s->n);
}

void orc_destroy(orc_state* s) {
    if (!s) return;
    for (int i = 0; i < 9; i++) {
        free(s->f[i]);
        free(s->fnew[i]);
        free(s->fcol[i]);
    }
    free(s->r);
    for (int a = 0; a < 2; a++) {
        free(s->j[a]);
        free(s->jnew[a]);
        free(s->jp[a]);
        free(s->m[a]);
        free(s->u[a]);
        free(s->us[a]);
        free(s->S[a]);
    }
    for (int k = 0; k < 4; k++) {
        free(s->P[k]);
        free(s->Pb[k]);
    }
    free(s);
}
