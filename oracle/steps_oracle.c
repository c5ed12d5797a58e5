/*
 * steps_oracle.c -- plain FP64 CPU oracle for the StePS direct-summation
 * hot path (Racz, Szapudi, Dobos, Csabai & Szalay, "StePS: A Multi-GPU
 * Cosmological N-body Code for Compactified Simulations").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the GPU library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * Every routine follows the paper's equations literally, in FP64, summing in
 * index order.  Compiled with -O2 -fno-fast-math -ffp-contract=off so that no
 * contraction or reassociation changes the arithmetic written here.  The O(N^2)
 * loops are split over targets with OpenMP; each target's sum still runs in
 * plain j order, so results do not depend on the thread count.
 *
 * Parity status: every function here is pinned by a CPU test against values
 * the paper or the mathematics fixes (see the test suite):
 *   oracle_spline_F      -- Gauss's law on the cubic-spline density, closed
 *                           values at r=h/2 and r=h, the small-r slope
 *   oracle_pair_acc      -- single-pair closed form, uniform-shell theorem,
 *                           Newton's third law, brute force in exact rationals
 *   oracle_pair_W        -- dW/dr = F, W(0) = -2.8/H, Kepler energy
 *   oracle_rk4_a         -- flat LambdaCDM closed form t(a)
 *   oracle_kdk_step      -- Kepler orbit (period, second order), energy
 *                           conservation, uniform comoving sphere at rest
 *   oracle_pair_acc_periodic -- a cubic lattice feels no force, translation
 *                           invariance, third law, quasi-periodic = open sum
 *                           for a compact cluster, the cut at 2.6 L
 *   oracle_timestep      -- closed forms: a bound pair, a lone particle at
 *                           rest off-centre (background term) and a moving
 *                           one (friction term); dt_max and t_end limits
 *   oracle_paircount     -- independent k-d tree counts
 *   oracle_mlp_*         -- finite-difference gradients
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Eq. 4: the spline softening kernel F(r, h).  h is the full support:  */
/* the force is exactly Newtonian (1/r^2) for r >= h.  Branch limits    */
/* (the paper omits equality): r < h/2, h/2 <= r < h, r >= h.           */
/* ------------------------------------------------------------------ */
double oracle_spline_F(double r, double h)
{
    if (r >= h)
        return 1.0 / (r * r);
    double h2 = h * h, h3 = h2 * h, h4 = h3 * h, h5 = h4 * h, h6 = h5 * h;
    double r2 = r * r, r3 = r2 * r, r4 = r3 * r;
    if (r < 0.5 * h)
        return 32.0 * r4 / h6 - 38.4 * r3 / h5 + 32.0 * r / (3.0 * h3);
    return -32.0 * r4 / (3.0 * h6) + 38.4 * r3 / h5 - 48.0 * r2 / h4
           + 64.0 * r / (3.0 * h3) - 1.0 / (15.0 * r2);
}

/* ------------------------------------------------------------------ */
/* Pair potential W(r, H) = -int_r^inf F(s, H) ds, per unit G m_i m_j.   */
/* The paper prints only the force; this antiderivative of Eq. 4 is     */
/* taken branch by branch and made continuous at s = H/2 and s = H:     */
/*   u >= 1      : W = -1/r                                             */
/*   1/2 <= u < 1: W = (1/H)(-16/5 - 32/15 u^5 + 48/5 u^4 - 16 u^3      */
/*                           + 32/3 u^2 + 1/(15 u))                     */
/*   u < 1/2     : W = (1/H)(-14/5 + 32/5 u^5 - 48/5 u^4 + 16/3 u^2)    */
/* with u = r/H, so W(0) = -2.8/H.                                       */
/* ------------------------------------------------------------------ */
double oracle_pair_W(double r, double H)
{
    if (r >= H)
        return -1.0 / r;
    double u = r / H, u2 = u * u, u3 = u2 * u, u4 = u3 * u, u5 = u4 * u;
    if (u < 0.5)
        return (-14.0 / 5.0 + 32.0 / 5.0 * u5 - 48.0 / 5.0 * u4 + 16.0 / 3.0 * u2) / H;
    return (-16.0 / 5.0 - 32.0 / 15.0 * u5 + 48.0 / 5.0 * u4 - 16.0 * u3 + 32.0 / 3.0 * u2
            + 1.0 / (15.0 * u)) / H;
}

/* ------------------------------------------------------------------ */
/* Eq. 7: h_i = (m_i / m_min)^(1/3) h_min.                              */
/* ------------------------------------------------------------------ */
void oracle_softening(int64_t n, const double *m, double h_min, double *h_out)
{
    double m_min = m[0];
    for (int64_t i = 1; i < n; i++)
        if (m[i] < m_min) m_min = m[i];
    for (int64_t i = 0; i < n; i++)
        h_out[i] = cbrt(m[i] / m_min) * h_min;
}

/* ------------------------------------------------------------------ */
/* Eq. 3 with the pair sum of Eq. 8 (and Eq. 2):                       */
/*   acc_i = sum_{j != i} m_j F(x_i - x_j, h_i + h_j)                  */
/*         = -G sum_{j != i} m_j Fcal(|x_i - x_j|, h_i + h_j)          */
/*                          (x_i - x_j)/|x_i - x_j|                    */
/* i.e. the pair term before the 1/a^3 of Eq. 8.  pos is [n][3].        */
/* targets (length nt) selects which rows to compute; NULL = all rows,  */
/* in which case nt must equal n.  acc_out is [nt][3].                  */
/* Coincident distinct particles contribute nothing (Fcal(0) = 0).      */
/* ------------------------------------------------------------------ */
void oracle_pair_acc(int64_t n, const double *pos, const double *m, const double *h,
                     double G, int64_t nt, const int64_t *targets, double *acc_out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets ? targets[t] : t;
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = pos[3 * i + 0] - pos[3 * j + 0];
            double dy = pos[3 * i + 1] - pos[3 * j + 1];
            double dz = pos[3 * i + 2] - pos[3 * j + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r == 0.0) continue;
            double f = -G * m[j] * oracle_spline_F(r, h[i] + h[j]) / r;
            ax += f * dx;
            ay += f * dy;
            az += f * dz;
        }
        acc_out[3 * t + 0] = ax;
        acc_out[3 * t + 1] = ay;
        acc_out[3 * t + 2] = az;
    }
}

/* Total pair potential energy, 1/2 sum_i sum_{j != i} G m_i m_j W(r_ij, h_i + h_j). */
double oracle_pair_potential(int64_t n, const double *pos, const double *m, const double *h,
                             double G)
{
    double *row = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = pos[3 * i + 0] - pos[3 * j + 0];
            double dy = pos[3 * i + 1] - pos[3 * j + 1];
            double dz = pos[3 * i + 2] - pos[3 * j + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            s += G * m[i] * m[j] * oracle_pair_W(r, h[i] + h[j]);
        }
        row[i] = s;
    }
    double e = 0.0;
    for (int64_t i = 0; i < n; i++) e += row[i];
    free(row);
    return 0.5 * e;
}

/* ------------------------------------------------------------------ */
/* Cosmology: Eq. 1, adot/a = H0 sqrt(Om a^-3 + Or a^-4 + OL + Ok a^-2) */
/* ------------------------------------------------------------------ */
typedef struct {
    double G, H0, Om, OL, Or, Ok;
    int comoving; /* 0: static Newtonian (the paper's non-comoving mode), 1: Eq. 8 */
    int reversed; /* 1: Eq. 8 with gravity reversed (glass relaxation, Sec. 3.1): the pair */
                  /*    term and the background term both change sign                       */
} oracle_cosmo;

/* G of the pair term: -G when gravity is reversed. */
static double pair_G(const oracle_cosmo *c) { return c->reversed ? -c->G : c->G; }

double oracle_hubble(double a, const oracle_cosmo *c)
{
    return c->H0 * sqrt(c->Om / (a * a * a) + c->Or / (a * a * a * a) + c->OL + c->Ok / (a * a));
}

static double adot(double a, const oracle_cosmo *c) { return a * oracle_hubble(a, c); }

/* One classical fourth-order Runge-Kutta step of da/dt = a H(a) with the  */
/* N-body time step (the paper integrates a(t) by RK4 with the same dt).   */
double oracle_rk4_a(double a, double dt, const oracle_cosmo *c)
{
    double k1 = adot(a, c);
    double k2 = adot(a + 0.5 * dt * k1, c);
    double k3 = adot(a + 0.5 * dt * k2, c);
    double k4 = adot(a + dt * k3, c);
    return a + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
}

/* ------------------------------------------------------------------ */
/* Eq. 8: the full acceleration for the kick.                            */
/*   comoving: A = acc/a^3 - 2 H v + (4 pi G / 3) rho_bar x / a^3,      */
/*             rho_bar = Om rho_crit, rho_crit = 3 H0^2 / (8 pi G)       */
/*   static  : A = acc                                                   */
/* acc is the pair term computed by oracle_pair_acc (G included).        */
/* The a^-3 on the background term is this oracle's reading: it makes a  */
/* uniform comoving sphere feel no peculiar acceleration at any a, which */
/* is what the shell-theorem derivation of Eq. 8 requires.               */
/* ------------------------------------------------------------------ */
static void kick(int64_t n, double *vel, const double *pos, const double *acc, double dtk,
                 double a, const oracle_cosmo *c)
{
    if (!c->comoving) {
        for (int64_t k = 0; k < 3 * n; k++) vel[k] += dtk * acc[k];
        return;
    }
    double H = oracle_hubble(a, c);
    double rho_crit = 3.0 * c->H0 * c->H0 / (8.0 * M_PI * c->G);
    double bg = 4.0 * M_PI * pair_G(c) / 3.0 * c->Om * rho_crit;
    double a3 = a * a * a;
    for (int64_t k = 0; k < 3 * n; k++) {
        double A = acc[k] / a3 - 2.0 * H * vel[k] + bg * pos[k] / a3;
        vel[k] += dtk * A;
    }
}

/* ------------------------------------------------------------------ */
/* Eq. 9-11: one kick-drift-kick step, U(dt) = K(dt/2) D(dt) K(dt/2).   */
/* On entry acc holds the pair term at the current positions (with the  */
/* sign of gravity of c, see pair_G); on exit                            */
/* it holds the pair term at the new positions (one force evaluation    */
/* per step).  *a and *t advance by RK4 over dt.  In each half-kick the  */
/* friction and background use a, H at that half-kick's own time point  */
/* and v at kick entry (explicit).                                       */
/* ------------------------------------------------------------------ */
void oracle_kdk_step(int64_t n, double *pos, double *vel, double *acc, const double *m,
                     const double *h, double dt, double *a, double *t, const oracle_cosmo *c)
{
    kick(n, vel, pos, acc, 0.5 * dt, *a, c);                  /* K(dt/2) */
    for (int64_t k = 0; k < 3 * n; k++) pos[k] += vel[k] * dt;  /* D(dt)   */
    if (c->comoving) *a = oracle_rk4_a(*a, dt, c);
    *t += dt;
    oracle_pair_acc(n, pos, m, h, pair_G(c), n, NULL, acc);   /* force   */
    kick(n, vel, pos, acc, 0.5 * dt, *a, c);                  /* K(dt/2) */
}

/* ------------------------------------------------------------------ */
/* Periodic pair term (Sec. 2.2, Eq. 2 with the image sum of Eq. 5):      */
/*   acc_i = -G sum_{j != i} m_j sum_n F(|d_n|, h_i + h_j) d_n / |d_n|,    */
/*   d_n = (x_i - x_j) - n L,                                            */
/* images = 0: every integer triplet n with |d_n| < 2.6 L (the cut of    */
/*             Sec. 2.2);                                                */
/* images = 1: quasi-periodic, the leading term only: the one n with     */
/*             d_n in [-L/2, L/2)^3, i.e. n = floor(d_0 / L + 1/2) per   */
/*             component.                                                */
/* Written without contraction: dx = (xi - xj) - nx * L, r2 = dx*dx +    */
/* dy*dy + dz*dz, compared with (2.6 L)^2.                               */
/* ------------------------------------------------------------------ */
static void add_image(double *acc, double dx, double dy, double dz, double mj, double H, double G)
{
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (r == 0.0) return;
    double f = G * mj * oracle_spline_F(r, H) / r;
    acc[0] -= f * dx;
    acc[1] -= f * dy;
    acc[2] -= f * dz;
}

void oracle_pair_acc_periodic(int64_t n, const double *pos, const double *m, const double *h, double G,
                              double L, int images, int64_t nt, const int64_t *targets, double *out)
{
    const double cut = 2.6 * L, cut2 = cut * cut;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets ? targets[t] : t;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double d0x = pos[3 * i] - pos[3 * j];
            double d0y = pos[3 * i + 1] - pos[3 * j + 1];
            double d0z = pos[3 * i + 2] - pos[3 * j + 2];
            double H = h[i] + h[j];
            if (images == 1) {
                double nx = floor(d0x / L + 0.5), ny = floor(d0y / L + 0.5), nz = floor(d0z / L + 0.5);
                add_image(acc, d0x - nx * L, d0y - ny * L, d0z - nz * L, m[j], H, G);
                continue;
            }
            long ax = (long)floor((d0x - cut) / L), bx = (long)ceil((d0x + cut) / L);
            long ay = (long)floor((d0y - cut) / L), by = (long)ceil((d0y + cut) / L);
            long az = (long)floor((d0z - cut) / L), bz = (long)ceil((d0z + cut) / L);
            for (long nx = ax; nx <= bx; nx++)
                for (long ny = ay; ny <= by; ny++)
                    for (long nz = az; nz <= bz; nz++) {
                        double dx = d0x - (double)nx * L;
                        double dy = d0y - (double)ny * L;
                        double dz = d0z - (double)nz * L;
                        double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 < cut2) add_image(acc, dx, dy, dz, m[j], H, G);
                    }
        }
        out[3 * t] = acc[0];
        out[3 * t + 1] = acc[1];
        out[3 * t + 2] = acc[2];
    }
}

/* One KDK step of the periodic comoving equation of motion (Eq. 2):      */
/* A = acc / a^3 - 2 H v (no background term), positions wrapped into    */
/* [0, L)^3 after the drift, acc from oracle_pair_acc_periodic.           */
void oracle_kdk_step_periodic(int64_t n, double *pos, double *vel, double *acc, const double *m,
                              const double *h, double dt, double *a, double *t, double G, double H0,
                              double Om, double OL, double Or, double Ok, double L, int images)
{
    oracle_cosmo c = {G, H0, Om, OL, Or, Ok, 1, 0};
    for (int half = 0; half < 2; half++) {
        if (half == 1) {
            for (int64_t k = 0; k < 3 * n; k++) {
                pos[k] += vel[k] * dt;
                pos[k] -= L * floor(pos[k] / L);
            }
            *a = oracle_rk4_a(*a, dt, &c);
            *t += dt;
            oracle_pair_acc_periodic(n, pos, m, h, G, L, images, n, NULL, acc);
        }
        double H = oracle_hubble(*a, &c), a3 = (*a) * (*a) * (*a);
        for (int64_t k = 0; k < 3 * n; k++) vel[k] += 0.5 * dt * (acc[k] / a3 - 2.0 * H * vel[k]);
    }
}

/* ------------------------------------------------------------------ */
/* Eq. 12: adaptive time step of the KDK integrator,                     */
/*   dt = min(dt_max, min_i sqrt(2 eta_i eps / |A_i|)),                  */
/* eta_i = 2.8 h_i as printed (the paper calls it the Plummer-equivalent */
/* softening length), eps the accuracy parameter, and A_i the            */
/* acceleration the next kick would apply at the current state: the      */
/* comoving Eq. 8 (pair term / a^3 - 2 H v + background) or, in static    */
/* mode, the pair term.  A particle with A_i = 0 sets no limit.  If       */
/* t_left is finite the step is also limited to t_left (never below 0).  */
/* acc holds the pair term at pos (G included), as for the kick.         */
/* ------------------------------------------------------------------ */
double oracle_timestep(int64_t n, const double *pos, const double *vel, const double *acc,
                       const double *h, double eps, double dt_max, double t_left, double a,
                       const oracle_cosmo *c)
{
    double q_min = INFINITY;
    double H = 0.0, bg = 0.0, a3 = 1.0;
    if (c->comoving) {
        double rho_crit = 3.0 * c->H0 * c->H0 / (8.0 * M_PI * c->G);
        H = oracle_hubble(a, c);
        bg = 4.0 * M_PI * pair_G(c) / 3.0 * c->Om * rho_crit;
        a3 = a * a * a;
    }
    for (int64_t i = 0; i < n; i++) {
        double A2 = 0.0;
        for (int k = 0; k < 3; k++) {
            double A = acc[3 * i + k];
            if (c->comoving) A = acc[3 * i + k] / a3 - 2.0 * H * vel[3 * i + k] + bg * pos[3 * i + k] / a3;
            A2 += A * A;
        }
        double Amag = sqrt(A2);
        if (Amag > 0.0) {
            double eta = 2.8 * h[i];
            double q = 2.0 * eta * eps / Amag;
            if (q < q_min) q_min = q;
        }
    }
    double dt = dt_max;
    if (q_min < INFINITY && sqrt(q_min) < dt) dt = sqrt(q_min);
    if (isfinite(t_left) && t_left < dt) dt = t_left > 0.0 ? t_left : 0.0;
    return dt;
}

/* Kinetic energy and momentum, 1/2 sum m v^2 and sum m v. */
void oracle_kinetic(int64_t n, const double *vel, const double *m, double *ekin, double p[3])
{
    double e = 0.0, px = 0.0, py = 0.0, pz = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
        e += 0.5 * m[i] * (vx * vx + vy * vy + vz * vz);
        px += m[i] * vx;
        py += m[i] * vy;
        pz += m[i] * vz;
    }
    *ekin = e;
    p[0] = px;
    p[1] = py;
    p[2] = pz;
}

/* ------------------------------------------------------------------ */
/* Pair counts DD(r) for the correlation-function targets.  Positions    */
/* are integer fixed-point coordinates q[n][3]; a pair (i<j) falls in    */
/* bin b when edge2[b] <= |q_i - q_j|^2 < edge2[b+1] (squared edges in   */
/* the same integer units, nbins+1 of them).  Exact in int64.            */
/* ------------------------------------------------------------------ */
void oracle_paircount(int64_t n, const int32_t *q, int nbins, const int64_t *edge2, uint64_t *dd)
{
    for (int b = 0; b < nbins; b++) dd[b] = 0;
    for (int64_t i = 0; i < n; i++) {
        for (int64_t j = i + 1; j < n; j++) {
            int64_t dx = (int64_t)q[3 * i] - q[3 * j];
            int64_t dy = (int64_t)q[3 * i + 1] - q[3 * j + 1];
            int64_t dz = (int64_t)q[3 * i + 2] - q[3 * j + 2];
            int64_t d2 = dx * dx + dy * dy + dz * dz;
            for (int b = 0; b < nbins; b++) {
                if (d2 >= edge2[b] && d2 < edge2[b + 1]) {
                    dd[b]++;
                    break;
                }
            }
        }
    }
}
