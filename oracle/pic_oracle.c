/*
 * FP64 CPU oracle of the boosted-frame (relativistic reference frame, RRF) PIC step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm may load this library.  It shares no code, header,
 * table or helper with the CUDA path; the two only share seeded input generators.
 *
 * Plain, slow, obviously-correct restatement of the method, one function per step:
 *   - Maxwell in normalised units (c = 1, time in 1/w_n, length in c/w_n, fields in
 *     m_e c w_n / e, density in n_n = m_e w_n^2/(4 pi e^2)):  dE/dt = curl B - J,
 *     dB/dt = -curl E, div E = rho  (Gaussian form of Eq. Max1-Max2 rescaled; the
 *     normalisation follows the rule stated with Table I, Sec. "Electron propagation").
 *   - Yee staggering; B split into two half steps so E^n and B^n are co-timed at the
 *     particle gather (reading: the paper does not state the time centring).
 *   - Leap-frog relativistic push (Sec. "Relativistic booster frame": second-order
 *     leap-frog); read as the Boris rotation.
 *   - Charge-conserving current weighting (Eq. Max3-Max4 solved by current weighting)
 *     read as the Esirkepov decomposition, for CIC (order 1) and TSC (order 2).
 *   - Ions are a separate population with the same weighting as the plasma electrons
 *     and their own current (Sec. "Relativistic booster frame", ion current j_i = v_R rho_i).
 *   - Lab -> RRF transform of events and momenta (Eq. Lor1, Lor2, RRFVel), ballistic drift
 *     to t' = 0 (Eq. BGauss/Belon are taken at t' = 0).
 *   - Static lab undulator field transformed into the RRF with Eq. M1-M4, moving at
 *     -c beta_R (Eq. Vprime).
 *   - Plasma density N' = gamma_R N (Eq. Nnormi) and drift -beta_R (Eq. Vprime).
 *   - Moving window, absorbing field boundaries (read as a convolutional PML) and
 *     "dummy" particles beyond the boundaries (Sec. "Relativistic booster frame").
 *   - Diagnostics in the RRF and back-transformed to the lab (Eq. Lor1-Lor2 inverted,
 *     drift to a common lab time; Eq. DT bounds the time spread).
 *
 * Positions are absolute FP64 grid coordinates in cell units (node i at coordinate i).
 * Every function cites the passage it follows.  Parity of the moving-window plasma
 * injection lattice and of the long-run ensemble physics is pinned only by the
 * invariants tested in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_MAXSP 8
enum { O_PERIODIC = 0, O_PML = 1, O_OPEN = 2 };
enum { O_EX = 0, O_EY, O_EZ, O_BX, O_BY, O_BZ, O_JX, O_JY, O_JZ };

typedef struct {
    double q, m;      /* charge in e, mass in m_e */
    int frozen;       /* 1: momentum never pushed (immobile lab ions drift at -beta_R) */
    long n, cap;
    double *X;        /* [3*cap] grid coordinates, particle-major */
    double *U;        /* [3*cap] u = p/(m c) */
    double *W;        /* [cap] weight: real particles per macroparticle, normalised */
    long *id;
    unsigned char *alive;
    long next_id;
} osp;

typedef struct {
    int n[3];
    double d[3], dt, gR, bR;
    int bc[3][2], pml, order;
    long ncell;
    double *F[9];
    double *psiE[3][3], *psiB[3][3]; /* [component][derivative dim] */
    double *sig_node[3], *sig_half[3];
    long step, shifts;
    int moving;
    double vw;
    int ext;
    double K, lam_u, ku, B0, phase0, z_start, ramp;
    int plasma, sp_e, sp_i, ppc[3], xr[4], nprof;
    double *zprof, *nprof_v;
    long m_last;
    int nsp;
    osp sp[O_MAXSP];
    long dropped; /* deposit contributions outside a non-periodic grid (should stay 0) */
    int pusher;   /* 0: Boris, 1: Vay */
    int gather;   /* 0: momentum-conserving (order everywhere), 1: energy-conserving */
    /* artificial neutralising ions fading over [ion_t0, ion_t0 + ion_T]: their current density
     * is ion_G / ion_T (z component, at the E_z points) while they fade */
    double *ion_G, ion_t0, ion_T;
    /* lab-frame snapshot of species snap_sp at lab time snap_T, by particle id: lab x, y, z,
     * u_x, u_y, u_z and weight, and a state (0 pending, 1 recorded, 2 missed) */
    int snap_sp;
    long snap_n;
    double snap_T, *snap;
    unsigned char *snap_state;
    int threads;  /* > 1: the particle loop runs on that many OpenMP threads (timing only) */
} osim;

/* ------------------------------------------------------------------ shapes */

/* Particle shape of order 1 (cloud-in-cell) or 2 (triangular-shaped cloud), as a
 * function of the distance from a node in cell units. */
static double o_shape(int order, double dd)
{
    double a = fabs(dd);
    if (order == 0) return (dd >= -0.5 && dd < 0.5) ? 1.0 : 0.0;   /* nearest grid point */
    if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
    if (a <= 0.5) return 0.75 - a * a;
    if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
    return 0.0;
}

static int o_margin_lo(int order) { return order == 1 ? 1 : 2; }
static int o_margin_hi(int order) { return order == 1 ? 2 : 3; }

/* ------------------------------------------------------------------ grid access */

static long o_wrap(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

/* Field value at integer index (i,j,k); outside a non-periodic face the value is 0. */
static double o_get(const osim *s, const double *f, long i, long j, long k)
{
    long c[3] = {i, j, k};
    for (int d = 0; d < 3; d++) {
        if (c[d] < 0 || c[d] >= s->n[d]) {
            if (s->bc[d][0] == O_PERIODIC) c[d] = o_wrap(c[d], s->n[d]);
            else return 0.0;
        }
    }
    return f[(c[2] * s->n[1] + c[1]) * s->n[0] + c[0]];
}

/* Linear index of (i,j,k) or -1 when outside a non-periodic face. */
static long o_index(const osim *s, long i, long j, long k)
{
    long c[3] = {i, j, k};
    for (int d = 0; d < 3; d++) {
        if (c[d] < 0 || c[d] >= s->n[d]) {
            if (s->bc[d][0] == O_PERIODIC) c[d] = o_wrap(c[d], s->n[d]);
            else return -1;
        }
    }
    return (c[2] * s->n[1] + c[1]) * s->n[0] + c[0];
}

/* ------------------------------------------------------------------ creation */

/* PML conductivity at coordinate pos (cells) in dim d: polynomial grading of order 3,
 * theoretical normal reflection 1e-8, layers of s->pml cells inside each PML face. */
static double o_sigma(const osim *s, int d, double pos)
{
    double L = (double)s->pml, depth = 0.0;
    if (s->pml <= 0) return 0.0;
    if (s->bc[d][0] == O_PML && pos < L) depth = L - pos;
    if (s->bc[d][1] == O_PML && pos > (double)(s->n[d] - 1) - L) {
        double dh = pos - ((double)(s->n[d] - 1) - L);
        if (dh > depth) depth = dh;
    }
    if (depth <= 0.0) return 0.0;
    double smax = 4.0 * (-log(1e-8)) / (2.0 * L * s->d[d]);
    double r = depth / L;
    return smax * r * r * r;
}

void *osim_create(int nx, int ny, int nz, double dx, double dy, double dz, double dt,
                  double gamma_R, const int *bc6, int pml, int order, int moving, double vw)
{
    osim *s = (osim *)calloc(1, sizeof(osim));
    s->n[0] = nx; s->n[1] = ny; s->n[2] = nz;
    s->d[0] = dx; s->d[1] = dy; s->d[2] = dz;
    s->dt = dt;
    s->gR = gamma_R;
    s->bR = sqrt(1.0 - 1.0 / (gamma_R * gamma_R)); /* Eq. RRFVel with c = 1 */
    for (int d = 0; d < 3; d++) { s->bc[d][0] = bc6[2 * d]; s->bc[d][1] = bc6[2 * d + 1]; }
    s->pml = pml;
    s->order = order;
    s->moving = moving;
    s->vw = vw;
    s->ncell = (long)nx * ny * nz;
    for (int f = 0; f < 9; f++) s->F[f] = (double *)calloc(s->ncell, sizeof(double));
    for (int c = 0; c < 3; c++)
        for (int d = 0; d < 3; d++) {
            s->psiE[c][d] = (double *)calloc(s->ncell, sizeof(double));
            s->psiB[c][d] = (double *)calloc(s->ncell, sizeof(double));
        }
    for (int d = 0; d < 3; d++) {
        s->sig_node[d] = (double *)calloc(s->n[d] + 1, sizeof(double));
        s->sig_half[d] = (double *)calloc(s->n[d] + 1, sizeof(double));
        for (int i = 0; i < s->n[d]; i++) {
            s->sig_node[d][i] = o_sigma(s, d, (double)i);
            s->sig_half[d][i] = o_sigma(s, d, (double)i + 0.5);
        }
    }
    return s;
}

void osim_destroy(void *h)
{
    osim *s = (osim *)h;
    if (!s) return;
    for (int f = 0; f < 9; f++) free(s->F[f]);
    for (int c = 0; c < 3; c++)
        for (int d = 0; d < 3; d++) { free(s->psiE[c][d]); free(s->psiB[c][d]); }
    for (int d = 0; d < 3; d++) { free(s->sig_node[d]); free(s->sig_half[d]); }
    for (int i = 0; i < s->nsp; i++) {
        osp *p = &s->sp[i];
        free(p->X); free(p->U); free(p->W); free(p->id); free(p->alive);
    }
    free(s->zprof); free(s->nprof_v);
    free(s->ion_G);
    free(s->snap);
    free(s->snap_state);
    free(s);
}

double osim_beta(void *h) { return ((osim *)h)->bR; }

int osim_add_species(void *h, double q, double m, int frozen, long cap)
{
    osim *s = (osim *)h;
    if (s->nsp >= O_MAXSP) return -1;
    osp *p = &s->sp[s->nsp];
    memset(p, 0, sizeof(*p));
    p->q = q; p->m = m; p->frozen = frozen; p->cap = cap > 0 ? cap : 1;
    p->X = (double *)calloc(3 * p->cap, sizeof(double));
    p->U = (double *)calloc(3 * p->cap, sizeof(double));
    p->W = (double *)calloc(p->cap, sizeof(double));
    p->id = (long *)calloc(p->cap, sizeof(long));
    p->alive = (unsigned char *)calloc(p->cap, 1);
    return s->nsp++;
}

static int o_grow(osp *p, long need)
{
    if (need <= p->cap) return 0;
    long cap = p->cap;
    while (cap < need) cap *= 2;
    p->X = (double *)realloc(p->X, 3 * cap * sizeof(double));
    p->U = (double *)realloc(p->U, 3 * cap * sizeof(double));
    p->W = (double *)realloc(p->W, cap * sizeof(double));
    p->id = (long *)realloc(p->id, cap * sizeof(long));
    p->alive = (unsigned char *)realloc(p->alive, cap);
    p->cap = cap;
    return 0;
}

/* Active-region test of a grid coordinate in the non-periodic dims: particles whose
 * cell leaves [margin_lo, n-1-margin_hi] become dummy particles (Sec. "Relativistic
 * booster frame": particles beyond the boundaries become dummy). */
static int o_inside(const osim *s, const double X[3])
{
    for (int d = 0; d < 3; d++) {
        if (s->bc[d][0] == O_PERIODIC) continue;
        double c = floor(X[d]);
        if (c < o_margin_lo(s->order) || c > s->n[d] - 1 - o_margin_hi(s->order)) return 0;
    }
    return 1;
}

static void o_wrap_pos(const osim *s, double X[3])
{
    for (int d = 0; d < 3; d++) {
        if (s->bc[d][0] != O_PERIODIC) continue;
        double n = (double)s->n[d];
        if (X[d] < 0.0) X[d] += n;
        else if (X[d] >= n) X[d] -= n;
        if (X[d] >= n) X[d] = 0.0; /* -tiny + n rounding to n */
    }
}

/* ------------------------------------------------------------------ external field */

/* Lorentz transform of lab fields (E, B) into a frame moving with velocity beta along z,
 * Eq. M1-M4 with c = 1:  E'par = Epar, B'par = Bpar, E'perp = g (Eperp + u x B),
 * B'perp = g (Bperp - u x E). */
void oracle_field_transform(const double E[3], const double B[3], double beta,
                            double Ep[3], double Bp[3])
{
    double g = 1.0 / sqrt(1.0 - beta * beta);
    double u[3] = {0.0, 0.0, beta};
    double uxB[3] = {u[1] * B[2] - u[2] * B[1], u[2] * B[0] - u[0] * B[2], u[0] * B[1] - u[1] * B[0]};
    double uxE[3] = {u[1] * E[2] - u[2] * E[1], u[2] * E[0] - u[0] * E[2], u[0] * E[1] - u[1] * E[0]};
    Ep[2] = E[2];
    Bp[2] = B[2];
    for (int c = 0; c < 2; c++) {
        Ep[c] = g * (E[c] + uxB[c]);
        Bp[c] = g * (B[c] - uxE[c]);
    }
}

/* Entrance ramp f(z) of the undulator: linear ("gentle slope", Sec. "Electron propagation"),
 * 0 before z_start, 1 after z_start + ramp (ramp < 0: field everywhere; ramp = 0: a step). */
static double o_ramp(const osim *s, double zlab)
{
    double f = 1.0;
    if (s->ramp > 0.0) {
        double r = (zlab - s->z_start) / s->ramp;
        f = r <= 0.0 ? 0.0 : (r >= 1.0 ? 1.0 : r);
    } else if (s->ramp == 0.0 && isfinite(s->z_start)) {
        f = zlab >= s->z_start ? 1.0 : 0.0;
    }
    return f;
}

/* Planar-undulator lab field at lab (y, z): type 1, the ideal on-axis form B_y = B0 f(z)
 * cos(k_u z + phi0); type 2, the vacuum field of a planar undulator with poles above and below
 * in y: B_y = B0 f cosh(k_u y) cos(k_u z + phi0), B_z = -B0 f sinh(k_u y) sin(k_u z + phi0)
 * (div B = curl B = 0 where f = 1), y measured from the undulator axis. */
static void o_undulator_lab_B(const osim *s, double y, double zlab, double Bl[3])
{
    double a = s->B0 * o_ramp(s, zlab), ph = s->ku * zlab + s->phase0;
    Bl[0] = 0.0;
    if (s->ext == 2) {
        Bl[1] = a * cosh(s->ku * y) * cos(ph);
        Bl[2] = -a * sinh(s->ku * y) * sin(ph);
    } else {
        Bl[1] = a * cos(ph);
        Bl[2] = 0.0;
    }
}

/* External field at RRF absolute position (y, z') (normalised length; y from the undulator
 * axis, which the transverse boost leaves unchanged) and time t': the static lab element sits
 * at lab z = gR (z' + bR t') (it moves at -c bR in the RRF, Eq. Vprime; inverse of Eq.
 * Lor1-Lor2) and is transformed with Eq. M1-M4. */
static void o_external(const osim *s, double y, double zp, double tp, double E[3], double B[3])
{
    E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = 0.0;
    if (!s->ext) return;
    double zlab = s->gR * (zp + s->bR * tp);
    double El[3] = {0, 0, 0}, Bl[3];
    o_undulator_lab_B(s, y, zlab, Bl);
    oracle_field_transform(El, Bl, s->bR, E, B);
}

/* The undulator axis: the grid's y mid-plane. */
static double o_axis_y(const osim *s) { return 0.5 * s->n[1] * s->d[1]; }

void osim_set_external(void *h, int type, double K, double lambda_u, double phase,
                       double z_start, double ramp)
{
    osim *s = (osim *)h;
    s->ext = type;
    s->K = K;
    s->lam_u = lambda_u;
    s->ku = 2.0 * M_PI / lambda_u;
    s->B0 = K * s->ku; /* K = e B0 /(m c k_u) in normalised units */
    s->phase0 = phase;
    s->z_start = z_start;
    s->ramp = ramp;
}

void osim_set_pusher(void *h, int pusher) { ((osim *)h)->pusher = pusher; }
void osim_set_gather(void *h, int gather) { ((osim *)h)->gather = gather; }

/* Arm a lab-frame snapshot of species spi at lab time T (o_snap_record).  A particle whose
 * current lab time is already at or past T cannot be reconstructed: it is marked missed (2). */
void osim_snapshot_begin(void *h, int spi, double T)
{
    osim *s = (osim *)h;
    osp *p = &s->sp[spi];
    free(s->snap);
    free(s->snap_state);
    s->snap_sp = spi;
    s->snap_T = T;
    s->snap_n = p->next_id;
    s->snap = (double *)calloc(7 * (s->snap_n > 0 ? s->snap_n : 1), sizeof(double));
    s->snap_state = (unsigned char *)calloc(s->snap_n > 0 ? s->snap_n : 1, 1);
    double tp = (double)s->step * s->dt;
    for (long i = 0; i < p->n; i++) {
        if (!p->alive[i] || p->id[i] >= s->snap_n) continue;
        double tl = s->gR * (tp + s->bR * (p->X[3 * i + 2] + (double)s->shifts) * s->d[2]);
        if (tl >= T) s->snap_state[p->id[i]] = 2;
    }
}

/* The snapshot's records (by id, [n][7] as recorded) and states; returns the number recorded. */
long osim_snapshot_get(void *h, double *rec, unsigned char *state)
{
    osim *s = (osim *)h;
    long m = 0;
    for (long i = 0; i < s->snap_n; i++) {
        if (rec) memcpy(rec + 7 * i, s->snap + 7 * i, 7 * sizeof(double));
        if (state) state[i] = s->snap_state[i];
        if (s->snap_state[i] == 1) m++;
    }
    return m;
}

long osim_snapshot_n(void *h) { return ((osim *)h)->snap_n; }

void osim_external_at(void *h, double y, double zp, double tp, double *E, double *B)
{
    o_external((osim *)h, y, zp, tp, E, B);
}

/* Undulator vector potential at lab (y, z) without ramp: A_x = (B0/k_u) sin(k_u z + phi0)
 * (type 1), times cosh(k_u y) for the type-2 field, a Lorentz-invariant transverse component
 * with B_y = dA_x/dz_lab and B_z = -dA_x/dy. */
static double o_undulator_Ax(const osim *s, double y, double zlab)
{
    double a = s->B0 / s->ku * sin(s->ku * zlab + s->phase0);
    return s->ext == 2 ? a * cosh(s->ku * y) : a;
}

double osim_undulator_Ax(void *h, double y, double zlab) { return o_undulator_Ax((osim *)h, y, zlab); }

/* ------------------------------------------------------------------ loading */

/* Lab event (x, t=0) with momentum u -> RRF event (x', t') and u' (Eq. Lor1, Lor2 and
 * the matching momentum boost), then ballistic RRF drift to t' = 0 (Eq. BGauss/Belon
 * evaluate the distribution at t' = 0). */
void oracle_lab_to_boosted(double gR, const double x[3], const double u[3], double xp[3], double up[3])
{
    double bR = sqrt(1.0 - 1.0 / (gR * gR));
    double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double t_ev = gR * (0.0 - bR * x[2]);       /* Eq. Lor2 at t = 0 */
    double z_ev = gR * (x[2] - bR * 0.0);       /* Eq. Lor1 at t = 0 */
    double gp = gR * (g - bR * u[2]);
    up[0] = u[0];
    up[1] = u[1];
    up[2] = gR * (u[2] - bR * g);
    double dt = 0.0 - t_ev;
    xp[0] = x[0] + dt * up[0] / gp;
    xp[1] = x[1] + dt * up[1] / gp;
    xp[2] = z_ev + dt * up[2] / gp;
}

/* Inverse transform of an RRF event and momentum to the lab. */
void oracle_boosted_to_lab(double gR, const double xp[3], double tp, const double up[3],
                           double x[3], double *t, double u[3])
{
    double bR = sqrt(1.0 - 1.0 / (gR * gR));
    double gp = sqrt(1.0 + up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
    x[0] = xp[0];
    x[1] = xp[1];
    x[2] = gR * (xp[2] + bR * tp);
    *t = gR * (tp + bR * xp[2]);
    u[0] = up[0];
    u[1] = up[1];
    u[2] = gR * (up[2] + bR * gp);
}

/* Load n particles.  frame 0: lab positions (normalised, relative to the beam reference
 * point, at lab t = 0) and momenta, transformed with oracle_lab_to_boosted; frame 1: RRF
 * positions at t' = 0.  Grid coordinate = position/d + origin (cells).  match != 0 (lab
 * frame only): the beam is already inside the undulator, so before the transform the lab
 * transverse momentum gets the matched canonical part u_x += -(q/m) A_x(z_lab) and u_z is
 * reduced so that the lab energy is unchanged (a static magnetic field does no work); z_lab
 * of the event is z + gamma_R origin_z dz.  Returns the number loaded. */
long osim_load(void *h, int spi, long n, const double *x, const double *u, const double *w,
               int frame, const double *origin, int match)
{
    osim *s = (osim *)h;
    osp *p = &s->sp[spi];
    o_grow(p, p->n + n);
    long loaded = 0;
    for (long i = 0; i < n; i++) {
        double xi[3] = {x[i], x[n + i], x[2 * n + i]}, ui[3] = {u[i], u[n + i], u[2 * n + i]};
        double xp[3], up[3];
        if (frame == 0 && match && s->ext) {
            double g = sqrt(1.0 + ui[0] * ui[0] + ui[1] * ui[1] + ui[2] * ui[2]);
            double zlab = xi[2] + s->gR * origin[2] * s->d[2];
            double yax = xi[1] + origin[1] * s->d[1] - o_axis_y(s);
            ui[0] += -(p->q / p->m) * o_undulator_Ax(s, yax, zlab);
            ui[2] = sqrt(g * g - 1.0 - ui[0] * ui[0] - ui[1] * ui[1]);
        }
        if (frame == 0) oracle_lab_to_boosted(s->gR, xi, ui, xp, up);
        else { memcpy(xp, xi, sizeof xp); memcpy(up, ui, sizeof up); }
        double X[3];
        for (int d = 0; d < 3; d++) X[d] = xp[d] / s->d[d] + origin[d];
        long id = p->next_id++;
        o_wrap_pos(s, X);
        if (!o_inside(s, X)) continue;
        long k = p->n++;
        memcpy(&p->X[3 * k], X, sizeof X);
        memcpy(&p->U[3 * k], up, sizeof up);
        p->W[k] = w ? w[i] : 1.0;
        p->id[k] = id;
        p->alive[k] = 1;
        loaded++;
    }
    return loaded;
}

/* Replace a species' content with a given grid-coordinate state (identical-state tests). */
void osim_set_state(void *h, int spi, long n, const double *X, const double *U, const double *W,
                    const long *id)
{
    osim *s = (osim *)h;
    osp *p = &s->sp[spi];
    p->n = 0;
    o_grow(p, n);
    for (long i = 0; i < n; i++) {
        for (int d = 0; d < 3; d++) { p->X[3 * i + d] = X[3 * i + d]; p->U[3 * i + d] = U[3 * i + d]; }
        p->W[i] = W[i];
        p->id[i] = id[i];
        p->alive[i] = 1;
        if (id[i] >= p->next_id) p->next_id = id[i] + 1;
    }
    p->n = n;
}

void osim_set_next_id(void *h, int spi, long next) { ((osim *)h)->sp[spi].next_id = next; }

void osim_set_time(void *h, long step, long shifts, long m_last)
{
    osim *s = (osim *)h;
    s->step = step;
    s->shifts = shifts;
    s->m_last = m_last;
}

void osim_get_time(void *h, long *out3)
{
    osim *s = (osim *)h;
    out3[0] = s->step;
    out3[1] = s->shifts;
    out3[2] = s->m_last;
}

long osim_count(void *h, int spi)
{
    osim *s = (osim *)h;
    osp *p = &s->sp[spi];
    long c = 0;
    for (long i = 0; i < p->n; i++) c += p->alive[i];
    return c;
}

void osim_get_particles(void *h, int spi, double *X, double *U, double *W, long *id)
{
    osim *s = (osim *)h;
    osp *p = &s->sp[spi];
    long k = 0;
    for (long i = 0; i < p->n; i++) {
        if (!p->alive[i]) continue;
        for (int d = 0; d < 3; d++) { X[3 * k + d] = p->X[3 * i + d]; U[3 * k + d] = p->U[3 * i + d]; }
        W[k] = p->W[i];
        id[k] = p->id[i];
        k++;
    }
}

void osim_set_field(void *h, int which, const double *src)
{
    osim *s = (osim *)h;
    memcpy(s->F[which], src, s->ncell * sizeof(double));
}

void osim_get_field(void *h, int which, double *dst)
{
    osim *s = (osim *)h;
    memcpy(dst, s->F[which], s->ncell * sizeof(double));
}

/* ------------------------------------------------------------------ plasma */

/* Lab density profile n(z_lab): piecewise linear through the nodes, 0 outside. */
static double o_profile(const osim *s, double zlab)
{
    if (s->nprof <= 0) return 0.0;
    if (zlab < s->zprof[0] || zlab > s->zprof[s->nprof - 1]) return 0.0;
    for (int i = 0; i + 1 < s->nprof; i++) {
        if (zlab <= s->zprof[i + 1]) {
            double h = s->zprof[i + 1] - s->zprof[i];
            double r = h > 0.0 ? (zlab - s->zprof[i]) / h : 0.0;
            return s->nprof_v[i] + r * (s->nprof_v[i + 1] - s->nprof_v[i]);
        }
    }
    return s->nprof_v[s->nprof - 1];
}

/* Largest lattice-plane index m whose grid coordinate at step n (after `shifts` window
 * shifts) lies below the injection threshold nz - margin_hi.  Plane m sits at absolute
 * RRF coordinate ((m + 1/2)/p_z) dz - beta_R t' (static lab plasma moving at -c beta_R,
 * Eq. Vprime; lattice spacing dz/p_z in the RRF, i.e. the lab density times gamma_R,
 * Eq. Nnormi). */
static long o_plane_max(const osim *s, long n, long shifts)
{
    double thr = (double)(s->n[2] - o_margin_hi(s->order));
    double xv = (double)s->ppc[2] * (thr + (double)shifts + s->bR * (double)n * s->dt / s->d[2]) - 0.5;
    return (long)ceil(xv) - 1;
}

static void o_inject_planes(osim *s, long m0, long m1)
{
    if (m1 < m0) return;
    osp *pe = &s->sp[s->sp_e], *pi = &s->sp[s->sp_i];
    double tp = (double)s->step * s->dt;
    double uz = -s->gR * s->bR; /* u'_z = -gamma_R beta_R for a lab-static particle */
    long per_plane = (long)(s->xr[1] - s->xr[0]) * s->ppc[0] * (long)(s->xr[3] - s->xr[2]) * s->ppc[1];
    o_grow(pe, pe->n + (m1 - m0 + 1) * per_plane);
    o_grow(pi, pi->n + (m1 - m0 + 1) * per_plane);
    for (long m = m0; m <= m1; m++) {
        double zabs = ((double)m + 0.5) / (double)s->ppc[2]; /* cells, at t' = 0 */
        double zlab = s->gR * zabs * s->d[2];                 /* static lab position */
        double dens = s->gR * o_profile(s, zlab);             /* Eq. Nnormi */
        double zg = zabs - s->bR * tp / s->d[2] - (double)s->shifts;
        double w = dens * s->d[0] * s->d[1] * s->d[2] / ((double)s->ppc[0] * s->ppc[1] * s->ppc[2]);
        if (s->bc[2][0] == O_PERIODIC) zg -= floor(zg / (double)s->n[2]) * (double)s->n[2];
        for (int j = s->xr[2]; j < s->xr[3]; j++)
            for (int i = s->xr[0]; i < s->xr[1]; i++)
                for (int b = 0; b < s->ppc[1]; b++)
                    for (int a = 0; a < s->ppc[0]; a++) {
                        double X[3] = {i + (a + 0.5) / s->ppc[0], j + (b + 0.5) / s->ppc[1], zg};
                        long ide = pe->next_id++, idi = pi->next_id++;
                        if (dens <= 0.0 || !o_inside(s, X)) continue;
                        long ke = pe->n++, ki = pi->n++;
                        memcpy(&pe->X[3 * ke], X, sizeof X);
                        memcpy(&pi->X[3 * ki], X, sizeof X);
                        pe->U[3 * ke] = pe->U[3 * ke + 1] = 0.0;
                        pe->U[3 * ke + 2] = uz;
                        pi->U[3 * ki] = pi->U[3 * ki + 1] = 0.0;
                        pi->U[3 * ki + 2] = uz;
                        pe->W[ke] = w;
                        pi->W[ki] = w;
                        pe->id[ke] = ide;
                        pi->id[ki] = idi;
                        pe->alive[ke] = pi->alive[ki] = 1;
                    }
    }
}

/* Background plasma: electrons (species sp_e) and co-located ions (sp_i, same weighting,
 * Sec. "Relativistic booster frame"), lab profile (z nodes, density nodes), p_x*p_y*p_z
 * particles per cell on a regular lattice in the transverse cell range xr = {x0,x1,y0,y1}.
 * Fills the window at the current time (fill != 0); later steps inject planes entering the
 * front. */
void osim_set_plasma(void *h, int sp_e, int sp_i, const int *ppc, const int *xr, int nprof,
                     const double *zn, const double *dn, int fill)
{
    osim *s = (osim *)h;
    s->plasma = 1;
    s->sp_e = sp_e;
    s->sp_i = sp_i;
    memcpy(s->ppc, ppc, 3 * sizeof(int));
    memcpy(s->xr, xr, 4 * sizeof(int));
    s->nprof = nprof;
    free(s->zprof); free(s->nprof_v);
    s->zprof = (double *)malloc(nprof * sizeof(double));
    s->nprof_v = (double *)malloc(nprof * sizeof(double));
    memcpy(s->zprof, zn, nprof * sizeof(double));
    memcpy(s->nprof_v, dn, nprof * sizeof(double));
    if (!fill) return; /* parameters only: the caller loads an existing plasma state */
    if (s->bc[2][0] == O_PERIODIC) {
        /* periodic box (reading): the lattice fills the whole box once, planes 0 .. p_z n_z - 1,
         * and drifts around it; the density of plane m is the profile at its lab position at
         * t' = 0 and travels with it.  No plane is ever injected. */
        long m1 = (long)s->ppc[2] * s->n[2] - 1;
        o_inject_planes(s, 0, m1);
        s->m_last = m1;
        return;
    }
    double lo = (double)o_margin_lo(s->order) + (double)s->shifts + s->bR * (double)s->step * s->dt / s->d[2];
    long m0 = (long)ceil((double)s->ppc[2] * lo - 0.5);
    long m1 = o_plane_max(s, s->step, s->shifts);
    o_inject_planes(s, m0, m1);
    s->m_last = m1;
}

/* ------------------------------------------------------------------ particle step */

/* Boris rotation (leap-frog momentum update u^{n-1/2} -> u^{n+1/2}) for charge-to-mass
 * ratio qm, with E and B at the particle (Sec. "Relativistic booster frame": leap-frog). */
void oracle_boris(double qm, double dt, const double E[3], const double B[3], double u[3])
{
    double h = 0.5 * qm * dt;
    double um[3] = {u[0] + h * E[0], u[1] + h * E[1], u[2] + h * E[2]};
    double g = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    double t[3] = {h * B[0] / g, h * B[1] / g, h * B[2] / g};
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    double sv[3] = {2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2), 2.0 * t[2] / (1.0 + t2)};
    double up[3] = {um[0] + um[1] * t[2] - um[2] * t[1],
                    um[1] + um[2] * t[0] - um[0] * t[2],
                    um[2] + um[0] * t[1] - um[1] * t[0]};
    double upl[3] = {um[0] + up[1] * sv[2] - up[2] * sv[1],
                     um[1] + up[2] * sv[0] - up[0] * sv[2],
                     um[2] + up[0] * sv[1] - up[1] * sv[0]};
    u[0] = upl[0] + h * E[0];
    u[1] = upl[1] + h * E[1];
    u[2] = upl[2] + h * E[2];
}

/* Vay's leap-frog push (the modified pusher the paper cites for boosted-frame runs, Sec. 1):
 * a half step with the old velocity, u_h = u + h (E + v x B); u' = u_h + h E; then the
 * new Lorentz factor solves gamma^2 = (sigma + sqrt(sigma^2 + 4 (tau^2 + (u'.tau)^2))) / 2 with
 * tau = h B, sigma = gamma'^2 - tau^2, and u+ = s (u' + (u'.t) t + u' x t), t = tau / gamma,
 * s = 1 / (1 + t^2); h = qm dt / 2.  It keeps E + v x B = 0 drifts exact. */
void oracle_vay(double qm, double dt, const double E[3], const double B[3], double u[3])
{
    double h = 0.5 * qm * dt;
    double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double v[3] = {u[0] / g, u[1] / g, u[2] / g};
    double vxb[3] = {v[1] * B[2] - v[2] * B[1], v[2] * B[0] - v[0] * B[2], v[0] * B[1] - v[1] * B[0]};
    double up[3];
    for (int c = 0; c < 3; c++) up[c] = u[c] + h * (E[c] + vxb[c]) + h * E[c];
    double tau[3] = {h * B[0], h * B[1], h * B[2]};
    double tau2 = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
    double ust = up[0] * tau[0] + up[1] * tau[1] + up[2] * tau[2];
    double sigma = 1.0 + up[0] * up[0] + up[1] * up[1] + up[2] * up[2] - tau2;
    double g1 = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (tau2 + ust * ust))));
    double t[3] = {tau[0] / g1, tau[1] / g1, tau[2] / g1};
    double s = 1.0 / (1.0 + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    double ut = up[0] * t[0] + up[1] * t[1] + up[2] * t[2];
    double uxt[3] = {up[1] * t[2] - up[2] * t[1], up[2] * t[0] - up[0] * t[2], up[0] * t[1] - up[1] * t[0]};
    for (int c = 0; c < 3; c++) u[c] = s * (up[c] + ut * t[c] + uxt[c]);
}

/* Interpolate grid component f, whose nodes sit at index + stag (cells), to X with the
 * particle shape.  Momentum-conserving gather: the deposit's order in every dim.  Energy-
 * conserving gather: one order lower along the dims where the component is staggered (the
 * x-shape of the Esirkepov current J_x is the lower-order shape at the half-integer nodes, so
 * E_x gathered this way is the transpose of the deposit; for a gradient field E = -grad_h phi it
 * gives exactly -d/dx of phi interpolated with the full-order shape). */
static double o_gather(const osim *s, const double *f, const double stag[3], const double X[3])
{
    long lo[3], cnt[3];
    double wv[3][6];
    for (int d = 0; d < 3; d++) {
        int ord = (s->gather == 1 && stag[d] != 0.0) ? s->order - 1 : s->order;
        double h = 0.5 * (ord + 1);
        lo[d] = (long)floor(X[d] - stag[d] - h);
        long hi = (long)floor(X[d] - stag[d] + h);
        cnt[d] = hi - lo[d] + 1;
        for (long a = 0; a < cnt[d]; a++) wv[d][a] = o_shape(ord, (double)(lo[d] + a) + stag[d] - X[d]);
    }
    double sum = 0.0;
    for (long c = 0; c < cnt[2]; c++)
        for (long b = 0; b < cnt[1]; b++)
            for (long a = 0; a < cnt[0]; a++) {
                double ww = wv[0][a] * wv[1][b] * wv[2][c];
                if (ww != 0.0) sum += ww * o_get(s, f, lo[0] + a, lo[1] + b, lo[2] + c);
            }
    return sum;
}

/* Yee positions: E_c staggered by 1/2 along c; B_c staggered by 1/2 along the other two. */
static const double O_STAG[6][3] = {
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}};

static void o_add(const osim *s, double *f, long *dropped, long i, long j, long k, double v)
{
    long ix = o_index(s, i, j, k);
    if (ix < 0) { if (v != 0.0) (*dropped)++; return; }
    f[ix] += v;
}

/* Esirkepov charge-conserving current of one particle of charge q and weight w moving
 * from X0 to X1 (cells) during dt: with S0, S1 the shapes at the old and new position
 * and DS = S1 - S0 per dimension,
 *   W_x = DS_x (S0_y S0_z + DS_y S0_z/2 + S0_y DS_z/2 + DS_y DS_z/3)   (cyclic for y, z),
 *   J_x(i+1/2) - J_x(i-1/2) = -q w (dx/dt) W_x(i) / V_cell,
 * accumulated from the low end of the stencil where J = 0. */
static void o_esirkepov(const osim *s, double *const J[3], long *dropped, double qw, const double X0[3],
                        const double X1[3])
{
    long lo[3], cnt[3];
    double S0[3][8], DS[3][8];
    double h = 0.5 * (s->order + 1);
    for (int d = 0; d < 3; d++) {
        double mn = X0[d] < X1[d] ? X0[d] : X1[d], mx = X0[d] < X1[d] ? X1[d] : X0[d];
        lo[d] = (long)floor(mn - h);
        long hi = (long)floor(mx + h);
        cnt[d] = hi - lo[d] + 1;
        if (cnt[d] > 8) cnt[d] = 8; /* a move below one cell keeps cnt <= 5 */
        for (long a = 0; a < cnt[d]; a++) {
            double node = (double)(lo[d] + a);
            S0[d][a] = o_shape(s->order, node - X0[d]);
            DS[d][a] = o_shape(s->order, node - X1[d]) - S0[d][a];
        }
    }
    double V = s->d[0] * s->d[1] * s->d[2];
    double cf[3] = {-qw * s->d[0] / (s->dt * V), -qw * s->d[1] / (s->dt * V), -qw * s->d[2] / (s->dt * V)};
    /* J_x: prefix along x for each (y, z) */
    for (long c = 0; c < cnt[2]; c++)
        for (long b = 0; b < cnt[1]; b++) {
            double acc = 0.0;
            for (long a = 0; a < cnt[0]; a++) {
                double Wx = DS[0][a] * (S0[1][b] * S0[2][c] + 0.5 * DS[1][b] * S0[2][c] +
                                        0.5 * S0[1][b] * DS[2][c] + DS[1][b] * DS[2][c] / 3.0);
                acc += Wx;
                o_add(s, J[0], dropped, lo[0] + a, lo[1] + b, lo[2] + c, cf[0] * acc);
            }
        }
    /* J_y: prefix along y for each (x, z) */
    for (long c = 0; c < cnt[2]; c++)
        for (long a = 0; a < cnt[0]; a++) {
            double acc = 0.0;
            for (long b = 0; b < cnt[1]; b++) {
                double Wy = DS[1][b] * (S0[2][c] * S0[0][a] + 0.5 * DS[2][c] * S0[0][a] +
                                        0.5 * S0[2][c] * DS[0][a] + DS[2][c] * DS[0][a] / 3.0);
                acc += Wy;
                o_add(s, J[1], dropped, lo[0] + a, lo[1] + b, lo[2] + c, cf[1] * acc);
            }
        }
    /* J_z: prefix along z for each (x, y) */
    for (long b = 0; b < cnt[1]; b++)
        for (long a = 0; a < cnt[0]; a++) {
            double acc = 0.0;
            for (long c = 0; c < cnt[2]; c++) {
                double Wz = DS[2][c] * (S0[0][a] * S0[1][b] + 0.5 * DS[0][a] * S0[1][b] +
                                        0.5 * S0[0][a] * DS[1][b] + DS[0][a] * DS[1][b] / 3.0);
                acc += Wz;
                o_add(s, J[2], dropped, lo[0] + a, lo[1] + b, lo[2] + c, cf[2] * acc);
            }
        }
}

/* Lab-frame reconstruction at one lab time (Sec. "Understanding the RRF", Eq. DT): the particles
 * of one RRF instant sit at different lab times, so a lab snapshot at lab time T is assembled
 * particle by particle across the RRF steps.  During a step a particle moves on a straight RRF
 * segment from (x'_n, t'_n) to (x'_{n+1}, t'_n + dt) with momentum u^{n+1/2}; its lab time
 * t = gamma_R (t' + beta_R z') grows monotonically along it.  When [t_a, t_b) of the step contains
 * T, the event on the segment at lab time T is transformed to the lab (inverse Eq. Lor1-Lor2:
 * x, y unchanged, z = gamma_R (z' + beta_R t')) with the lab momentum of u^{n+1/2}
 * (u_z = gamma_R (u'_z + beta_R gamma')) and recorded under the particle's id.  z' counts the
 * window shifts; a periodic z is taken in the box's own image. */
static void o_snap_record(const osim *s, const osp *p, long i, const double X0[3], const double X1[3])
{
    long id = p->id[i];
    if (id < 0 || id >= s->snap_n || s->snap_state[id] != 0) return;
    double t0 = (double)s->step * s->dt;
    double z0 = (X0[2] + (double)s->shifts) * s->d[2], z1 = (X1[2] + (double)s->shifts) * s->d[2];
    double ta = s->gR * (t0 + s->bR * z0), tb = s->gR * (t0 + s->dt + s->bR * z1);
    if (!(ta < s->snap_T && s->snap_T <= tb)) return;
    double a = (s->snap_T - ta) / (tb - ta);
    double xp[3] = {(X0[0] + a * (X1[0] - X0[0])) * s->d[0], (X0[1] + a * (X1[1] - X0[1])) * s->d[1],
                    z0 + a * (z1 - z0)};
    double tp = t0 + a * s->dt;
    const double *U = &p->U[3 * i];
    double xl[3], ul[3], tl;
    oracle_boosted_to_lab(s->gR, xp, tp, U, xl, &tl, ul);
    double *r = &s->snap[7 * id];
    r[0] = xl[0]; r[1] = xl[1]; r[2] = xl[2];
    r[3] = ul[0]; r[4] = ul[1]; r[5] = ul[2];
    r[6] = p->W[i];
    s->snap_state[id] = 1;
}

/* Gather + push + move + deposit of particle i of species p (one leap-frog step); the current
 * goes to J[3], deposits outside a non-periodic grid are counted in *dropped. */
static void o_push_one(const osim *s, osp *p, long i, double *const J[3], long *dropped)
{
    double tp = (double)s->step * s->dt;
    double qm = p->q / p->m;
    double *X = &p->X[3 * i], *U = &p->U[3 * i];
    if (!p->frozen) {
        double E[3], B[3], Ee[3], Be[3];
        for (int c = 0; c < 3; c++) {
            E[c] = o_gather(s, s->F[O_EX + c], O_STAG[c], X);
            B[c] = o_gather(s, s->F[O_BX + c], O_STAG[3 + c], X);
        }
        o_external(s, X[1] * s->d[1] - o_axis_y(s), (X[2] + (double)s->shifts) * s->d[2], tp, Ee, Be);
        for (int c = 0; c < 3; c++) { E[c] += Ee[c]; B[c] += Be[c]; }
        if (s->pusher == 1) oracle_vay(qm, s->dt, E, B, U);
        else oracle_boris(qm, s->dt, E, B, U);
    }
    double g = sqrt(1.0 + U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
    double X1[3];
    for (int d = 0; d < 3; d++) X1[d] = X[d] + s->dt * U[d] / (g * s->d[d]);
    double Xw[3] = {X1[0], X1[1], X1[2]};
    o_wrap_pos(s, Xw);
    if (!o_inside(s, Xw)) { p->alive[i] = 0; return; }
    o_esirkepov(s, J, dropped, p->q * p->W[i], X, X1);
    if (s->snap && p == &s->sp[s->snap_sp]) o_snap_record(s, p, i, X, X1);
    memcpy(X, Xw, sizeof Xw);
}

/* Every live particle of species p, in index order, depositing into the grid's J. */
static void o_push_species(osim *s, osp *p)
{
    double *const J[3] = {s->F[O_JX], s->F[O_JY], s->F[O_JZ]};
#ifdef _OPENMP
    if (s->threads > 1) {
        /* Timing aid only: the particles are split over threads, each depositing into a private
         * copy of J that is added to the grid's J afterwards.  The sums then run in another order,
         * so the results differ from the serial loop at FP64 rounding; the serial loop is the
         * reference. */
        long dropped = 0;
#pragma omp parallel num_threads(s->threads) reduction(+ : dropped)
        {
            double *Jt = (double *)calloc(3 * s->ncell, sizeof(double));
            double *const Jl[3] = {Jt, Jt + s->ncell, Jt + 2 * s->ncell};
#pragma omp for schedule(static)
            for (long i = 0; i < p->n; i++)
                if (p->alive[i]) o_push_one(s, p, i, Jl, &dropped);
#pragma omp critical
            for (int c = 0; c < 3; c++)
                for (long k = 0; k < s->ncell; k++) J[c][k] += Jl[c][k];
            free(Jt);
        }
        s->dropped += dropped;
        return;
    }
#endif
    for (long i = 0; i < p->n; i++)
        if (p->alive[i]) o_push_one(s, p, i, J, &s->dropped);
}

/* Threads of the particle loop (1: the serial reference loop).  Returns the number used: 1
 * when the library was built without OpenMP. */
int osim_set_threads(void *h, int n)
{
    osim *s = (osim *)h;
#ifdef _OPENMP
    s->threads = n > 1 ? n : 1;
#else
    (void)n;
    s->threads = 1;
#endif
    return s->threads;
}

/* ------------------------------------------------------------------ fields */

static double o_b(double sig, double dtt) { return exp(-sig * dtt); }

/* Half (or full) step of B: B -= dtt curl E, with CPML auxiliary terms
 * psi = b psi + (b - 1) dF/ds in the PML slabs (kappa = 1, alpha = 0). */
static void o_update_B(osim *s, double dtt)
{
    const long nx = s->n[0], ny = s->n[1], nz = s->n[2];
    double *Ex = s->F[O_EX], *Ey = s->F[O_EY], *Ez = s->F[O_EZ];
    double dx = s->d[0], dy = s->d[1], dz = s->d[2];
    for (long k = 0; k < nz; k++)
        for (long j = 0; j < ny; j++)
            for (long i = 0; i < nx; i++) {
                long ix = (k * ny + j) * nx + i;
                double dEz_dy = (o_get(s, Ez, i, j + 1, k) - o_get(s, Ez, i, j, k)) / dy;
                double dEy_dz = (o_get(s, Ey, i, j, k + 1) - o_get(s, Ey, i, j, k)) / dz;
                double dEx_dz = (o_get(s, Ex, i, j, k + 1) - o_get(s, Ex, i, j, k)) / dz;
                double dEz_dx = (o_get(s, Ez, i + 1, j, k) - o_get(s, Ez, i, j, k)) / dx;
                double dEy_dx = (o_get(s, Ey, i + 1, j, k) - o_get(s, Ey, i, j, k)) / dx;
                double dEx_dy = (o_get(s, Ex, i, j + 1, k) - o_get(s, Ex, i, j, k)) / dy;
                /* B_x at (i, j+1/2, k+1/2), B_y at (i+1/2, j, k+1/2), B_z at (i+1/2, j+1/2, k) */
                double sy = s->sig_half[1][j], sz = s->sig_half[2][k], sx = s->sig_half[0][i];
                if (sy > 0) { double b = o_b(sy, dtt); s->psiB[0][1][ix] = b * s->psiB[0][1][ix] + (b - 1) * dEz_dy; dEz_dy += s->psiB[0][1][ix]; }
                if (sz > 0) { double b = o_b(sz, dtt); s->psiB[0][2][ix] = b * s->psiB[0][2][ix] + (b - 1) * dEy_dz; dEy_dz += s->psiB[0][2][ix]; }
                if (sz > 0) { double b = o_b(sz, dtt); s->psiB[1][2][ix] = b * s->psiB[1][2][ix] + (b - 1) * dEx_dz; dEx_dz += s->psiB[1][2][ix]; }
                if (sx > 0) { double b = o_b(sx, dtt); s->psiB[1][0][ix] = b * s->psiB[1][0][ix] + (b - 1) * dEz_dx; dEz_dx += s->psiB[1][0][ix]; }
                if (sx > 0) { double b = o_b(sx, dtt); s->psiB[2][0][ix] = b * s->psiB[2][0][ix] + (b - 1) * dEy_dx; dEy_dx += s->psiB[2][0][ix]; }
                if (sy > 0) { double b = o_b(sy, dtt); s->psiB[2][1][ix] = b * s->psiB[2][1][ix] + (b - 1) * dEx_dy; dEx_dy += s->psiB[2][1][ix]; }
                s->F[O_BX][ix] -= dtt * (dEz_dy - dEy_dz);
                s->F[O_BY][ix] -= dtt * (dEx_dz - dEz_dx);
                s->F[O_BZ][ix] -= dtt * (dEy_dx - dEx_dy);
            }
}

/* E += dt (curl B - J) (Eq. Max1 normalised), CPML as for B. */
static void o_update_E(osim *s)
{
    const long nx = s->n[0], ny = s->n[1], nz = s->n[2];
    double *Bx = s->F[O_BX], *By = s->F[O_BY], *Bz = s->F[O_BZ];
    double dx = s->d[0], dy = s->d[1], dz = s->d[2], dt = s->dt;
    for (long k = 0; k < nz; k++)
        for (long j = 0; j < ny; j++)
            for (long i = 0; i < nx; i++) {
                long ix = (k * ny + j) * nx + i;
                double dBz_dy = (o_get(s, Bz, i, j, k) - o_get(s, Bz, i, j - 1, k)) / dy;
                double dBy_dz = (o_get(s, By, i, j, k) - o_get(s, By, i, j, k - 1)) / dz;
                double dBx_dz = (o_get(s, Bx, i, j, k) - o_get(s, Bx, i, j, k - 1)) / dz;
                double dBz_dx = (o_get(s, Bz, i, j, k) - o_get(s, Bz, i - 1, j, k)) / dx;
                double dBy_dx = (o_get(s, By, i, j, k) - o_get(s, By, i - 1, j, k)) / dx;
                double dBx_dy = (o_get(s, Bx, i, j, k) - o_get(s, Bx, i, j - 1, k)) / dy;
                /* E_x at (i+1/2, j, k), E_y at (i, j+1/2, k), E_z at (i, j, k+1/2) */
                double sy = s->sig_node[1][j], sz = s->sig_node[2][k], sx = s->sig_node[0][i];
                if (sy > 0) { double b = o_b(sy, dt); s->psiE[0][1][ix] = b * s->psiE[0][1][ix] + (b - 1) * dBz_dy; dBz_dy += s->psiE[0][1][ix]; }
                if (sz > 0) { double b = o_b(sz, dt); s->psiE[0][2][ix] = b * s->psiE[0][2][ix] + (b - 1) * dBy_dz; dBy_dz += s->psiE[0][2][ix]; }
                if (sz > 0) { double b = o_b(sz, dt); s->psiE[1][2][ix] = b * s->psiE[1][2][ix] + (b - 1) * dBx_dz; dBx_dz += s->psiE[1][2][ix]; }
                if (sx > 0) { double b = o_b(sx, dt); s->psiE[1][0][ix] = b * s->psiE[1][0][ix] + (b - 1) * dBz_dx; dBz_dx += s->psiE[1][0][ix]; }
                if (sx > 0) { double b = o_b(sx, dt); s->psiE[2][0][ix] = b * s->psiE[2][0][ix] + (b - 1) * dBy_dx; dBy_dx += s->psiE[2][0][ix]; }
                if (sy > 0) { double b = o_b(sy, dt); s->psiE[2][1][ix] = b * s->psiE[2][1][ix] + (b - 1) * dBx_dy; dBx_dy += s->psiE[2][1][ix]; }
                s->F[O_EX][ix] += dt * (dBz_dy - dBy_dz - s->F[O_JX][ix]);
                s->F[O_EY][ix] += dt * (dBx_dz - dBz_dx - s->F[O_JY][ix]);
                s->F[O_EZ][ix] += dt * (dBy_dx - dBx_dy - s->F[O_JZ][ix]);
            }
}

/* Field part of one step: B^{n+1/2} = B^n - dt/2 curl E^n; E^{n+1} = E^n + dt (curl B^{n+1/2} - J);
 * B^{n+1} = B^{n+1/2} - dt/2 curl E^{n+1}. */
void osim_fdtd(void *h)
{
    osim *s = (osim *)h;
    o_update_B(s, 0.5 * s->dt);
    o_update_E(s);
    o_update_B(s, 0.5 * s->dt);
}

/* Moving window: shift every grid array down by one z plane, zero the new front plane,
 * move particles by -1 cell in z and drop those that leave the window. */
static void o_window_shift(osim *s)
{
    long plane = (long)s->n[0] * s->n[1], nz = s->n[2];
    double *arr[9 + 18];
    int na = 0;
    for (int f = 0; f < 9; f++) arr[na++] = s->F[f];
    for (int c = 0; c < 3; c++)
        for (int d = 0; d < 3; d++) { arr[na++] = s->psiE[c][d]; arr[na++] = s->psiB[c][d]; }
    for (int a = 0; a < na; a++) {
        memmove(arr[a], arr[a] + plane, (nz - 1) * plane * sizeof(double));
        memset(arr[a] + (nz - 1) * plane, 0, plane * sizeof(double));
    }
    for (int q = 0; q < s->nsp; q++) {
        osp *p = &s->sp[q];
        for (long i = 0; i < p->n; i++) {
            if (!p->alive[i]) continue;
            p->X[3 * i + 2] -= 1.0;
            if (!o_inside(s, &p->X[3 * i])) p->alive[i] = 0;
        }
    }
    if (s->ion_G) {
        /* the artificial ions move with the window: the z prefix of the shifted density is the old
         * prefix one plane up minus the dropped plane's part; no ions enter at the front */
        for (long c = 0; c < plane; c++) {
            double g0 = s->ion_G[c];
            for (long k = 0; k + 1 < nz; k++) s->ion_G[k * plane + c] = s->ion_G[(k + 1) * plane + c] - g0;
            if (nz > 1) s->ion_G[(nz - 1) * plane + c] = s->ion_G[(nz - 2) * plane + c];
        }
    }
    s->shifts++;
}

/* Number of window shifts due by step n: floor(v_w n dt / dz). */
static long o_shifts_due(const osim *s, long n)
{
    return (long)floor(s->vw * (double)n * s->dt / s->d[2]);
}

/* One full PIC step in the RRF: particles (gather E^n, B^n; push; move; deposit J^{n+1/2}),
 * then fields to n+1; then the window and the plasma are brought to time n+1 (window shifts
 * due by then, lattice planes that crossed the front threshold injected), so that the state
 * at every time n has floor(v_w n dt / dz) shifts and its full plasma lattice. */
/* Current of the fading artificial ions during step n (t_n to t_n + dt): the part of the ramp
 * the step covers, as a step average. */
static void o_ion_current(osim *s)
{
    if (!s->ion_G) return;
    double t0 = (double)s->step * s->dt, t1 = t0 + s->dt;
    double a = t0 > s->ion_t0 ? t0 : s->ion_t0, b = t1 < s->ion_t0 + s->ion_T ? t1 : s->ion_t0 + s->ion_T;
    if (b <= a) return;
    double f = (b - a) / (s->ion_T * s->dt);
    for (long i = 0; i < s->ncell; i++) s->F[O_JZ][i] += f * s->ion_G[i];
}

static void o_step(osim *s)
{
    for (int f = O_JX; f <= O_JZ; f++) memset(s->F[f], 0, s->ncell * sizeof(double));
    for (int q = 0; q < s->nsp; q++) o_push_species(s, &s->sp[q]);
    o_ion_current(s);
    osim_fdtd(s);
    s->step++;
    if (s->moving) {
        long due = o_shifts_due(s, s->step);
        while (s->shifts < due) o_window_shift(s);
    }
    if (s->plasma && s->bc[2][0] != O_PERIODIC) {
        long m1 = o_plane_max(s, s->step, s->shifts);
        o_inject_planes(s, s->m_last + 1, m1);
        if (m1 > s->m_last) s->m_last = m1;
    }
}

void osim_step(void *h, long nsteps)
{
    osim *s = (osim *)h;
    for (long i = 0; i < nsteps; i++) o_step(s);
}

long osim_dropped(void *h) { return ((osim *)h)->dropped; }

/* Charge density at the nodes, rho = sum q w S(node - X) / V, with the deposit's shape: of
 * species `only`, or of every live species when only < 0. */
static void o_rho(const osim *s, int only, double *rho)
{
    memset(rho, 0, s->ncell * sizeof(double));
    double V = s->d[0] * s->d[1] * s->d[2], h2 = 0.5 * (s->order + 1);
    for (int q = 0; q < s->nsp; q++) {
        if (only >= 0 && q != only) continue;
        const osp *p = &s->sp[q];
        for (long i = 0; i < p->n; i++) {
            if (!p->alive[i]) continue;
            const double *X = &p->X[3 * i];
            long lo[3], cnt[3];
            double wv[3][6];
            for (int d = 0; d < 3; d++) {
                lo[d] = (long)floor(X[d] - h2);
                cnt[d] = (long)floor(X[d] + h2) - lo[d] + 1;
                for (long a = 0; a < cnt[d]; a++) wv[d][a] = o_shape(s->order, (double)(lo[d] + a) - X[d]);
            }
            for (long c = 0; c < cnt[2]; c++)
                for (long b = 0; b < cnt[1]; b++)
                    for (long a = 0; a < cnt[0]; a++) {
                        long ix = o_index(s, lo[0] + a, lo[1] + b, lo[2] + c);
                        if (ix >= 0) rho[ix] += p->q * p->W[i] * wv[0][a] * wv[1][b] * wv[2][c] / V;
                    }
        }
    }
}

void osim_rho(void *h, double *rho) { o_rho((const osim *)h, -1, rho); }

/* Artificial neutralising ions (Sec. "Electron propagation in vacuum and under external field"):
 * a static background compensating the charge of species spi at the current time, faded
 * linearly to zero over T (the paper's T_ion).  Reading: a charge can only fade in a
 * charge-conserving scheme through a current, so the ions carry J_z with div J = -d rho_ion/dt:
 * J_z(i, j, k + 1/2) = -(dz / T) sum_{k' <= k} rho'(i, j, k'), the prefix along z from the low
 * face, while they fade.  rho' is the species' density; on a periodic z it is taken relative to
 * each column's mean (the net column charge of a periodic box cannot leave it: that mean stays as
 * the usual uniform neutralising background).  Fields start consistent: E = 0 with total charge
 * zero.  T <= 0 removes the ions at once (no current). */
void osim_set_ion_ramp(void *h, int spi, double T)
{
    osim *s = (osim *)h;
    free(s->ion_G);
    s->ion_G = NULL;
    if (!(T > 0.0)) return;
    double *rho = (double *)malloc(s->ncell * sizeof(double));
    o_rho(s, spi, rho);
    s->ion_G = (double *)calloc(s->ncell, sizeof(double));
    long nx = s->n[0], ny = s->n[1], nz = s->n[2];
    int zper = s->bc[2][0] == O_PERIODIC;
    for (long j = 0; j < ny; j++)
        for (long i = 0; i < nx; i++) {
            double mean = 0.0;
            if (zper) {
                for (long k = 0; k < nz; k++) mean += rho[(k * ny + j) * nx + i];
                mean /= (double)nz;
            }
            double acc = 0.0;
            for (long k = 0; k < nz; k++) {
                acc += rho[(k * ny + j) * nx + i] - mean;
                s->ion_G[(k * ny + j) * nx + i] = -s->d[2] * acc;
            }
        }
    free(rho);
    s->ion_t0 = (double)s->step * s->dt;
    s->ion_T = T;
}

/* Discrete divergence of E at the nodes (backward differences matching the Yee stagger). */
void osim_divE(void *h, double *out)
{
    osim *s = (osim *)h;
    for (long k = 0; k < s->n[2]; k++)
        for (long j = 0; j < s->n[1]; j++)
            for (long i = 0; i < s->n[0]; i++) {
                long ix = (k * s->n[1] + j) * s->n[0] + i;
                out[ix] = (o_get(s, s->F[O_EX], i, j, k) - o_get(s, s->F[O_EX], i - 1, j, k)) / s->d[0] +
                          (o_get(s, s->F[O_EY], i, j, k) - o_get(s, s->F[O_EY], i, j - 1, k)) / s->d[1] +
                          (o_get(s, s->F[O_EZ], i, j, k) - o_get(s, s->F[O_EZ], i, j, k - 1)) / s->d[2];
            }
}

/* Single-particle Esirkepov deposit into a zeroed J (unit tests of the deposit alone). */
void osim_deposit_one(void *h, double qw, const double *X0, const double *X1)
{
    osim *s = (osim *)h;
    for (int f = O_JX; f <= O_JZ; f++) memset(s->F[f], 0, s->ncell * sizeof(double));
    double *const J[3] = {s->F[O_JX], s->F[O_JY], s->F[O_JZ]};
    o_esirkepov(s, J, &s->dropped, qw, X0, X1);
}

/* Gather of all six field components at X (unit tests of the gather alone). */
void osim_gather_at(void *h, const double *X, double *EB)
{
    osim *s = (osim *)h;
    for (int c = 0; c < 6; c++) EB[c] = o_gather(s, s->F[c], O_STAG[c], X);
}

/* ------------------------------------------------------------------ sort */

/* Sort key of a particle at grid coordinate X: tiles of tx*ty*tz cells in x-fastest order;
 * inside a tile the cells in (x fastest, then z, then y) order; inside a cell the octant of
 * the in-cell offset (bit 0: frac(x) >= 1/2, bit 1: frac(y) >= 1/2, bit 2: frac(z) >= 1/2).
 * The sort reorders particles by ascending key; among equal keys the original order is kept
 * (stable), so the result is a plain definition to compare against. */
static long o_tile_key(const int n[3], const int T[3], const double X[3])
{
    long c[3];
    int oct = 0;
    for (int d = 0; d < 3; d++) {
        double fl = floor(X[d]);
        c[d] = (long)fl;
        if (X[d] - fl >= 0.5) oct |= 1 << d;
    }
    long ntx = (n[0] + T[0] - 1) / T[0], nty = (n[1] + T[1] - 1) / T[1];
    long tile = ((c[2] / T[2]) * nty + (c[1] / T[1])) * ntx + (c[0] / T[0]);
    long local = ((c[1] % T[1]) * T[2] + (c[2] % T[2])) * T[0] + (c[0] % T[0]);
    return (tile * (long)T[0] * T[1] * T[2] + local) * 8 + oct;
}

typedef struct { long key, idx; } o_kv;
static int o_kv_cmp(const void *a, const void *b)
{
    const o_kv *x = (const o_kv *)a, *y = (const o_kv *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

void oracle_tile_sort(long n, const double *X /*[3n] grid coordinates*/, const int *grid3, const int *tile3,
                      long *order_out, long *keys_out)
{
    o_kv *kv = (o_kv *)malloc((n > 0 ? n : 1) * sizeof(o_kv));
    for (long p = 0; p < n; p++) {
        kv[p].key = o_tile_key(grid3, tile3, &X[3 * p]);
        kv[p].idx = p;
    }
    qsort(kv, n, sizeof(o_kv), o_kv_cmp);
    for (long p = 0; p < n; p++) { order_out[p] = kv[p].idx; keys_out[p] = kv[p].key; }
    free(kv);
}

/* ------------------------------------------------------------------ diagnostics */

enum {
    OM_COUNT = 0, OM_SUMW, OM_CHARGE, OM_MX, OM_MY, OM_MZ, OM_SX, OM_SY, OM_SZ,
    OM_MUX, OM_MUY, OM_MUZ, OM_MG, OM_SG_REL, OM_EMX, OM_EMY, OM_BUNCH, OM_EKIN, OM_MT,
    OM_EFIELD, OM_N
};

/* Weighted statistics of m particles (weights w summing to sw > 0): means, rms sizes, mean
 * momenta and gamma, relative energy spread, normalised emittances sqrt(<dx^2><du^2> -
 * <dx du>^2) from central weighted moments, kinetic energy sum w mass (gamma - 1) and bunching
 * |sum w exp(-i k z)| / sum w. */
static void o_beam_stats(long m, const double *w, double sw, const double *x, const double *y, const double *z,
                         const double *ux, const double *uy, const double *uz, const double *g, double mass,
                         double k, double *out)
{
    double mean[7] = {0};
    const double *cols[7] = {x, y, z, ux, uy, uz, g};
    for (int q = 0; q < 7; q++) {
        for (long i = 0; i < m; i++) mean[q] += w[i] * cols[q][i];
        mean[q] /= sw;
    }
    double vx = 0, vy = 0, vz = 0, vux = 0, vuy = 0, cxu = 0, cyu = 0, vg = 0, ek = 0;
    double cr = 0, ci = 0;
    for (long i = 0; i < m; i++) {
        double dxx = x[i] - mean[0], dyy = y[i] - mean[1], dzz = z[i] - mean[2];
        double dux = ux[i] - mean[3], duy = uy[i] - mean[4], dg = g[i] - mean[6];
        vx += w[i] * dxx * dxx; vy += w[i] * dyy * dyy; vz += w[i] * dzz * dzz;
        vux += w[i] * dux * dux; vuy += w[i] * duy * duy;
        cxu += w[i] * dxx * dux; cyu += w[i] * dyy * duy;
        vg += w[i] * dg * dg;
        ek += w[i] * mass * (g[i] - 1.0);
        cr += w[i] * cos(k * z[i]);
        ci += -w[i] * sin(k * z[i]);
    }
    vx /= sw; vy /= sw; vz /= sw; vux /= sw; vuy /= sw; cxu /= sw; cyu /= sw; vg /= sw;
    out[OM_MX] = mean[0]; out[OM_MY] = mean[1]; out[OM_MZ] = mean[2];
    out[OM_SX] = sqrt(vx); out[OM_SY] = sqrt(vy); out[OM_SZ] = sqrt(vz);
    out[OM_MUX] = mean[3]; out[OM_MUY] = mean[4]; out[OM_MUZ] = mean[5];
    out[OM_MG] = mean[6];
    out[OM_SG_REL] = sqrt(vg) / mean[6];
    double ex = vx * vux - cxu * cxu, ey = vy * vuy - cyu * cyu;
    out[OM_EMX] = sqrt(ex > 0 ? ex : 0);
    out[OM_EMY] = sqrt(ey > 0 ? ey : 0);
    out[OM_BUNCH] = sqrt(cr * cr + ci * ci) / sw;
    out[OM_EKIN] = ek;
}

/* Weighted beam moments of species spi.  frame 0: RRF at t' = step dt (positions in
 * normalised RRF length, z' absolute).  frame 1: lab — each particle's event (z', t') and
 * momentum are transformed back (inverse Eq. Lor1-Lor2) and drifted ballistically to the
 * weighted mean lab time (the time spread of one RRF instant is Eq. DT).  Bunching
 * |sum w exp(-i k z)| / sum w at wavenumber k (lab k in frame 1, RRF k' in frame 0).
 * Normalised emittance sqrt(<dx^2><du^2> - <dx du>^2) with central weighted moments. */
void osim_moments(void *h, int spi, int frame, double k, double *out)
{
    osim *s = (osim *)h;
    osp *p = &s->sp[spi];
    memset(out, 0, OM_N * sizeof(double));
    long n = p->n;
    double *x = (double *)malloc((n > 0 ? n : 1) * 8 * sizeof(double));
    double *y = x + n, *z = x + 2 * n, *ux = x + 3 * n, *uy = x + 4 * n, *uz = x + 5 * n, *g = x + 6 * n, *t = x + 7 * n;
    double tp = (double)s->step * s->dt;
    long m = 0;
    for (long i = 0; i < n; i++) {
        if (!p->alive[i]) continue;
        double xp[3] = {p->X[3 * i] * s->d[0], p->X[3 * i + 1] * s->d[1], (p->X[3 * i + 2] + (double)s->shifts) * s->d[2]};
        double up[3] = {p->U[3 * i], p->U[3 * i + 1], p->U[3 * i + 2]};
        if (frame == 0) {
            x[m] = xp[0]; y[m] = xp[1]; z[m] = xp[2]; t[m] = tp;
            ux[m] = up[0]; uy[m] = up[1]; uz[m] = up[2];
        } else {
            double xl[3], ul[3], tl;
            oracle_boosted_to_lab(s->gR, xp, tp, up, xl, &tl, ul);
            x[m] = xl[0]; y[m] = xl[1]; z[m] = xl[2]; t[m] = tl;
            ux[m] = ul[0]; uy[m] = ul[1]; uz[m] = ul[2];
        }
        g[m] = sqrt(1.0 + ux[m] * ux[m] + uy[m] * uy[m] + uz[m] * uz[m]);
        m++;
    }
    /* weights of the live particles in the same order */
    double *w = (double *)malloc((m > 0 ? m : 1) * sizeof(double));
    long c = 0;
    for (long i = 0; i < n; i++) if (p->alive[i]) w[c++] = p->W[i];
    double sw = 0.0;
    for (long i = 0; i < m; i++) sw += w[i];
    out[OM_COUNT] = (double)m;
    out[OM_SUMW] = sw;
    out[OM_CHARGE] = p->q * sw;
    if (m > 0 && sw > 0.0) {
        double mt = 0.0;
        for (long i = 0; i < m; i++) mt += w[i] * t[i];
        mt /= sw;
        if (frame == 1) {
            for (long i = 0; i < m; i++) {
                double dtl = mt - t[i];
                x[i] += dtl * ux[i] / g[i];
                y[i] += dtl * uy[i] / g[i];
                z[i] += dtl * uz[i] / g[i];
            }
        }
        o_beam_stats(m, w, sw, x, y, z, ux, uy, uz, g, p->m, k, out);
        out[OM_MT] = mt;
    }
    double fe = 0.0;
    for (int f = O_EX; f <= O_BZ; f++)
        for (long i = 0; i < s->ncell; i++) fe += s->F[f][i] * s->F[f][i];
    out[OM_EFIELD] = 0.5 * fe * s->d[0] * s->d[1] * s->d[2];
    free(w);
    free(x);
}

/* Moments of the recorded lab snapshot (statistics of o_beam_stats; lab wavenumber k; mean_t is
 * the snapshot's lab time, field_energy 0). */
void osim_snapshot_moments(void *h, double k, double *out)
{
    osim *s = (osim *)h;
    memset(out, 0, OM_N * sizeof(double));
    long m = 0;
    for (long i = 0; i < s->snap_n; i++) m += s->snap_state[i] == 1;
    double *buf = (double *)malloc((m > 0 ? m : 1) * 8 * sizeof(double));
    double *x = buf, *y = x + m, *z = y + m, *ux = z + m, *uy = ux + m, *uz = uy + m, *g = uz + m, *w = g + m;
    long c = 0;
    double sw = 0.0;
    for (long i = 0; i < s->snap_n; i++) {
        if (s->snap_state[i] != 1) continue;
        const double *r = &s->snap[7 * i];
        x[c] = r[0]; y[c] = r[1]; z[c] = r[2]; ux[c] = r[3]; uy[c] = r[4]; uz[c] = r[5]; w[c] = r[6];
        g[c] = sqrt(1.0 + r[3] * r[3] + r[4] * r[4] + r[5] * r[5]);
        sw += w[c];
        c++;
    }
    const osp *p = &s->sp[s->snap_sp];
    out[OM_COUNT] = (double)m;
    out[OM_SUMW] = sw;
    out[OM_CHARGE] = p->q * sw;
    if (m > 0 && sw > 0.0) o_beam_stats(m, w, sw, x, y, z, ux, uy, uz, g, p->m, k, out);
    out[OM_MT] = s->snap_T;
    free(buf);
}

/* ------------------------------------------------------------------ resonance */

/* FEL resonant wavelength lambda_l = lambda_u (1 + K^2/2) / (2 gamma_B^2)  (Eq. RadLambda). */
double oracle_resonant_wavelength(double lambda_u, double K, double gamma_B)
{
    return lambda_u * (1.0 + 0.5 * K * K) / (2.0 * gamma_B * gamma_B);
}

/* Wavelength seen in the RRF of a wave travelling along the boost:
 * lambda' = lambda sqrt((1 + beta_R)/(1 - beta_R))  (Eq. Uelon, exact form). */
double oracle_doppler_rrf(double lambda, double gamma_R)
{
    double b = sqrt(1.0 - 1.0 / (gamma_R * gamma_R));
    return lambda * sqrt((1.0 + b) / (1.0 - b));
}

/* Beam length in the RRF (Eq. Belon): sigma' = sigma gamma_B / (gamma_B gamma_R -
 * sqrt(gamma_B^2 - 1) sqrt(gamma_R^2 - 1)). */
double oracle_beam_elongation(double gamma_B, double gamma_R)
{
    return gamma_B / (gamma_B * gamma_R - sqrt(gamma_B * gamma_B - 1.0) * sqrt(gamma_R * gamma_R - 1.0));
}
