/*
 * FP64 CPU oracle of the diffuse-interface lattice Boltzmann method (DI-LBM)
 * for fluid-particle interaction (Liu, Huang, Chai & Shi, arXiv:2106.08950).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product path never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Every step follows the paper's procedure (Sec. 2.3) literally, in double
 * precision, with an explicit loop over the nine lattice directions:
 *   1. solid fraction phi (Eq. 14) at every node from every particle;
 *   2. pull streaming of the post-collision populations (Eq. 13, left side),
 *      then non-equilibrium extrapolation on the domain edges (Sec. 3, the
 *      boundary scheme of Guo et al. 2002);
 *   3. density and uncorrected velocity u* (Eq. 5, Eq. 16);
 *   4. corrected velocity u = u* + phi (u_s - u*) / 2 (Eq. 17);
 *   5. equilibrium f^eq(rho, u) (Eq. 2);
 *   6. discrete force term F_i (Eq. 15);
 *   7. collision f' = f - (f - f^eq)/tau + phi F_i (Eq. 13);
 *   8. hydrodynamic force and torque by explicit double sums (Eqs. 18-19);
 *   9. Newton-Euler update of each free particle (Eqs. 22-24) with the
 *      Wan-Turek short-range repulsion (Eqs. 28-29).
 *
 * Readings where the paper is silent (the same ones the CUDA path takes):
 *   - l in Eq. 14 is the signed distance r - |x - X|, positive inside;
 *   - several particles: phi = max over particles, the owner is the argmax
 *     (lowest index on ties); a node's force goes to its owner only;
 *   - u_s at a node is the rigid-body velocity U + omega x (x - X);
 *   - f^eq in Eq. 13 takes the corrected velocity of Eq. 17;
 *   - phi, u_s and X at the start of a step are used for the whole step,
 *     then the particles advance (symplectic Euler, dt = 1);
 *   - m = rho_s pi r^2, I = m r^2 / 2 (a disc of unit depth); gravity g is
 *     the physical acceleration (pointing down for settling), so the
 *     buoyancy-reduced weight is (1 - rho_f/rho_s) m g (Eq. 22 up to the
 *     sign convention of g);
 *   - force_model 0 uses Eq. 18 as printed; force_model 1 uses the momentum
 *     the collision hands to the fluid, -sum_i c_i (f'_i - f_i);
 *   - initial populations are f^eq(rho_init, u0) everywhere.
 *
 * method 1 replaces steps 1, 4-8 by the paper's comparison method, the
 * partially saturated LBM with the SP collision (Sec. 2.2):
 *   1'. solid volume fraction eps_s of every node's unit cell, the exact area
 *       of the cell covered by the disc (the paper requires it and gives no
 *       algorithm: here the integral of the covered chord length over the
 *       cell's width, in closed form), B = eps_s (Eq. 8);
 *   5'-7'. f' = f + (1 - B)(-(f - f^eq(rho, u*))/tau) + B Omega^s with the
 *       additional collision term Omega^s of Eq. 9 (f^eq takes the fluid
 *       velocity u*: there is no correction step);
 *   8'. force and torque by the double sums of Eqs. 10-11.
 * The same max rule picks a node's owner (the largest covered fraction).
 *
 * Moving computational domain (Sec. 3.5, after Wang et al. 2013): the paper
 * moves the domain one lattice unit whenever the tracked particle has moved
 * one lattice unit, and gives no further detail.  Reading: at the end of a
 * step, with d the tracked particle's x at the start of that step minus the
 * reference x_ref (minimum image on a periodic x axis), the frame moves by
 * s = +1 column if d >= 1, by -1 if d <= -1, else not at all.  Moving by s
 * takes the post-collision populations of column x + s to column x (on a
 * periodic axis the columns roll; otherwise the entering column repeats its
 * neighbour, a zero-gradient state that the edge scheme then overwrites),
 * subtracts s from every particle's new x and adds s to the frame offset.
 * The move is plain: in a pressure-driven channel it displaces the linear
 * pressure field by one column against the fixed end densities (a step of
 * (rho_in - rho_out) / (nx - 1)), which the ends re-absorb acoustically.
 *
 * Memory layout: populations f[i][y][x], x fastest, i = 0..8 in the order of
 * Eq. 3: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Eq. 3: the D2Q9 velocities. */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* Eq. 4: the weights. */
static const double W[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* Sound speed squared in lattice units (dx = dt = 1). */
static const double CS2 = 1.0 / 3.0;

enum { SIDE_PERIODIC = 0, SIDE_VELOCITY = 1, SIDE_PRESSURE = 2 };
enum { WEST = 0, EAST = 1, SOUTH = 2, NORTH = 3 };

typedef struct {
    int nx, ny;
    int side_kind[4];            /* west, east, south, north */
    double side_ux[4], side_uy[4], side_rho[4];
    double tau;                  /* relaxation time, Eq. 1 */
    double eps;                  /* interface width, Eq. 14 */
    double gx, gy;               /* gravity acting on the particles, Eq. 22 */
    double rho_f;                /* fluid density in the buoyancy term, Eq. 22 */
    double rho_init, u0x, u0y;   /* initial state */
    int force_model;             /* 0: Eq. 18 as printed, 1: momentum exchange */
    double eps_p, eps_p2, eps_w, eps_w2, xi;  /* Eqs. 28-29 */
    double phi_cutoff;           /* 0: every particle at every node; > 0: a particle
                                    reaches only nodes with l >= -phi_cutoff */
    int method;                  /* 0: DI-LBM (Eq. 13); 1: PS-LBM with the SP collision (Eqs. 7-11) */
} orc_params;

typedef struct {
    double x, y, r, ux, uy, omega, theta, rho_s;
    int fixed;
} orc_particle;

typedef struct {
    orc_params p;
    int np;
    orc_particle *parts;
    double *f;          /* post-collision populations, 9 planes */
    double *fpre;       /* streamed (pre-collision) populations */
    double *phi;        /* solid fraction per node */
    int *owner;         /* owning particle per node, -1 if none */
    double *usx, *usy;  /* particle velocity at the node */
    double *rx, *ry;    /* node position relative to the owner (min-image) */
    double *gx, *gy;    /* per-node hydrodynamic force on the owner */
    double *force;      /* np x 3: Fx, Fy, T of the last step */
    double *fcol;       /* np x 2: Wan-Turek force of the last step */
    long long steps;
    int track;          /* moving frame: tracked particle, -1 when off */
    double track_x;     /* its reference x in the frame */
    long long offset;   /* columns the frame has moved (x_lab = x + offset) */
} orc_sim;

/* ---------------------------------------------------------------- helpers */

static int periodic_x(const orc_params *p) { return p->side_kind[WEST] == SIDE_PERIODIC; }
static int periodic_y(const orc_params *p) { return p->side_kind[SOUTH] == SIDE_PERIODIC; }

/* Minimum-image displacement along a periodic axis of length L. */
static double min_image(double d, double L)
{
    while (d >= 0.5 * L) d -= L;
    while (d < -0.5 * L) d += L;
    return d;
}

/* Eq. 2: equilibrium populations. */
void orc_equilibrium(double rho, double ux, double uy, double feq[9])
{
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        feq[i] = W[i] * rho * (1.0 + cu / CS2 + (cu * cu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Eq. 14: solid fraction from the signed distance l (positive inside). */
double orc_phi(double l, double eps)
{
    return 0.5 * (1.0 + tanh(2.0 * l / eps));
}

/* Eq. 15: the discrete force term, written with the full tensor contraction
 * (u_s u_s - u* u*) : (c_i c_i - cs^2 I). */
void orc_force_term(double tau, double rho, double usx_, double usy_, double uax, double uay,
                    double Fi[9])
{
    double us[2] = {usx_, usy_};
    double ua[2] = {uax, uay};
    double A[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            A[a][b] = us[a] * us[b] - ua[a] * ua[b];
    for (int i = 0; i < 9; ++i) {
        double c[2] = {(double)CX[i], (double)CY[i]};
        double cdu = c[0] * (us[0] - ua[0]) + c[1] * (us[1] - ua[1]);
        double contr = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                contr += A[a][b] * (c[a] * c[b] - CS2 * (a == b ? 1.0 : 0.0));
        Fi[i] = (1.0 - 1.0 / (2.0 * tau)) * W[i] * rho *
                (cdu / CS2 + contr / (2.0 * CS2 * CS2));
    }
}

/* Steps 3-7 at one node.  mom receives rho, u*x, u*y, ux, uy. */
void orc_collide_node(double tau, const double f[9], double phi, double usx_, double usy_,
                      double fout[9], double Fi[9], double mom[5])
{
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {       /* Eq. 5 / Eq. 16 */
        rho += f[i];
        jx += CX[i] * f[i];
        jy += CY[i] * f[i];
    }
    double uax = jx / rho, uay = jy / rho;
    double ux = uax + 0.5 * phi * (usx_ - uax);   /* Eq. 17 */
    double uy = uay + 0.5 * phi * (usy_ - uay);
    double feq[9];
    orc_equilibrium(rho, ux, uy, feq);           /* Eq. 2 with the corrected u */
    orc_force_term(tau, rho, usx_, usy_, uax, uay, Fi);   /* Eq. 15 */
    for (int i = 0; i < 9; ++i)                  /* Eq. 13 */
        fout[i] = f[i] - (f[i] - feq[i]) / tau + phi * Fi[i];
    mom[0] = rho; mom[1] = uax; mom[2] = uay; mom[3] = ux; mom[4] = uy;
}

/* Solid volume fraction for the PS-LBM (Sec. 2.2): the area of the unit cell
 * [dx - 1/2, dx + 1/2] x [dy - 1/2, dy + 1/2] covered by the disc of radius r
 * centred at the origin.  The area is the integral over the cell's width of
 * the covered length of the vertical line at x,
 *   L(x) = max(0, min(y1, h(x)) - max(y0, -h(x))),  h(x) = sqrt(r^2 - x^2),
 * which on each piece between the abscissae where h crosses y0 or y1 is
 * 0, y1 - y0, h - y0, y1 + h or 2h; the integral of h has the closed form
 * (x h + r^2 asin(x / r)) / 2.  h is formed as sqrt((r - x)(r + x)) and
 * asin(x / r) as atan2(x, h), which stay accurate where x approaches r. */
static double half_chord(double x, double r) { return sqrt((r - x) * (r + x)); }

static double int_h(double x, double r)
{
    if (x <= -r) return -0.25 * M_PI * r * r;
    if (x >= r) return 0.25 * M_PI * r * r;
    double h = half_chord(x, r);
    return 0.5 * (x * h + r * r * atan2(x, h));
}

double orc_cell_fraction(double dx, double dy, double r)
{
    double x0 = dx - 0.5, x1 = dx + 0.5, y0 = dy - 0.5, y1 = dy + 0.5;
    if (x0 < -r) x0 = -r;
    if (x1 > r) x1 = r;
    if (x0 >= x1) return 0.0;
    /* breakpoints: |x| where h(x) = |y0| or |y1| */
    double br[6];
    int nb = 0;
    br[nb++] = x0;
    const double ys[2] = {y0, y1};
    for (int k = 0; k < 2; ++k) {
        if (fabs(ys[k]) < r) {
            double xb = half_chord(fabs(ys[k]), r);
            if (xb > x0 && xb < x1) br[nb++] = xb;
            if (-xb > x0 && -xb < x1) br[nb++] = -xb;
        }
    }
    br[nb++] = x1;
    for (int a = 1; a < nb; ++a)              /* sort the few breakpoints */
        for (int b = a; b > 0 && br[b] < br[b - 1]; --b) {
            double t = br[b]; br[b] = br[b - 1]; br[b - 1] = t;
        }
    double area = 0.0;
    for (int k = 0; k + 1 < nb; ++k) {
        double a = br[k], b = br[k + 1];
        if (b <= a) continue;
        double xm = 0.5 * (a + b), hm = half_chord(xm, r);
        /* with no breakpoint inside the piece, h - y1 and h + y0 keep their
         * sign on it (<=: a circle tangent to y1 at x = 0 touches it there only) */
        int top = hm <= y1;        /* the disc's upper edge lies inside the cell on this piece */
        int bot = -hm >= y0;       /* the lower edge does */
        double lo = bot ? -hm : y0, hi = top ? hm : y1;
        if (hi <= lo) continue;    /* the line misses the covered part */
        double ih = int_h(b, r) - int_h(a, r);
        if (top && bot) area += 2.0 * ih;
        else if (top) area += ih - y0 * (b - a);
        else if (bot) area += y1 * (b - a) + ih;
        else area += (y1 - y0) * (b - a);
    }
    return area;
}

/* Eq. 7 with the SP term Omega^s of Eq. 9 (B = eps_s, Eq. 8) at one node.
 * omega_s receives Omega^s; mom receives rho, u*x, u*y. */
void orc_collide_node_ps(double tau, const double f[9], double B, double usx_, double usy_,
                         double fout[9], double omega_s[9], double mom[3])
{
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        rho += f[i];
        jx += CX[i] * f[i];
        jy += CY[i] * f[i];
    }
    double ux = jx / rho, uy = jy / rho;
    double feq[9], feqs[9];
    orc_equilibrium(rho, ux, uy, feq);
    orc_equilibrium(rho, usx_, usy_, feqs);
    for (int i = 0; i < 9; ++i) {
        omega_s[i] = feqs[i] - f[i] + (1.0 - 1.0 / tau) * (f[i] - feq[i]);
        fout[i] = f[i] + (1.0 - B) * (-(f[i] - feq[i]) / tau) + B * omega_s[i];
    }
    mom[0] = rho; mom[1] = ux; mom[2] = uy;
}

/* Eqs. 28-29: Wan-Turek repulsion on every particle from the others and from
 * the walls (mirror image of the centre across each non-periodic wall). */
void orc_wan_turek(const orc_params *p, const orc_particle *pt, int np, double *out)
{
    double Lx = p->nx, Ly = p->ny;
    for (int i = 0; i < np; ++i) {
        double fx = 0.0, fy = 0.0;
        for (int j = 0; j < np; ++j) {
            if (j == i) continue;
            double dx = pt[i].x - pt[j].x, dy = pt[i].y - pt[j].y;
            if (periodic_x(p)) dx = min_image(dx, Lx);
            if (periodic_y(p)) dy = min_image(dy, Ly);
            double d = sqrt(dx * dx + dy * dy);
            double rr = pt[i].r + pt[j].r;
            double s = 0.0;
            if (d <= rr)
                s = (rr - d) / p->eps_p2;
            else if (d <= rr + p->xi)
                s = (rr + p->xi - d) * (rr + p->xi - d) / p->eps_p;
            fx += s * dx;
            fy += s * dy;
        }
        /* walls lie on the first and last node column / row */
        for (int w = 0; w < 4; ++w) {
            if (p->side_kind[w] == SIDE_PERIODIC) continue;
            double ix = pt[i].x, iy = pt[i].y;
            if (w == WEST) ix = -pt[i].x;
            if (w == EAST) ix = 2.0 * (p->nx - 1) - pt[i].x;
            if (w == SOUTH) iy = -pt[i].y;
            if (w == NORTH) iy = 2.0 * (p->ny - 1) - pt[i].y;
            double dx = pt[i].x - ix, dy = pt[i].y - iy;
            double d = sqrt(dx * dx + dy * dy);
            double rr = 2.0 * pt[i].r;
            double s = 0.0;
            if (d <= rr)
                s = (rr - d) / p->eps_w2;
            else if (d <= rr + p->xi)
                s = (rr + p->xi - d) * (rr + p->xi - d) / p->eps_w;
            fx += s * dx;
            fy += s * dy;
        }
        out[2 * i] = fx;
        out[2 * i + 1] = fy;
    }
}

/* ------------------------------------------------------------ simulation */

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

orc_sim *orc_create(const orc_params *p, const orc_particle *parts, int np)
{
    if (p->nx < 3 || p->ny < 3 || p->tau <= 0.5 || p->eps <= 0.0 || np < 0) return NULL;
    if ((p->side_kind[WEST] == SIDE_PERIODIC) != (p->side_kind[EAST] == SIDE_PERIODIC)) return NULL;
    if ((p->side_kind[SOUTH] == SIDE_PERIODIC) != (p->side_kind[NORTH] == SIDE_PERIODIC)) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    size_t n = (size_t)p->nx * p->ny;
    s->p = *p;
    s->np = np;
    s->parts = (orc_particle *)calloc(np > 0 ? np : 1, sizeof(orc_particle));
    if (np > 0) memcpy(s->parts, parts, sizeof(orc_particle) * np);
    s->f = (double *)malloc(sizeof(double) * 9 * n);
    s->fpre = (double *)malloc(sizeof(double) * 9 * n);
    s->phi = (double *)malloc(sizeof(double) * n);
    s->owner = (int *)malloc(sizeof(int) * n);
    s->usx = (double *)malloc(sizeof(double) * n);
    s->usy = (double *)malloc(sizeof(double) * n);
    s->rx = (double *)malloc(sizeof(double) * n);
    s->ry = (double *)malloc(sizeof(double) * n);
    s->gx = (double *)malloc(sizeof(double) * n);
    s->gy = (double *)malloc(sizeof(double) * n);
    s->force = (double *)calloc(3 * (np > 0 ? np : 1), sizeof(double));
    s->fcol = (double *)calloc(2 * (np > 0 ? np : 1), sizeof(double));
    s->track = -1;
    double feq[9];
    orc_equilibrium(p->rho_init, p->u0x, p->u0y, feq);
    for (int i = 0; i < 9; ++i)
        for (size_t k = 0; k < n; ++k) s->f[i * n + k] = feq[i];
    return s;
}

/* Moving frame (Sec. 3.5): track `particle` (-1: off) about x_ref. */
int orc_set_moving_frame(orc_sim *s, int particle, double x_ref)
{
    if (particle < -1 || particle >= s->np || !isfinite(x_ref)) return -1;
    s->track = particle;
    s->track_x = x_ref;
    return 0;
}

long long orc_frame_offset(const orc_sim *s) { return s->offset; }

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    free(s->parts); free(s->f); free(s->fpre); free(s->phi); free(s->owner);
    free(s->usx); free(s->usy); free(s->rx); free(s->ry); free(s->gx); free(s->gy);
    free(s->force); free(s->fcol);
    free(s);
}

static void set_particle_velocity(orc_sim *s, size_t k)
{
    int own = s->owner[k];
    if (own >= 0) {
        const orc_particle *P = &s->parts[own];
        s->usx[k] = P->ux - P->omega * s->ry[k];
        s->usy[k] = P->uy + P->omega * s->rx[k];
    } else {
        s->usx[k] = 0.0;
        s->usy[k] = 0.0;
    }
}

/* Step 1 with a cutoff: each particle, in index order, visits the nodes of
 * its bounding box (radius + cutoff) and takes every node where its phi is
 * strictly larger than what earlier particles left: the same max rule and
 * tie order as the full sum, for the particles that reach the node. */
static void solid_fraction_cutoff(orc_sim *s)
{
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    for (size_t k = 0; k < n; ++k) { s->phi[k] = 0.0; s->owner[k] = -1; s->rx[k] = 0.0; s->ry[k] = 0.0; }
    for (int q = 0; q < s->np; ++q) {
        const orc_particle *P = &s->parts[q];
        double R = P->r + p->phi_cutoff;
        int x0 = (int)floor(P->x - R), x1 = (int)ceil(P->x + R);
        int y0 = (int)floor(P->y - R), y1 = (int)ceil(P->y + R);
        if (periodic_x(p)) {
            if (x1 - x0 + 1 > nx) { x0 = 0; x1 = nx - 1; }   /* else wrapped below */
        } else {
            if (x0 < 0) x0 = 0;
            if (x1 > nx - 1) x1 = nx - 1;
        }
        if (periodic_y(p)) {
            if (y1 - y0 + 1 > ny) { y0 = 0; y1 = ny - 1; }   /* else wrapped below */
        } else {
            if (y0 < 0) y0 = 0;
            if (y1 > ny - 1) y1 = ny - 1;
        }
#pragma omp parallel for schedule(static)
        for (int yy = y0; yy <= y1; ++yy) {
            int y = periodic_y(p) ? ((yy % ny) + ny) % ny : yy;
            for (int xx = x0; xx <= x1; ++xx) {
                int x = periodic_x(p) ? ((xx % nx) + nx) % nx : xx;
                size_t k = (size_t)y * nx + x;
                double dx = x - P->x, dy = y - P->y;
                if (periodic_x(p)) dx = min_image(dx, nx);
                if (periodic_y(p)) dy = min_image(dy, ny);
                double l = P->r - sqrt(dx * dx + dy * dy);
                if (l < -p->phi_cutoff) continue;
                double ph = orc_phi(l, p->eps);
                if (ph > s->phi[k]) {
                    s->phi[k] = ph; s->owner[k] = q; s->rx[k] = dx; s->ry[k] = dy;
                }
            }
        }
    }
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < (long long)n; ++k) set_particle_velocity(s, (size_t)k);
}

/* Step 1' (PS-LBM): B = eps_s, owner and u_s at every node.  A disc covers
 * no part of a cell whose centre is farther than r + sqrt(2)/2, so only
 * nearer particles are evaluated (this skips nothing). */
static void solid_fraction_ps(orc_sim *s)
{
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t k = (size_t)y * nx + x;
            double best = 0.0, brx = 0.0, bry = 0.0;
            int own = -1;
            for (int q = 0; q < s->np; ++q) {
                const orc_particle *P = &s->parts[q];
                double dx = x - P->x, dy = y - P->y;
                if (periodic_x(p)) dx = min_image(dx, nx);
                if (periodic_y(p)) dy = min_image(dy, ny);
                if (sqrt(dx * dx + dy * dy) > P->r + 0.7072) continue;
                double e = orc_cell_fraction(dx, dy, P->r);
                if (e > best) { best = e; own = q; brx = dx; bry = dy; }
            }
            s->phi[k] = best;
            s->owner[k] = own;
            s->rx[k] = brx;
            s->ry[k] = bry;
            set_particle_velocity(s, k);
        }
    }
}

/* Step 1: phi, owner and u_s at every node from the current particle state. */
static void solid_fraction(orc_sim *s)
{
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny;
    if (p->method == 1) {
        solid_fraction_ps(s);
        return;
    }
    if (p->phi_cutoff > 0.0) {
        solid_fraction_cutoff(s);
        return;
    }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t k = (size_t)y * nx + x;
            double best = 0.0, brx = 0.0, bry = 0.0;
            int own = -1;
            for (int q = 0; q < s->np; ++q) {
                const orc_particle *P = &s->parts[q];
                double dx = x - P->x, dy = y - P->y;
                if (periodic_x(p)) dx = min_image(dx, nx);
                if (periodic_y(p)) dy = min_image(dy, ny);
                double l = P->r - sqrt(dx * dx + dy * dy);
                double ph = orc_phi(l, p->eps);
                if (ph > best) {          /* strict: ties keep the lower index */
                    best = ph; own = q; brx = dx; bry = dy;
                }
            }
            s->phi[k] = best;
            s->owner[k] = own;
            s->rx[k] = brx;
            s->ry[k] = bry;
            set_particle_velocity(s, k);
        }
    }
}

/* Step 2: pull streaming into fpre, then non-equilibrium extrapolation. */
static void stream_and_boundaries(orc_sim *s)
{
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    int px = periodic_x(p), py = periodic_y(p);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            for (int i = 0; i < 9; ++i) {
                int sx = x - CX[i], sy = y - CY[i];
                if (px) sx = (sx + nx) % nx;
                if (py) sy = (sy + ny) % ny;
                double v = 0.0;   /* unknown: only on edge nodes, replaced below */
                if (sx >= 0 && sx < nx && sy >= 0 && sy < ny) v = s->f[i * n + (size_t)sy * nx + sx];
                s->fpre[i * n + (size_t)y * nx + x] = v;
            }
        }
    }
    if (px && py) return;
    /* Edge nodes: f(b) = f^eq(rho_b, u_b) + [f(n) - f^eq(rho_n, u_n)] with n the
     * inner neighbour (diagonal at corners).  A corner takes the condition of
     * its south/north side.  Neighbours are inner nodes, so every edge node
     * reads values that this loop does not change. */
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            int onx = !px && (x == 0 || x == nx - 1);
            int ony = !py && (y == 0 || y == ny - 1);
            if (!onx && !ony) continue;
            int side = ony ? (y == 0 ? SOUTH : NORTH) : (x == 0 ? WEST : EAST);
            int nxn = x, nyn = y;
            if (onx) nxn = (x == 0) ? 1 : nx - 2;
            if (ony) nyn = (y == 0) ? 1 : ny - 2;
            size_t kb = (size_t)y * nx + x, kn = (size_t)nyn * nx + nxn;
            double fn[9], rho_n = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < 9; ++i) {
                fn[i] = s->fpre[i * n + kn];
                rho_n += fn[i];
                jx += CX[i] * fn[i];
                jy += CY[i] * fn[i];
            }
            double unx = jx / rho_n, uny = jy / rho_n;
            double rho_b, ubx, uby;
            if (p->side_kind[side] == SIDE_VELOCITY) {
                rho_b = rho_n; ubx = p->side_ux[side]; uby = p->side_uy[side];
            } else {
                rho_b = p->side_rho[side]; ubx = unx; uby = uny;
            }
            double eb[9], en[9];
            orc_equilibrium(rho_b, ubx, uby, eb);
            orc_equilibrium(rho_n, unx, uny, en);
            for (int i = 0; i < 9; ++i) s->fpre[i * n + kb] = eb[i] + (fn[i] - en[i]);
        }
    }
}

/* The frame's move at the end of this step, from the tracked particle's x
 * at its start. */
static int frame_shift(const orc_sim *s)
{
    if (s->track < 0) return 0;
    double d = s->parts[s->track].x - s->track_x;
    if (periodic_x(&s->p)) d = min_image(d, s->p.nx);
    return d >= 1.0 ? 1 : (d <= -1.0 ? -1 : 0);
}

/* Column x takes the post-collision populations of column x + sh. */
static void shift_populations(orc_sim *s, int sh)
{
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    double *row = (double *)malloc(sizeof(double) * nx);
    for (int i = 0; i < 9; ++i) {
        for (int y = 0; y < ny; ++y) {
            double *f = s->f + i * n + (size_t)y * nx;
            memcpy(row, f, sizeof(double) * nx);
            for (int x = 0; x < nx; ++x) {
                int src = x + sh;
                if (periodic_x(p)) src = (src % nx + nx) % nx;
                else src = src < 0 ? 0 : (src > nx - 1 ? nx - 1 : src);
                f[x] = row[src];
            }
        }
    }
    free(row);
}

/* Steps 8-9: force/torque sums and the rigid-body update; then the frame
 * moves by sh columns. */
static void particles_update(orc_sim *s, int sh)
{
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    for (int q = 0; q < 3 * s->np; ++q) s->force[q] = 0.0;
    for (size_t k = 0; k < n; ++k) {          /* Eqs. 18-19, row-major order */
        int q = s->owner[k];
        if (q < 0) continue;
        s->force[3 * q] += s->gx[k];
        s->force[3 * q + 1] += s->gy[k];
        s->force[3 * q + 2] += s->rx[k] * s->gy[k] - s->ry[k] * s->gx[k];
    }
    orc_wan_turek(p, s->parts, s->np, s->fcol);
    for (int q = 0; q < s->np; ++q) {         /* Eqs. 22-24 */
        orc_particle *P = &s->parts[q];
        if (P->fixed) continue;
        double m = P->rho_s * M_PI * P->r * P->r;
        double I = 0.5 * m * P->r * P->r;
        /* Eq. 22 prints (rho_f/rho_s - 1) m g, which with g pointing down lifts a
         * heavy particle (Eq. 27 carries the same sign): g is read as the
         * physical acceleration and the buoyancy-reduced weight as
         * (1 - rho_f/rho_s) m g. */
        double buoy = (1.0 - p->rho_f / P->rho_s) * m;
        P->ux += (s->force[3 * q] + s->fcol[2 * q] + buoy * p->gx) / m;
        P->uy += (s->force[3 * q + 1] + s->fcol[2 * q + 1] + buoy * p->gy) / m;
        P->omega += s->force[3 * q + 2] / I;
        P->x += P->ux;
        P->y += P->uy;
        P->theta += P->omega;
        if (periodic_x(p)) { P->x = fmod(P->x, (double)nx); if (P->x < 0.0) P->x += nx; }
        if (periodic_y(p)) { P->y = fmod(P->y, (double)ny); if (P->y < 0.0) P->y += ny; }
    }
    if (sh) {
        for (int q = 0; q < s->np; ++q) {
            orc_particle *P = &s->parts[q];
            P->x -= sh;
            if (periodic_x(p)) { P->x = fmod(P->x, (double)nx); if (P->x < 0.0) P->x += nx; }
        }
        shift_populations(s, sh);
        s->offset += sh;
    }
}

int orc_step(orc_sim *s, long long nsteps)
{
    const orc_params *p = &s->p;
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * ny;
    for (long long t = 0; t < nsteps; ++t) {
        solid_fraction(s);
        stream_and_boundaries(s);
        int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                size_t k = (size_t)y * nx + x;
                double f[9], fo[9], Fi[9], mom[5];
                for (int i = 0; i < 9; ++i) f[i] = s->fpre[i * n + k];
                double gx = 0.0, gy = 0.0;
                if (p->method == 1) {               /* PS-LBM: Eq. 7, force of Eq. 10 */
                    orc_collide_node_ps(p->tau, f, s->phi[k], s->usx[k], s->usy[k], fo, Fi, mom);
                    if (!(mom[0] > 0.0) || !isfinite(mom[1]) || !isfinite(mom[2])) bad = 1;
                    for (int i = 0; i < 9; ++i) {
                        gx += Fi[i] * CX[i];
                        gy += Fi[i] * CY[i];
                    }
                    gx *= -s->phi[k];
                    gy *= -s->phi[k];
                    s->gx[k] = gx;
                    s->gy[k] = gy;
                    for (int i = 0; i < 9; ++i) s->f[i * n + k] = fo[i];
                    continue;
                }
                orc_collide_node(p->tau, f, s->phi[k], s->usx[k], s->usy[k], fo, Fi, mom);
                if (!(mom[0] > 0.0) || !isfinite(mom[1]) || !isfinite(mom[2])) bad = 1;
                if (p->force_model == 0) {          /* Eq. 18 as printed */
                    for (int i = 0; i < 9; ++i) {
                        gx += Fi[i] * CX[i];
                        gy += Fi[i] * CY[i];
                    }
                    gx *= -s->phi[k];
                    gy *= -s->phi[k];
                } else {                            /* momentum the fluid gained */
                    for (int i = 0; i < 9; ++i) {
                        gx -= CX[i] * (fo[i] - f[i]);
                        gy -= CY[i] * (fo[i] - f[i]);
                    }
                }
                s->gx[k] = gx;
                s->gy[k] = gy;
                for (int i = 0; i < 9; ++i) s->f[i * n + k] = fo[i];
            }
        }
        particles_update(s, frame_shift(s));
        s->steps++;
        if (bad) return -4;
    }
    return 0;
}

/* Macroscopic state at the current time level: the populations a next step
 * would collide (streamed, edges extrapolated), their density, the corrected
 * velocity of Eq. 17 and phi from the current particle state. */
void orc_fields(orc_sim *s, double *rho, double *ux, double *uy, double *phi, int *owner)
{
    const orc_params *p = &s->p;
    size_t n = (size_t)p->nx * p->ny;
    solid_fraction(s);
    stream_and_boundaries(s);
    for (size_t k = 0; k < n; ++k) {
        double r = 0.0, jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; ++i) {
            double v = s->fpre[i * n + k];
            r += v; jx += CX[i] * v; jy += CY[i] * v;
        }
        double uax = jx / r, uay = jy / r;
        if (rho) rho[k] = r;
        /* DI: the corrected velocity of Eq. 17; PS: the fluid velocity u* */
        double c = p->method == 1 ? 0.0 : 0.5 * s->phi[k];
        if (ux) ux[k] = uax + c * (s->usx[k] - uax);
        if (uy) uy[k] = uay + c * (s->usy[k] - uay);
        if (phi) phi[k] = s->phi[k];
        if (owner) owner[k] = s->owner[k];
    }
}

void orc_forces(const orc_sim *s, double *force, double *fcol, orc_particle *state)
{
    if (force) memcpy(force, s->force, sizeof(double) * 3 * s->np);
    if (fcol) memcpy(fcol, s->fcol, sizeof(double) * 2 * s->np);
    if (state) memcpy(state, s->parts, sizeof(orc_particle) * s->np);
}

void orc_get_populations(const orc_sim *s, double *out)
{
    memcpy(out, s->f, sizeof(double) * 9 * (size_t)s->p.nx * s->p.ny);
}

void orc_set_populations(orc_sim *s, const double *in)
{
    memcpy(s->f, in, sizeof(double) * 9 * (size_t)s->p.nx * s->p.ny);
}

void orc_set_particles(orc_sim *s, const orc_particle *in)
{
    memcpy(s->parts, in, sizeof(orc_particle) * s->np);
}

long long orc_steps_done(const orc_sim *s) { return s->steps; }
