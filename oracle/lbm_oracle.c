/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of the D2Q9 lattice Boltzmann cavity method
 * of Xiang & Shi, "Flow Simulation of Lid-Driven Rectangular Cavity by Using Lattice
 * Boltzmann Method" (arXiv 2211.05009).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is checked against.
 * Only the test suite, the package smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header, table or helper with the CUDA library: it keeps
 * its own copy of every constant below.  It is written for readability, not speed: AoS
 * layout f[(y*nx + x)*9 + j], one node at a time, FP64, compiled with -ffp-contract=off.
 *
 * Algorithm per time step (Sec. 2.1 Eq. 1 and Sec. 2.2):
 *   1. streaming   f_j(x, t+1) <- f*_j(x - c_j, t)                      (Eq. 1, left side)
 *   2. boundary    wall nodes are rebuilt by non-equilibrium extrapolation
 *                  f_j(x_b) = f_j^eq(rho_f, u_w) + [f_j(x_f) - f_j^eq(rho_f, u_f)]  (Sec. 2.2 ii)
 *   3. collision   f*_j = f_j - (f_j - f_j^eq(rho, u)) / tau               (Eq. 1, right side)
 * with f^eq of Eq. 2 and the moments of Eq. 3.  The stored state is always the
 * post-collision field f* of the last step.
 *
 * Readings of points the paper leaves open (each is listed in the design notes):
 *  - velocity order 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)
 *  - walls lie on the outer ring of the nx*ny grid; the lid is the top row y = ny-1
 *  - the two top corners are stationary unless corner_moving is set
 *  - the NEE reference node x_f is the inner neighbour along the inward normal
 *    (the diagonal inner node for corners), and the wall density is rho_f
 *
 * Threads: compiled a second time with -fopenmp (liblbm_oracle_omp.so), the three node loops
 * of orc_step split their rows over the host's cores.  Every node is still computed by the
 * same arithmetic from the same inputs (step 2 reads only fluid nodes written in step 1), so
 * the result is bitwise that of the single-thread build; without -fopenmp the pragmas are
 * ignored.
 *
 * Test-only boundary modes (not in the paper; they exist to pin the oracle against
 * closed forms): halfway bounce-back cavity, fully periodic box, and a channel that is
 * periodic in x with NEE walls on rows 0 and ny-1; an optional body force uses the
 * forcing scheme of Guo, Zheng and Shi (Phys. Rev. E 65, 046308, 2002).
 */
#include <math.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

/* D2Q9 lattice, Sec. 2.1 (after Eq. 2): c = 1 (Sec. 3), weights 4/9, 1/9, 1/36. */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* c_s^2 = c^2/3 with c = 1 (Sec. 2.1): 1/c_s^2 = 3, 1/(2 c_s^4) = 9/2, 1/(2 c_s^2) = 3/2. */
#define INV_CS2 3.0
#define INV_2CS4 4.5
#define INV_2CS2 1.5

enum { ORC_CAVITY_NEE = 0, ORC_CAVITY_BB = 1, ORC_PERIODIC = 2, ORC_CHANNEL_NEE = 3 };

typedef struct {
    int nx, ny;        /* nodes along x (width) and y (height), walls included            */
    double tau;        /* relaxation time, Eq. 1                                            */
    double U;          /* lid (top wall) velocity along +x                                  */
    int mode;          /* one of ORC_*                                                      */
    int corner_moving; /* 1: the two top corner nodes move with the lid                     */
    double Fx, Fy;     /* body force (test-only channel flow); 0 for the paper's cavity     */
} orc_params;

static size_t node(const orc_params *p, int x, int y) { return (size_t)y * (size_t)p->nx + (size_t)x; }

/* Eq. 2: f_j^eq = w_j rho [1 + c_j.u / c_s^2 + (c_j.u)^2 / (2 c_s^4) - u.u / (2 c_s^2)]. */
void orc_feq(double rho, double ux, double uy, double *feq)
{
    double uu = ux * ux + uy * uy;
    for (int j = 0; j < 9; ++j) {
        double cu = CX[j] * ux + CY[j] * uy;
        feq[j] = W[j] * rho * (1.0 + INV_CS2 * cu + INV_2CS4 * cu * cu - INV_2CS2 * uu);
    }
}

/* Eq. 3: rho = sum_j f_j, rho u = sum_j c_j f_j (plus half the body force, Guo et al.). */
static void moments9(const double *f, double Fx, double Fy, double *rho, double *ux, double *uy)
{
    double r = 0.0, mx = 0.0, my = 0.0;
    for (int j = 0; j < 9; ++j) {
        r += f[j];
        mx += CX[j] * f[j];
        my += CY[j] * f[j];
    }
    *rho = r;
    *ux = (mx + 0.5 * Fx) / r;
    *uy = (my + 0.5 * Fy) / r;
}

/* Is (x, y) a wall node of an NEE mode?  Fills the wall velocity and the reference node. */
static int nee_wall(const orc_params *p, int x, int y, double *uwx, double *uwy, int *xf, int *yf)
{
    int nx = p->nx, ny = p->ny;
    if (p->mode == ORC_CAVITY_NEE) {
        int on = (x == 0 || x == nx - 1 || y == 0 || y == ny - 1);
        if (!on) return 0;
        /* inward normal neighbour; for corners the diagonal inner node */
        *xf = x == 0 ? 1 : (x == nx - 1 ? nx - 2 : x);
        *yf = y == 0 ? 1 : (y == ny - 1 ? ny - 2 : y);
        int lid = (y == ny - 1) && (p->corner_moving || (x > 0 && x < nx - 1));
        *uwx = lid ? p->U : 0.0;
        *uwy = 0.0;
        return 1;
    }
    if (p->mode == ORC_CHANNEL_NEE) {
        if (y != 0 && y != ny - 1) return 0;
        *xf = x;
        *yf = y == 0 ? 1 : ny - 2;
        *uwx = (y == ny - 1) ? p->U : 0.0;
        *uwy = 0.0;
        return 1;
    }
    return 0;
}

/* Step 1 at one fluid node: pull f_j(x) = f*_j(x - c_j) from the previous post-collision
 * field (Eq. 1).  Periodic directions wrap; in bounce-back mode a population whose source
 * lies outside the box is the reflected one, with the moving-wall term of Ladd
 * (-2 w_j rho_0 c_j.u_w / c_s^2, rho_0 = 1) on links that cross the lid. */
static void pull_node(const orc_params *p, const double *fin, int x, int y, double *f)
{
    int nx = p->nx, ny = p->ny;
    for (int j = 0; j < 9; ++j) {
        int sx = x - CX[j], sy = y - CY[j];
        if (p->mode == ORC_PERIODIC || p->mode == ORC_CHANNEL_NEE) sx = (sx + nx) % nx;
        if (p->mode == ORC_PERIODIC) sy = (sy + ny) % ny;
        if (p->mode == ORC_CAVITY_BB && (sx < 0 || sx >= nx || sy < 0 || sy >= ny)) {
            /* the population leaving (x, y) along c_opp(j) comes back reversed */
            int o = OPP[j];
            double term = 0.0;
            if (sy >= ny) term = 2.0 * W[o] * 1.0 * (CX[o] * p->U) * INV_CS2;
            f[j] = fin[node(p, x, y) * 9 + o] - term;
            continue;
        }
        f[j] = fin[node(p, sx, sy) * 9 + j];
    }
}

/* Step 3 at one node: BGK collision of Eq. 1, with the Guo et al. source when a force is set. */
static void collide_node(const orc_params *p, const double *f, int forced, double *out)
{
    double Fx = forced ? p->Fx : 0.0, Fy = forced ? p->Fy : 0.0;
    double rho, ux, uy, feq[9];
    moments9(f, Fx, Fy, &rho, &ux, &uy);
    orc_feq(rho, ux, uy, feq);
    for (int j = 0; j < 9; ++j) {
        double src = 0.0;
        if (forced && (Fx != 0.0 || Fy != 0.0)) {
            double cu = CX[j] * ux + CY[j] * uy;
            double ax = INV_CS2 * (CX[j] - ux) + INV_CS2 * INV_CS2 * cu * CX[j];
            double ay = INV_CS2 * (CY[j] - uy) + INV_CS2 * INV_CS2 * cu * CY[j];
            src = (1.0 - 0.5 / p->tau) * W[j] * (ax * Fx + ay * Fy);
        }
        out[j] = f[j] - (f[j] - feq[j]) / p->tau + src;
    }
}

/* Step 2 at one wall node, given the streamed populations fxf of its reference node. */
static void nee_set(const double *fxf, double uwx, double uwy, double *fb)
{
    double rho_f, uxf, uyf, eq_w[9], eq_f[9];
    moments9(fxf, 0.0, 0.0, &rho_f, &uxf, &uyf);
    orc_feq(rho_f, uwx, uwy, eq_w);
    orc_feq(rho_f, uxf, uyf, eq_f);
    for (int j = 0; j < 9; ++j) fb[j] = eq_w[j] + (fxf[j] - eq_f[j]);
}

/* One time step over the whole grid: stream, then NEE boundary, then collide.
 * fin and fout are distinct [ny*nx*9] arrays; fin is left unchanged. */
void orc_step(const orc_params *p, const double *fin, double *fout)
{
    int nx = p->nx, ny = p->ny;
    double uwx, uwy;
    int xf, yf;
    /* 1. streaming into fout (fluid nodes only) */
#pragma omp parallel for private(uwx, uwy, xf, yf) schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (nee_wall(p, x, y, &uwx, &uwy, &xf, &yf)) continue;
            pull_node(p, fin, x, y, &fout[node(p, x, y) * 9]);
        }
    /* 2. non-equilibrium extrapolation at wall nodes, from the streamed reference nodes */
#pragma omp parallel for private(uwx, uwy, xf, yf) schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            if (nee_wall(p, x, y, &uwx, &uwy, &xf, &yf))
                nee_set(&fout[node(p, xf, yf) * 9], uwx, uwy, &fout[node(p, x, y) * 9]);
    /* 3. collision at every node (no body force on wall nodes) */
#pragma omp parallel for private(uwx, uwy, xf, yf) schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double tmp[9];
            int wall = nee_wall(p, x, y, &uwx, &uwy, &xf, &yf);
            memcpy(tmp, &fout[node(p, x, y) * 9], sizeof tmp);
            collide_node(p, tmp, !wall, &fout[node(p, x, y) * 9]);
        }
}

/* The same step evaluated at a single node (x, y) of a full-size field: the value
 * orc_step would store there.  Used to check large GPU runs at sampled nodes. */
void orc_step_node(const orc_params *p, const double *fin, int x, int y, double *out9)
{
    double uwx, uwy, f[9];
    int xf, yf;
    if (nee_wall(p, x, y, &uwx, &uwy, &xf, &yf)) {
        double fxf[9];
        pull_node(p, fin, xf, yf, fxf);
        nee_set(fxf, uwx, uwy, f);
        collide_node(p, f, 0, out9);
    } else {
        pull_node(p, fin, x, y, f);
        collide_node(p, f, 1, out9);
    }
}

/* Sec. 2.2 (i): rho = 1, u = 0 except the lid nodes (u_x = U); f = f^eq. */
void orc_init(const orc_params *p, double *f)
{
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            double uwx = 0.0, uwy = 0.0;
            int xf, yf;
            if (!nee_wall(p, x, y, &uwx, &uwy, &xf, &yf)) uwx = uwy = 0.0;
            orc_feq(1.0, uwx, uwy, &f[node(p, x, y) * 9]);
        }
}

/* f = f^eq(rho, u) node by node from given macroscopic fields [ny*nx]. */
void orc_init_moments(const orc_params *p, const double *rho, const double *ux, const double *uy,
                      double *f)
{
    size_t n = (size_t)p->nx * (size_t)p->ny;
    for (size_t k = 0; k < n; ++k) orc_feq(rho[k], ux[k], uy[k], &f[k * 9]);
}

/* Derivative along one grid line of a node field (grid spacing 1): central difference
 * (a[i+1] - a[i-1]) / 2 inside, the three-point one-sided formula (-3 a0 + 4 a1 - a2) / 2 (and
 * its mirror) at the two end nodes; both exact for quadratics.  line[k * stride] is node k. */
static double d_line(const double *line, size_t stride, int i, int n)
{
    if (i == 0) return (-3.0 * line[0] + 4.0 * line[stride] - line[2 * stride]) / 2.0;
    if (i == n - 1)
        return (3.0 * line[(size_t)(n - 1) * stride] - 4.0 * line[(size_t)(n - 2) * stride] +
                line[(size_t)(n - 3) * stride]) / 2.0;
    return (line[(size_t)(i + 1) * stride] - line[(size_t)(i - 1) * stride]) / 2.0;
}

/* Not part of the paper: a post-collision state consistent with given macroscopic fields to
 * first order in the Chapman-Enskog expansion of BGK (a warm start that does not begin with a
 * stress-free field).  Pre-collision f = f^eq + f^neq with
 *     f^neq_j = -tau w_j rho / c_s^2 (c_ja c_jb - c_s^2 delta_ab) d_a u_b,   c_s^2 = 1/3,
 * and one BGK collision keeps (1 - 1/tau) of it:  f*_j = f^eq_j(rho, u) + (1 - 1/tau) f^neq_j.
 * f^neq carries no mass or momentum, so the moments of f* are (rho, u).  Derivatives by d_line;
 * needs nx, ny >= 3. */
void orc_init_moments_neq(const orc_params *p, const double *rho, const double *ux, const double *uy,
                          double *f)
{
    const double cs2 = 1.0 / 3.0;
    const double keep = 1.0 - 1.0 / p->tau;
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const size_t k = node(p, x, y);
            const double *rx = ux + (size_t)y * (size_t)p->nx, *ry = uy + (size_t)y * (size_t)p->nx;
            const double dxux = d_line(rx, 1, x, p->nx), dxuy = d_line(ry, 1, x, p->nx);
            const double dyux = d_line(ux + x, (size_t)p->nx, y, p->ny);
            const double dyuy = d_line(uy + x, (size_t)p->nx, y, p->ny);
            double *fk = &f[k * 9];
            orc_feq(rho[k], ux[k], uy[k], fk);
            for (int j = 0; j < 9; ++j) {
                const double qxx = CX[j] * CX[j] - cs2, qyy = CY[j] * CY[j] - cs2;
                const double qxy = (double)(CX[j] * CY[j]);
                /* Q:grad u = Q_ab d_a u_b, Q symmetric */
                const double qdu = qxx * dxux + qxy * (dxuy + dyux) + qyy * dyuy;
                const double fneq = -p->tau * W[j] * rho[k] / cs2 * qdu;
                fk[j] += keep * fneq;
            }
        }
}

/* Eq. 3 at every node of a post-collision field.  Wall nodes report (rho_f, u_w), the
 * moments their post-collision populations carry. */
void orc_moments(const orc_params *p, const double *f, double *rho, double *ux, double *uy)
{
    size_t n = (size_t)p->nx * (size_t)p->ny;
    for (size_t k = 0; k < n; ++k) {
        int x = (int)(k % (size_t)p->nx), y = (int)(k / (size_t)p->nx);
        double uwx, uwy;
        int xf, yf;
        int wall = nee_wall(p, x, y, &uwx, &uwy, &xf, &yf);
        /* A forced post-collision field carries rho u + F/2 (BGK adds F/(2 tau), the Guo
         * source F (1 - 1/(2 tau))), so half the force is taken off here. */
        double F = wall ? 0.0 : -1.0;
        moments9(&f[k * 9], F * p->Fx, F * p->Fy, &rho[k], &ux[k], &uy[k]);
    }
}

/* Eq. 6: sqrt( sum[(ux1-ux0)^2 + (uy1-uy0)^2] / sum[ux0^2 + uy0^2] ) over all nodes. */
double orc_residual(size_t n, const double *ux1, const double *uy1, const double *ux0,
                    const double *uy0)
{
    double num = 0.0, den = 0.0;
    for (size_t k = 0; k < n; ++k) {
        double dx = ux1[k] - ux0[k], dy = uy1[k] - uy0[k];
        num += dx * dx + dy * dy;
        den += ux0[k] * ux0[k] + uy0[k] * uy0[k];
    }
    return sqrt(num / den);
}

/* Total mass sum_x rho(x) of a population field. */
double orc_mass(const orc_params *p, const double *f)
{
    size_t n = (size_t)p->nx * (size_t)p->ny * 9;
    double m = 0.0;
    for (size_t k = 0; k < n; ++k) m += f[k];
    return m;
}

/* Stream function with u_x = dPsi/dy (Table 1, Table 2 post-processing): Psi = 0 on the
 * bottom wall, trapezoid rule in y with dy = 1.  Writes psi[ny*nx] and the minimum with
 * its node (first in row-major order on ties) and the maximum with its node. */
void orc_stream_function(const orc_params *p, const double *ux, double *psi, double *psi_min,
                         int *imin, int *jmin, double *psi_max, int *imax, int *jmax)
{
    int nx = p->nx, ny = p->ny;
    for (int x = 0; x < nx; ++x) {
        psi[node(p, x, 0)] = 0.0;
        for (int y = 1; y < ny; ++y)
            psi[node(p, x, y)] = psi[node(p, x, y - 1)] +
                                 0.5 * (ux[node(p, x, y - 1)] + ux[node(p, x, y)]);
    }
    *psi_min = psi[0];
    *psi_max = psi[0];
    *imin = *jmin = *imax = *jmax = 0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double v = psi[node(p, x, y)];
            if (v < *psi_min) { *psi_min = v; *imin = x; *jmin = y; }
            if (v > *psi_max) { *psi_max = v; *imax = x; *jmax = y; }
        }
}

/* Host threads the node loops of orc_step use: 1 unless built with -fopenmp. */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Convenience driver: n steps from f (in place), ping-ponging through tmp.
 * Returns 0, or 1 if a non-finite value appears. */
int orc_run(const orc_params *p, double *f, double *tmp, long n)
{
    size_t bytes = (size_t)p->nx * (size_t)p->ny * 9 * sizeof(double);
    for (long s = 0; s < n; ++s) {
        orc_step(p, f, tmp);
        memcpy(f, tmp, bytes);
    }
    size_t cnt = (size_t)p->nx * (size_t)p->ny * 9;
    for (size_t k = 0; k < cnt; ++k)
        if (!isfinite(f[k])) return 1;
    return 0;
}
