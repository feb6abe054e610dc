/*
 * FP64 CPU oracle for the column-physics step of
 * "Dynamic Load Balancing in GPU-Based Systems - Early Experiments"
 * (Fazenda, Mendes, Kale, Panetta, Rodrigues, 2013).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library, and the library never calls it.
 *
 * What one time step computes (in the order the paper's application runs its
 * phases, Fig. 2: dynamics kernel, then physics kernel):
 *
 *  1. Dynamics (Sec. IV, "3D Jacobi solver" phase; stand-in: first-order
 *     upwind advection).  Convex donor-cell form
 *        q*[k][j][i] = (1-|cx|-|cy|-|cz|) q + |cx| q[i-sx] + |cy| q[j-sy]
 *                      + |cz| q[k-sz]
 *     with s = sign of the velocity (upwind neighbour), periodic in x and y.
 *     Vertically the two end faces carry no flux: the cell next to the closed
 *     downwind face keeps the |cz| q it would have sent out, and the cell next
 *     to the closed upwind face receives nothing.
 *
 *  2. Physics (Fig. 1 and Fig. 4, Sec. IV and Sec. VI-B): a serial-in-k
 *     recurrence per column whose trip count is multiplied by the load array
 *     C(i,j).  Stand-in: k_c(i,j,t) passes of one implicit vertical-diffusion
 *     solve  M x = d,  M = tridiag(-r, 1+2r, -r) with zero-flux (Neumann)
 *     ends (first and last diagonal entry 1+r), solved by the textbook
 *     Thomas algorithm, then d <- x.  k_c = 0 leaves the column unchanged.
 *
 *  3. The load array moves through the domain "similar to advection
 *     transport" (Sec. VI-B): the moving-disk rule gives k_in inside a disk of
 *     radius R whose centre is (x0,y0) + t (vx,vy) (periodic, minimum-image
 *     distance, integer cell indices), k_out outside.  A caller-supplied
 *     array is the other source.
 *
 *  4. Diagnostic: the global sum of q after the step (Neumaier-compensated).
 *
 *  Dynamics, second form (dynamics == 1): the Sec. IV "3D Jacobi solver",
 *  read as one sweep per step of the weighted Jacobi iteration for Laplace's
 *  equation on the 7-point stencil,
 *        q*[k][j][i] = (1 - 6 nu) q + nu (q[i-1] + q[i+1] + q[j-1] + q[j+1]
 *                                         + q[k-1] + q[k+1]),
 *  periodic in x and y; vertically the end faces carry no flux (mirror
 *  ghosts: the missing neighbour of an end cell is the cell itself).  The
 *  paper gives neither weight nor sweep count; nu = 1/7 (the 7-point mean)
 *  is the default reading, 0 < nu <= 1/6 keeps every weight non-negative.
 *
 * Layout: x fastest, idx = (k*ny + j)*nx + i.  All arithmetic is FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nx, ny, nz;
    double cx, cy, cz, r;
    int32_t kc_mode;        /* 0: kc array (ny*nx, row j, column i); 1: moving disk */
    const int32_t *kc;      /* used when kc_mode == 0 */
    int32_t disk_x0, disk_y0, disk_vx, disk_vy, disk_r, k_in, k_out;
    int32_t dynamics;       /* 0: upwind advection; 1: weighted Jacobi sweep */
    double nu;              /* Jacobi weight (dynamics == 1) */
} orc_grid;

static long wrap(long a, long n) {
    long m = a % n;
    return m < 0 ? m + n : m;
}

/* Moving-disk load rule (Sec. VI-B).  Exact integer arithmetic. */
int32_t orc_kc_disk(const orc_grid *g, long i, long j, long t) {
    long cxt = wrap((long)g->disk_x0 + t * (long)g->disk_vx, g->nx);
    long cyt = wrap((long)g->disk_y0 + t * (long)g->disk_vy, g->ny);
    long dx = wrap(i - cxt, g->nx);
    long dy = wrap(j - cyt, g->ny);
    if (dx > g->nx / 2) dx -= g->nx;
    if (dy > g->ny / 2) dy -= g->ny;
    long R = g->disk_r;
    return (dx * dx + dy * dy <= R * R) ? g->k_in : g->k_out;
}

/* Fill kc_out[ny*nx] with k_c(i,j,t) of the grid's rule. */
void orc_kc_field(const orc_grid *g, long t, int32_t *kc_out) {
    for (long j = 0; j < g->ny; ++j)
        for (long i = 0; i < g->nx; ++i)
            kc_out[j * g->nx + i] = g->kc_mode ? orc_kc_disk(g, i, j, t)
                                               : g->kc[j * g->nx + i];
}

/*
 * One implicit vertical-diffusion solve, textbook Thomas algorithm
 * (forward elimination, back substitution), in place on d[0..nz-1].
 * Row k:  a_k x_{k-1} + b_k x_k + c_k x_{k+1} = d_k, with
 *   a_k = -r (k>0), c_k = -r (k<nz-1), b_k = 1 + r * (number of neighbours).
 * cp and dp are scratch arrays of length nz.
 */
void orc_thomas(int32_t nz, double r, double *d, double *cp, double *dp) {
    if (nz <= 0) return;
    double b0 = 1.0 + r * (nz > 1 ? 1.0 : 0.0);
    double c0 = nz > 1 ? -r : 0.0;
    cp[0] = c0 / b0;
    dp[0] = d[0] / b0;
    for (int32_t k = 1; k < nz; ++k) {
        double a = -r;
        double b = 1.0 + r * (k < nz - 1 ? 2.0 : 1.0);
        double c = k < nz - 1 ? -r : 0.0;
        double den = b - a * cp[k - 1];
        cp[k] = c / den;
        dp[k] = (d[k] - a * dp[k - 1]) / den;
    }
    d[nz - 1] = dp[nz - 1];
    for (int32_t k = nz - 2; k >= 0; --k) d[k] = dp[k] - cp[k] * d[k + 1];
}

/*
 * Upwind advection, convex donor-cell form.  periodic != 0: x/y wrap.
 * periodic == 0 ("window" mode): a neighbour outside the array is NaN, so
 * every cell whose dependence reaches outside the window becomes NaN.
 */
void orc_advect(const orc_grid *g, int periodic, const double *q, double *qs) {
    const long nx = g->nx, ny = g->ny, nz = g->nz;
    const double ax = fabs(g->cx), ay = fabs(g->cy), az = fabs(g->cz);
    const long sx = g->cx >= 0 ? 1 : -1, sy = g->cy >= 0 ? 1 : -1;
    const long sz = g->cz >= 0 ? 1 : -1;
    for (long k = 0; k < nz; ++k) {
        /* vertical neighbour and whether this cell's downwind face is closed */
        long ku = k - sz;
        int has_up = (ku >= 0 && ku < nz);
        long kd = k + sz;
        int down_open = (kd >= 0 && kd < nz);
        double w0 = 1.0 - ax - ay - (down_open ? az : 0.0);
        for (long j = 0; j < ny; ++j) {
            long ju = j - sy;
            int jin = periodic || (ju >= 0 && ju < ny);
            if (periodic) ju = wrap(ju, ny);
            for (long i = 0; i < nx; ++i) {
                long iu = i - sx;
                int iin = periodic || (iu >= 0 && iu < nx);
                if (periodic) iu = wrap(iu, nx);
                /* terms with a zero weight are left out, so that a window
                   run is not poisoned by a neighbour the step never uses */
                double v = 0.0;
                if (w0 != 0.0) v += w0 * q[(k * ny + j) * nx + i];
                if (ax != 0.0) v += ax * (iin ? q[(k * ny + j) * nx + iu] : NAN);
                if (ay != 0.0) v += ay * (jin ? q[(k * ny + ju) * nx + i] : NAN);
                if (az != 0.0 && has_up) v += az * q[(ku * ny + j) * nx + i];
                qs[(k * ny + j) * nx + i] = v;
            }
        }
    }
}

/*
 * Weighted Jacobi sweep of the 7-point stencil (dynamics == 1).
 * periodic != 0: x/y wrap; periodic == 0 (window mode): a neighbour outside
 * the array is NaN.  Vertical ends: mirror ghosts (zero flux).
 */
void orc_jacobi(const orc_grid *g, int periodic, const double *q, double *qs) {
    const long nx = g->nx, ny = g->ny, nz = g->nz;
    const double nu = g->nu, w0 = 1.0 - 6.0 * g->nu;
    for (long k = 0; k < nz; ++k) {
        const long kd = k > 0 ? k - 1 : 0, ku = k < nz - 1 ? k + 1 : nz - 1;
        for (long j = 0; j < ny; ++j) {
            long jm = j - 1, jp = j + 1;
            const int jmin = periodic || jm >= 0, jpin = periodic || jp < ny;
            if (periodic) {
                jm = wrap(jm, ny);
                jp = wrap(jp, ny);
            }
            for (long i = 0; i < nx; ++i) {
                long im = i - 1, ip = i + 1;
                const int imin = periodic || im >= 0, ipin = periodic || ip < nx;
                if (periodic) {
                    im = wrap(im, nx);
                    ip = wrap(ip, nx);
                }
                const double c = q[(k * ny + j) * nx + i];
                double sum = 0.0;
                sum += imin ? q[(k * ny + j) * nx + im] : NAN;
                sum += ipin ? q[(k * ny + j) * nx + ip] : NAN;
                sum += jmin ? q[(k * ny + jm) * nx + i] : NAN;
                sum += jpin ? q[(k * ny + jp) * nx + i] : NAN;
                sum += q[(kd * ny + j) * nx + i];
                sum += q[(ku * ny + j) * nx + i];
                qs[(k * ny + j) * nx + i] = w0 * c + nu * sum;
            }
        }
    }
}

/* Neumaier-compensated sum; returns sum, writes the compensation term. */
double orc_sum(const double *x, long n, double *comp) {
    double s = 0.0, c = 0.0;
    for (long m = 0; m < n; ++m) {
        double v = x[m];
        double t = s + v;
        if (fabs(s) >= fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    if (comp) *comp = c;
    return s + c;
}

/*
 * One full step on a grid (or on a window of it).
 *   q_in, q_out: nz*ny*nx arrays (may not alias).
 *   kc: ny*nx k_c values for this step (already evaluated).
 */
void orc_step(const orc_grid *g, int periodic, const int32_t *kc,
              const double *q_in, double *q_out) {
    const long nx = g->nx, ny = g->ny, nz = g->nz;
    if (g->dynamics == 1) orc_jacobi(g, periodic, q_in, q_out);
    else orc_advect(g, periodic, q_in, q_out);
    double *col = (double *)malloc(sizeof(double) * 3 * (size_t)nz);
    double *cp = col + nz, *dp = col + 2 * nz;
    for (long j = 0; j < ny; ++j)
        for (long i = 0; i < nx; ++i) {
            int32_t n = kc[j * nx + i];
            if (n <= 0) continue;
            for (long k = 0; k < nz; ++k) col[k] = q_out[(k * ny + j) * nx + i];
            for (int32_t s = 0; s < n; ++s) orc_thomas((int32_t)nz, g->r, col, cp, dp);
            for (long k = 0; k < nz; ++k) q_out[(k * ny + j) * nx + i] = col[k];
        }
    free(col);
}

/*
 * Run nsteps periodic steps starting at global step index t0.  q is updated
 * in place.  mass[s] (if non-NULL) receives the compensated sum after step s.
 * kc_fields (kc_mode 0 only, may be NULL): nsteps arrays of ny*nx, one per
 * step; when NULL the grid's kc array is used for every step.
 */
void orc_run(const orc_grid *g, long t0, int32_t nsteps, double *q,
             double *mass, const int32_t *kc_fields) {
    const long ncol = (long)g->nx * g->ny, n = ncol * g->nz;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *kc = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncol);
    for (int32_t s = 0; s < nsteps; ++s) {
        if (g->kc_mode == 0 && kc_fields)
            memcpy(kc, kc_fields + (size_t)s * ncol, sizeof(int32_t) * (size_t)ncol);
        else
            orc_kc_field(g, t0 + s, kc);
        orc_step(g, 1, kc, q, tmp);
        memcpy(q, tmp, sizeof(double) * (size_t)n);
        if (mass) mass[s] = orc_sum(q, n, NULL);
    }
    free(tmp);
    free(kc);
}

/*
 * Window run: the same steps on the sub-box of columns
 * [i0, i0+wx) x [j0, j0+wy) of a periodic grid (full size g->nx x g->ny).
 * q holds nz*wy*wx values on entry (x fastest) and is updated in place;
 * outside the window every neighbour is NaN, so after s steps only the
 * columns whose whole dependence (upwind side, or both sides for the Jacobi
 * sweep) lies in the window stay finite.
 * k_c of a window column is the full grid's value at its global position:
 * the disk rule is evaluated at (i0+i, j0+j) wrapped; for kc_mode 0,
 * kc_fields holds nsteps windows of wy*wx values (or one, if kc_per_step==0).
 */
void orc_run_window(const orc_grid *g, long i0, long j0, int32_t wx, int32_t wy,
                    long t0, int32_t nsteps, double *q,
                    const int32_t *kc_fields, int32_t kc_per_step) {
    orc_grid w = *g;
    w.nx = wx;
    w.ny = wy;
    const long ncol = (long)wx * wy, n = ncol * g->nz;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *kc = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncol);
    for (int32_t s = 0; s < nsteps; ++s) {
        for (long j = 0; j < wy; ++j)
            for (long i = 0; i < wx; ++i) {
                if (g->kc_mode)
                    kc[j * wx + i] = orc_kc_disk(g, wrap(i0 + i, g->nx), wrap(j0 + j, g->ny), t0 + s);
                else
                    kc[j * wx + i] = kc_fields[(kc_per_step ? (size_t)s * ncol : 0) + j * wx + i];
            }
        orc_step(&w, 0, kc, q, tmp);
        memcpy(q, tmp, sizeof(double) * (size_t)n);
    }
    free(tmp);
    free(kc);
}
