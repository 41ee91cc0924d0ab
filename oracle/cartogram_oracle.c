/*
 * Plain FP64 CPU oracle of the diffusion-driven flow cartogram.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library. It shares no code, header, table or
 * constant with the CUDA path: it is written directly from the paper's equations,
 * slowly and plainly, so that a reader can check each function against the text.
 *
 * Paper: M. T. Gastner, V. Seguy, P. More, "Fast flow-based algorithm for creating
 * density-equalizing map projections", PNAS 115, E2156 (2018), arXiv:1802.07625.
 *
 * Conventions (readings of the paper, shared with the CUDA path only as prose):
 *  - grid points are cell centres x_i = i + 1/2, y_j = j + 1/2 (SI Eq. rhoxyt with
 *    the integrals of the cosine transform taken by the midpoint rule);
 *  - fields are row-major, index [j*Lx + i] (x fastest); spectra [n*Lx + m];
 *  - time uses D = 1: f_mn(t) = exp(-pi^2 (m^2/Lx^2 + n^2/Ly^2) t), which is SI
 *    Eq. fmn_diff with t_paper = pi^2 t, and v = -grad(rho)/rho (Fick's law in the
 *    main text's section on flow-based cartograms);
 *  - the Gaussian blur of width sigma multiplies every cosine coefficient by
 *    exp(-pi^2 sigma^2 (m^2/Lx^2 + n^2/Ly^2) / 2);
 *  - the predictor-corrector is Heun's method with error ||r_corr - r_pred||.
 *
 * Parity status per function (what pins it in tests/test_oracle_pins.py):
 *  orc_forward, orc_fields        brute-force 2-D double sums, round trip, single
 *                                 cosine mode, conserved mean (pinned)
 *  orc_velocity, orc_interp       closed-form single-mode velocity, no-flux walls,
 *                                 exact reproduction of linear fields (pinned)
 *  orc_heun_step                  closed form of Heun's method for linear fields (pinned)
 *  orc_integrate, orc_integrate_replay   uniform density -> identity; x-only density ->
 *                                 closed-form 1-D equalising map (pinned to the
 *                                 discretisation error only)
 *  orc_rasterize, orc_coverage    hand-computed coverages, total mass; the density as
 *                                 the coverage-weighted sum of the region densities (pinned)
 *  orc_region_areas, orc_area_errors, orc_map_points   closed forms (pinned)
 *  orc_flux_linear                single-mode and 2-D-mode closed forms, discrete
 *                                 continuity against the density change (pinned)
 *  orc_integrate_linear           x-only density -> closed-form 1-D map at t = 1 (pinned
 *                                 to the discretisation error)
 *  orc_cartogram                  invariants only (strip map converges to the 1-D
 *                                 closed form); the exact 2-D result of a Voronoi map
 *                                 is not fixed by the paper: parity unpinned there.
 *  orc_distortion                 affine grids (closed-form singular values), their
 *                                 composition, identity (pinned)
 *  orc_inverse_points             affine grids (closed-form inverse), round trip
 *                                 through orc_map_points on cartogram grids (pinned)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    int Lx, Ly;
    double blur;       /* Gaussian blur width sigma, in cells */
    double dt0;        /* first trial time step (D = 1 units) */
    double atol;       /* accept a step if ||r_corr - r_pred|| <= atol (cells) */
    double grow;       /* step factor after an accepted step */
    double shrink;     /* step factor after a rejected step */
    double cfl;        /* cap: h * max|v| <= cfl cells */
    double rho_tol;    /* stop once max |rho - rho_bar| / rho_bar <= rho_tol */
    double area_tol;   /* outer loop stops once max relative area error < area_tol */
    int max_steps;     /* per integration (accepted + rejected) */
    int max_iter;      /* outer iterations */
    double blur_decay; /* iteration k blurs with width blur * blur_decay^k */
    int flow;          /* 0: diffusion flow (SI Eq. fmn_diff); 1: linear equalisation (Eq. fmn_fast) */
} orc_params;

typedef struct {
    int iterations;
    int converged;
    int status;                 /* 0 ok, -4 no convergence, -6 step failure */
    long long steps_accepted;   /* summed over iterations */
    long long steps_rejected;
    double max_area_error;
    double t_end_last;
} orc_stats;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* cos(pi*m*(i+1/2)/L) for all m, i, evaluated through the exact integer reduction
 * k = m*(2i+1) mod 4L of the angle pi*k/(2L). C[i*L + m]. */
static double* cos_matrix(int L) {
    double* tab = (double*)malloc(sizeof(double) * 4 * L);
    for (int k = 0; k < 4 * L; ++k) tab[k] = cos(ORC_PI * k / (2.0 * L));
    double* C = (double*)malloc(sizeof(double) * (size_t)L * L);
    for (int i = 0; i < L; ++i)
        for (int m = 0; m < L; ++m)
            C[(size_t)i * L + m] = tab[((long long)m * (2 * i + 1)) % (4 * L)];
    free(tab);
    return C;
}

/* sin(pi*m*(i+1/2)/L), S[i*L + m], same reduction. */
static double* sin_matrix(int L) {
    double* tab = (double*)malloc(sizeof(double) * 4 * L);
    for (int k = 0; k < 4 * L; ++k) tab[k] = sin(ORC_PI * k / (2.0 * L));
    double* S = (double*)malloc(sizeof(double) * (size_t)L * L);
    for (int i = 0; i < L; ++i)
        for (int m = 0; m < L; ++m)
            S[(size_t)i * L + m] = tab[((long long)m * (2 * i + 1)) % (4 * L)];
    free(tab);
    return S;
}

/* Forward cosine transform of the density with the Gaussian blur (main text Eq.
 * rhotilde_mn; SI Eq. rhoxyt's coefficient formula; blur from the section on
 * benchmarking, "Gaussian blur of moderate width"):
 *   spec[n][m] = 4/((1+d_m0)(1+d_n0)) sum_ij rho[j][i] cos(pi m x_i/Lx) cos(pi n y_j/Ly)
 *                * exp(-pi^2 sigma^2 (m^2/Lx^2 + n^2/Ly^2)/2).
 * The double sum is evaluated as two nested single sums (distributive law). */
void orc_forward(int Lx, int Ly, const double* rho, double blur, double* spec) {
    double* Cx = cos_matrix(Lx);
    double* Cy = cos_matrix(Ly);
    double* tmp = (double*)calloc((size_t)Lx * Ly, sizeof(double)); /* tmp[j][m] */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < Ly; ++j)
        for (int m = 0; m < Lx; ++m) {
            double s = 0.0;
            for (int i = 0; i < Lx; ++i) s += rho[(size_t)j * Lx + i] * Cx[(size_t)i * Lx + m];
            tmp[(size_t)j * Lx + m] = s;
        }
#pragma omp parallel for schedule(static)
    for (int n = 0; n < Ly; ++n) {
        double* row = spec + (size_t)n * Lx;
        for (int m = 0; m < Lx; ++m) row[m] = 0.0;
        for (int j = 0; j < Ly; ++j) {
            double c = Cy[(size_t)j * Ly + n];
            const double* t = tmp + (size_t)j * Lx;
            for (int m = 0; m < Lx; ++m) row[m] += c * t[m];
        }
        for (int m = 0; m < Lx; ++m) {
            double w = (m == 0 ? 2.0 : 4.0) / (n == 0 ? 2.0 : 1.0);
            double k2 = (double)m * m / ((double)Lx * Lx) + (double)n * n / ((double)Ly * Ly);
            row[m] *= w * exp(-ORC_PI * ORC_PI * blur * blur * k2 / 2.0);
        }
    }
    free(tmp); free(Cx); free(Cy);
}

/* Density and its gradient at time t from the cosine coefficients (SI Eq. rhoxyt
 * with f_mn = exp(-pi^2 (m^2/Lx^2 + n^2/Ly^2) t), SI Eq. fmn_diff in D = 1 time):
 *   rho(x,y,t) = 1/(Lx Ly) sum_mn spec_mn f_mn(t) cos(pi m x/Lx) cos(pi n y/Ly)
 *   d_x rho    = 1/(Lx Ly) sum_mn spec_mn f_mn(t) (-pi m/Lx) sin(pi m x/Lx) cos(pi n y/Ly)
 *   d_y rho    = 1/(Lx Ly) sum_mn spec_mn f_mn(t) cos(pi m x/Lx) (-pi n/Ly) sin(pi n y/Ly)
 * evaluated at the cell centres. Any output pointer may be NULL. */
void orc_fields(int Lx, int Ly, const double* spec, double t,
                double* rho, double* gx, double* gy) {
    double* Cx = cos_matrix(Lx);
    double* Sx = sin_matrix(Lx);
    double* Cy = cos_matrix(Ly);
    double* Sy = sin_matrix(Ly);
    double* damped = (double*)malloc(sizeof(double) * (size_t)Lx * Ly);
    double* P = (double*)malloc(sizeof(double) * (size_t)Lx * Ly); /* P[n][i] */
    double* Q = (double*)malloc(sizeof(double) * (size_t)Lx * Ly); /* Q[n][i] */
    for (int n = 0; n < Ly; ++n)
        for (int m = 0; m < Lx; ++m) {
            double k2 = (double)m * m / ((double)Lx * Lx) + (double)n * n / ((double)Ly * Ly);
            damped[(size_t)n * Lx + m] = spec[(size_t)n * Lx + m] * exp(-ORC_PI * ORC_PI * k2 * t);
        }
#pragma omp parallel for schedule(static)
    for (int n = 0; n < Ly; ++n)
        for (int i = 0; i < Lx; ++i) {
            double p = 0.0, q = 0.0;
            for (int m = 0; m < Lx; ++m) {
                double a = damped[(size_t)n * Lx + m];
                p += a * Cx[(size_t)i * Lx + m];
                q += a * (-ORC_PI * m / Lx) * Sx[(size_t)i * Lx + m];
            }
            P[(size_t)n * Lx + i] = p;
            Q[(size_t)n * Lx + i] = q;
        }
    const double norm = 1.0 / ((double)Lx * Ly);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < Ly; ++j) {
        for (int i = 0; i < Lx; ++i) {
            if (rho) rho[(size_t)j * Lx + i] = 0.0;
            if (gx) gx[(size_t)j * Lx + i] = 0.0;
            if (gy) gy[(size_t)j * Lx + i] = 0.0;
        }
        for (int n = 0; n < Ly; ++n) {
            double c = Cy[(size_t)j * Ly + n] * norm;
            double s = (-ORC_PI * n / Ly) * Sy[(size_t)j * Ly + n] * norm;
            const double* p = P + (size_t)n * Lx;
            const double* q = Q + (size_t)n * Lx;
            for (int i = 0; i < Lx; ++i) {
                if (rho) rho[(size_t)j * Lx + i] += c * p[i];
                if (gx) gx[(size_t)j * Lx + i] += c * q[i];
                if (gy) gy[(size_t)j * Lx + i] += s * p[i];
            }
        }
    }
    free(Cx); free(Sx); free(Cy); free(Sy); free(damped); free(P); free(Q);
}

/* Fick's law with D = 1 (main text, section on flow-based cartograms):
 * v = -grad(rho)/rho at every grid point. Returns max_ij |v_ij|. */
double orc_velocity(int Lx, int Ly, const double* rho, const double* gx, const double* gy,
                    double* vx, double* vy) {
    double vmax = 0.0;
    for (size_t k = 0; k < (size_t)Lx * Ly; ++k) {
        vx[k] = -gx[k] / rho[k];
        vy[k] = -gy[k] / rho[k];
        double a = sqrt(vx[k] * vx[k] + vy[k] * vy[k]);
        if (a > vmax) vmax = a;
    }
    return vmax;
}

/* Velocity at an arbitrary point by bilinear interpolation between grid points
 * (main text: "interpolating between the grid points"). The interpolation lattice
 * along x is {0, 1/2, 3/2, ..., Lx-1/2, Lx}: the two walls are extra lattice lines
 * on which the normal component vanishes (no flux through the box edges, main text
 * and SI Eqs. Jx, Jy) and the tangential component equals that of the nearest
 * interior grid point; likewise along y. */
static double lattice_pos(int a, int L) {
    if (a == 0) return 0.0;
    if (a == L + 1) return (double)L;
    return a - 0.5;
}

static void lattice_value(int Lx, int Ly, const double* vx, const double* vy,
                          int a, int b, double* ox, double* oy) {
    int ghost_x = (a == 0 || a == Lx + 1);
    int ghost_y = (b == 0 || b == Ly + 1);
    int ia = a == 0 ? 0 : (a == Lx + 1 ? Lx - 1 : a - 1);
    int jb = b == 0 ? 0 : (b == Ly + 1 ? Ly - 1 : b - 1);
    *ox = ghost_x ? 0.0 : vx[(size_t)jb * Lx + ia];
    *oy = ghost_y ? 0.0 : vy[(size_t)jb * Lx + ia];
}

static int lattice_cell(double x, int L) {
    if (x < 0.5) return 0;
    if (x >= L - 0.5) return L;
    return (int)floor(x - 0.5) + 1;
}

void orc_interp(int Lx, int Ly, const double* vx, const double* vy, double x, double y,
                double* ux, double* uy) {
    int a = lattice_cell(x, Lx), b = lattice_cell(y, Ly);
    double xa = lattice_pos(a, Lx), xb = lattice_pos(a + 1, Lx);
    double ya = lattice_pos(b, Ly), yb = lattice_pos(b + 1, Ly);
    double wx = (x - xa) / (xb - xa), wy = (y - ya) / (yb - ya);
    double v00x, v00y, v10x, v10y, v01x, v01y, v11x, v11y;
    lattice_value(Lx, Ly, vx, vy, a, b, &v00x, &v00y);
    lattice_value(Lx, Ly, vx, vy, a + 1, b, &v10x, &v10y);
    lattice_value(Lx, Ly, vx, vy, a, b + 1, &v01x, &v01y);
    lattice_value(Lx, Ly, vx, vy, a + 1, b + 1, &v11x, &v11y);
    *ux = (1 - wx) * (1 - wy) * v00x + wx * (1 - wy) * v10x + (1 - wx) * wy * v01x + wx * wy * v11x;
    *uy = (1 - wx) * (1 - wy) * v00y + wx * (1 - wy) * v10y + (1 - wx) * wy * v01y + wx * wy * v11y;
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* One predictor-corrector (Heun) step of r' = v(r, t) for n points (main text Eq.
 * rt_diff integrated with "a predictor-corrector method"):
 *   r*  = r + h v(r, t)                     (predictor, v0 = field at t)
 *   r'  = r + h/2 (v(r, t) + v(r*, t+h))    (corrector, v1 = field at t+h)
 * each stage clamped to the box. Writes r* and r'; returns max_p ||r'_p - r*_p||. */
double orc_heun_step(int Lx, int Ly, const double* v0x, const double* v0y,
                     const double* v1x, const double* v1y, long long n,
                     const double* x, const double* y, double h,
                     double* xp, double* yp, double* xc, double* yc) {
    double err = 0.0;
#pragma omp parallel for schedule(static) reduction(max : err)
    for (long long p = 0; p < n; ++p) {
        double ax, ay, bx, by;
        orc_interp(Lx, Ly, v0x, v0y, x[p], y[p], &ax, &ay);
        double px = clampd(x[p] + h * ax, 0.0, Lx);
        double py = clampd(y[p] + h * ay, 0.0, Ly);
        orc_interp(Lx, Ly, v1x, v1y, px, py, &bx, &by);
        double cx = clampd(x[p] + 0.5 * h * (ax + bx), 0.0, Lx);
        double cy = clampd(y[p] + 0.5 * h * (ay + by), 0.0, Ly);
        if (xp) { xp[p] = px; yp[p] = py; }
        xc[p] = cx; yc[p] = cy;
        double e = sqrt((cx - px) * (cx - px) + (cy - py) * (cy - py));
        if (e > err) err = e;
    }
    return err;
}

/* Velocity field at time t: returns max |v|, and max |rho - rho_bar|/rho_bar in *dev. */
static double field_at(int Lx, int Ly, const double* spec, double t, double rho_bar,
                       double* rho, double* gx, double* gy, double* vx, double* vy, double* dev) {
    orc_fields(Lx, Ly, spec, t, rho, gx, gy);
    double d = 0.0;
    for (size_t k = 0; k < (size_t)Lx * Ly; ++k) {
        double e = fabs(rho[k] - rho_bar) / rho_bar;
        if (e > d) d = e;
    }
    *dev = d;
    return orc_velocity(Lx, Ly, rho, gx, gy, vx, vy);
}

/* One integration of the flow from t = 0 toward t = infinity (main text Eq. rt_diff;
 * SI Eq. T_integral) for all Lx*Ly grid points, with adaptive steps:
 *   start: h = dt0, positions = cell centres, v0 = field at t = 0;
 *   attempt: h <- min(h, cfl/max|v0|); v1 = field at t+h; Heun step;
 *   accept if ||r' - r*|| <= atol for every point: r <- r', t <- t+h, v0 <- v1,
 *     stop if max|rho(t) - rho_bar|/rho_bar <= rho_tol, else h <- grow*h;
 *   reject otherwise: h <- shrink*h.
 * X, Y (Lx*Ly each) receive the projected grid. If sched_h/sched_acc are non-NULL
 * they receive the attempted steps (at most sched_cap entries). Returns 0, or -6
 * when max_steps attempts did not reach the stopping rule. */
int orc_integrate(const orc_params* P, const double* spec, double* X, double* Y,
                  long long* n_acc, long long* n_rej, double* t_end,
                  double* sched_h, int* sched_acc, int sched_cap) {
    const int Lx = P->Lx, Ly = P->Ly;
    const size_t N = (size_t)Lx * Ly;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* gx = (double*)malloc(sizeof(double) * N);
    double* gy = (double*)malloc(sizeof(double) * N);
    double* v0x = (double*)malloc(sizeof(double) * N);
    double* v0y = (double*)malloc(sizeof(double) * N);
    double* v1x = (double*)malloc(sizeof(double) * N);
    double* v1y = (double*)malloc(sizeof(double) * N);
    double* cx = (double*)malloc(sizeof(double) * N);
    double* cy = (double*)malloc(sizeof(double) * N);
    const double rho_bar = spec[0] / ((double)Lx * Ly); /* rho~_00 = rho_bar Lx Ly */
    for (int j = 0; j < Ly; ++j)
        for (int i = 0; i < Lx; ++i) {
            X[(size_t)j * Lx + i] = i + 0.5;
            Y[(size_t)j * Lx + i] = j + 0.5;
        }
    double dev;
    double vmax = field_at(Lx, Ly, spec, 0.0, rho_bar, rho, gx, gy, v0x, v0y, &dev);
    long long acc = 0, rej = 0;
    double t = 0.0, h = P->dt0;
    int status = 0;
    int done = dev <= P->rho_tol;
    while (!done) {
        if (acc + rej >= P->max_steps) { status = -6; break; }
        if (vmax > 0.0 && h * vmax > P->cfl) h = P->cfl / vmax;
        double dev1;
        double vmax1 = field_at(Lx, Ly, spec, t + h, rho_bar, rho, gx, gy, v1x, v1y, &dev1);
        double err = orc_heun_step(Lx, Ly, v0x, v0y, v1x, v1y, (long long)N, X, Y, h,
                                   NULL, NULL, cx, cy);
        int accepted = err <= P->atol;
        if (sched_h && acc + rej < sched_cap) {
            sched_h[acc + rej] = h;
            sched_acc[acc + rej] = accepted;
        }
        if (accepted) {
            memcpy(X, cx, sizeof(double) * N);
            memcpy(Y, cy, sizeof(double) * N);
            double* s;
            s = v0x; v0x = v1x; v1x = s;
            s = v0y; v0y = v1y; v1y = s;
            vmax = vmax1;
            t += h;
            ++acc;
            if (dev1 <= P->rho_tol) done = 1;
            else h *= P->grow;
        } else {
            ++rej;
            h *= P->shrink;
        }
    }
    *n_acc = acc;
    *n_rej = rej;
    *t_end = t;
    free(rho); free(gx); free(gy); free(v0x); free(v0y); free(v1x); free(v1y); free(cx); free(cy);
    return status;
}


/* The integration with a fixed step schedule: the accepted step sizes h[0..n) of an
 * adaptive run, taken in order with no acceptance test (the function whose derivative
 * the gradient entry point computes). */
void orc_integrate_replay(const orc_params* P, const double* spec, const double* h, int n, double* X,
                          double* Y) {
    const int Lx = P->Lx, Ly = P->Ly;
    const size_t N = (size_t)Lx * Ly;
    double* rho = (double*)malloc(sizeof(double) * N);
    double* gx = (double*)malloc(sizeof(double) * N);
    double* gy = (double*)malloc(sizeof(double) * N);
    double* v0x = (double*)malloc(sizeof(double) * N);
    double* v0y = (double*)malloc(sizeof(double) * N);
    double* v1x = (double*)malloc(sizeof(double) * N);
    double* v1y = (double*)malloc(sizeof(double) * N);
    double* cx = (double*)malloc(sizeof(double) * N);
    double* cy = (double*)malloc(sizeof(double) * N);
    const double rho_bar = spec[0] / ((double)Lx * Ly);
    for (int j = 0; j < Ly; ++j)
        for (int i = 0; i < Lx; ++i) {
            X[(size_t)j * Lx + i] = i + 0.5;
            Y[(size_t)j * Lx + i] = j + 0.5;
        }
    double dev;
    double t = 0.0;
    field_at(Lx, Ly, spec, 0.0, rho_bar, rho, gx, gy, v0x, v0y, &dev);
    for (int k = 0; k < n; ++k) {
        field_at(Lx, Ly, spec, t + h[k], rho_bar, rho, gx, gy, v1x, v1y, &dev);
        orc_heun_step(Lx, Ly, v0x, v0y, v1x, v1y, (long long)N, X, Y, h[k], NULL, NULL, cx, cy);
        memcpy(X, cx, sizeof(double) * N);
        memcpy(Y, cy, sizeof(double) * N);
        double* s;
        s = v0x; v0x = v1x; v1x = s;
        s = v0y; v0y = v1y; v1y = s;
        t = t + h[k];
    }
    free(rho); free(gx); free(gy); free(v0x); free(v0y); free(v1x); free(v1y); free(cx); free(cy);
}

/* Flux of the linear-equalisation flow (SI Eq. fmn_fast, f_mn = 1 - t for t <= 1): with
 * f'_mn = -1, SI Eqs. Jxmn and Jymn give the t-independent coefficients
 *   Jx~_mn = m Lx Ly^2 rho~_mn / (pi (m^2 Ly^2 + n^2 Lx^2)),
 *   Jy~_mn = n Lx^2 Ly rho~_mn / (pi (m^2 Ly^2 + n^2 Lx^2)),
 * and SI Eqs. Jx, Jy the flux at the cell centres:
 *   Jx = 1/(Lx Ly) sum_{m>=1,n>=0} Jx~_mn sin(pi m x/Lx) cos(pi n y/Ly),
 *   Jy = 1/(Lx Ly) sum_{m>=0,n>=1} Jy~_mn cos(pi m x/Lx) sin(pi n y/Ly).
 * (Main text Eqs. vx_cable, vy_cable print this velocity with a leading minus; the
 * continuity equation with rho(t) = (1-t) rho0 + t rho_bar fixes the plus sign used here.)
 * The double sums are evaluated as nested single sums. */
void orc_flux_linear(int Lx, int Ly, const double* spec, double* jx, double* jy) {
    double* Cx = cos_matrix(Lx);
    double* Sx = sin_matrix(Lx);
    double* Cy = cos_matrix(Ly);
    double* Sy = sin_matrix(Ly);
    double* ax = (double*)malloc(sizeof(double) * (size_t)Lx * Ly); /* Jx~[n][m] */
    double* ay = (double*)malloc(sizeof(double) * (size_t)Lx * Ly); /* Jy~[n][m] */
    for (int n = 0; n < Ly; ++n)
        for (int m = 0; m < Lx; ++m) {
            const double den = ORC_PI * ((double)m * m * Ly * Ly + (double)n * n * Lx * Lx);
            const double r = spec[(size_t)n * Lx + m];
            ax[(size_t)n * Lx + m] = (m == 0) ? 0.0 : m * (double)Lx * Ly * Ly * r / den;
            ay[(size_t)n * Lx + m] = (n == 0) ? 0.0 : n * (double)Lx * Lx * Ly * r / den;
        }
    double* P = (double*)malloc(sizeof(double) * (size_t)Lx * Ly); /* sum_m Jx~ sin, [n][i] */
    double* Q = (double*)malloc(sizeof(double) * (size_t)Lx * Ly); /* sum_m Jy~ cos, [n][i] */
#pragma omp parallel for schedule(static)
    for (int n = 0; n < Ly; ++n)
        for (int i = 0; i < Lx; ++i) {
            double p = 0.0, q = 0.0;
            for (int m = 0; m < Lx; ++m) {
                p += ax[(size_t)n * Lx + m] * Sx[(size_t)i * Lx + m];
                q += ay[(size_t)n * Lx + m] * Cx[(size_t)i * Lx + m];
            }
            P[(size_t)n * Lx + i] = p;
            Q[(size_t)n * Lx + i] = q;
        }
    const double norm = 1.0 / ((double)Lx * Ly);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < Ly; ++j) {
        for (int i = 0; i < Lx; ++i) {
            jx[(size_t)j * Lx + i] = 0.0;
            jy[(size_t)j * Lx + i] = 0.0;
        }
        for (int n = 0; n < Ly; ++n) {
            const double c = Cy[(size_t)j * Ly + n] * norm;
            const double sn = Sy[(size_t)j * Ly + n] * norm;
            for (int i = 0; i < Lx; ++i) {
                jx[(size_t)j * Lx + i] += c * P[(size_t)n * Lx + i];
                jy[(size_t)j * Lx + i] += sn * Q[(size_t)n * Lx + i];
            }
        }
    }
    free(Cx); free(Sx); free(Cy); free(Sy); free(ax); free(ay); free(P); free(Q);
}

/* Velocity of the linear flow at the grid points at time t (main text Eq. rho_ffb and
 * the paragraph after it: v = J / rho with rho(t) = (1-t) rho0 + t rho_bar, t <= 1).
 * Returns max |v|. */
static double linear_velocity(int Lx, int Ly, const double* jx, const double* jy, const double* rho0,
                              double rho_bar, double t, double* vx, double* vy) {
    double vmax = 0.0;
    for (size_t k = 0; k < (size_t)Lx * Ly; ++k) {
        const double r = (1.0 - t) * rho0[k] + t * rho_bar;
        vx[k] = jx[k] / r;
        vy[k] = jy[k] / r;
        const double a = sqrt(vx[k] * vx[k] + vy[k] * vy[k]);
        if (a > vmax) vmax = a;
    }
    return vmax;
}

/* One integration of the linear flow from t = 0 to t = 1 (main text: "integrate Eq.
 * rt_diff only until t = 1"), with the same adaptive predictor-corrector as
 * orc_integrate: h <- min(h, cfl/max|v(t)|, 1 - t); accept if ||r' - r*|| <= atol; the
 * integration ends with the accepted step that reaches t = 1. */
int orc_integrate_linear(const orc_params* P, const double* spec, double* X, double* Y,
                         long long* n_acc, long long* n_rej, double* t_end) {
    const int Lx = P->Lx, Ly = P->Ly;
    const size_t N = (size_t)Lx * Ly;
    double* jx = (double*)malloc(sizeof(double) * N);
    double* jy = (double*)malloc(sizeof(double) * N);
    double* rho0 = (double*)malloc(sizeof(double) * N);
    double* v0x = (double*)malloc(sizeof(double) * N);
    double* v0y = (double*)malloc(sizeof(double) * N);
    double* v1x = (double*)malloc(sizeof(double) * N);
    double* v1y = (double*)malloc(sizeof(double) * N);
    double* cx = (double*)malloc(sizeof(double) * N);
    double* cy = (double*)malloc(sizeof(double) * N);
    const double rho_bar = spec[0] / ((double)Lx * Ly);
    orc_flux_linear(Lx, Ly, spec, jx, jy);
    orc_fields(Lx, Ly, spec, 0.0, rho0, NULL, NULL);
    for (int j = 0; j < Ly; ++j)
        for (int i = 0; i < Lx; ++i) {
            X[(size_t)j * Lx + i] = i + 0.5;
            Y[(size_t)j * Lx + i] = j + 0.5;
        }
    double vmax = linear_velocity(Lx, Ly, jx, jy, rho0, rho_bar, 0.0, v0x, v0y);
    long long acc = 0, rej = 0;
    double t = 0.0, h = P->dt0;
    int status = 0;
    while (t < 1.0) {
        if (acc + rej >= P->max_steps) { status = -6; break; }
        if (vmax > 0.0 && h * vmax > P->cfl) h = P->cfl / vmax;
        if (h > 1.0 - t) h = 1.0 - t;
        const double t1 = (t + h >= 1.0) ? 1.0 : t + h;
        const double vmax1 = linear_velocity(Lx, Ly, jx, jy, rho0, rho_bar, t1, v1x, v1y);
        const double err = orc_heun_step(Lx, Ly, v0x, v0y, v1x, v1y, (long long)N, X, Y, t1 - t,
                                         NULL, NULL, cx, cy);
        if (err <= P->atol) {
            memcpy(X, cx, sizeof(double) * N);
            memcpy(Y, cy, sizeof(double) * N);
            double* s;
            s = v0x; v0x = v1x; v1x = s;
            s = v0y; v0y = v1y; v1y = s;
            vmax = vmax1;
            t = t1;
            ++acc;
            h *= P->grow;
        } else {
            ++rej;
            h *= P->shrink;
        }
    }
    *n_acc = acc;
    *n_rej = rej;
    *t_end = t;
    free(jx); free(jy); free(rho0); free(v0x); free(v0y); free(v1x); free(v1y); free(cx); free(cy);
    return status;
}

/* Shoelace area of one ring (signed: counter-clockwise positive). */
static double ring_area(const double* xy, long long a, long long b) {
    double s = 0.0;
    for (long long k = a; k < b; ++k) {
        long long l = (k + 1 < b) ? k + 1 : a;
        s += xy[2 * k] * xy[2 * l + 1] - xy[2 * l] * xy[2 * k + 1];
    }
    return 0.5 * s;
}

/* Area of every region = sum of the signed areas of its rings. */
void orc_region_areas(int n_regions, long long n_rings, const long long* ring_offsets,
                      const int* ring_region, const double* xy, double* areas) {
    for (int r = 0; r < n_regions; ++r) areas[r] = 0.0;
    for (long long k = 0; k < n_rings; ++k)
        areas[ring_region[k]] += ring_area(xy, ring_offsets[k], ring_offsets[k + 1]);
}

/* Relative area error (main text, stopping criterion; the printed formula names the
 * same quantity twice, read here as current area over target area minus one):
 *   err_i = A_i / A^_i - 1,  A^_i = V_i * sum(A) / sum(V).
 * Returns max_i |err_i|. */
double orc_area_errors(int n_regions, const double* values, const double* areas, double* err) {
    double sv = 0.0, sa = 0.0, mx = 0.0;
    for (int r = 0; r < n_regions; ++r) { sv += values[r]; sa += areas[r]; }
    for (int r = 0; r < n_regions; ++r) {
        double target = values[r] * sa / sv;
        err[r] = areas[r] / target - 1.0;
        if (fabs(err[r]) > mx) mx = fabs(err[r]);
    }
    return mx;
}

/* Sutherland-Hodgman clip of polygon (n points in px,py) by the half-plane
 * s*(coord - c) >= 0 where coord is x (axis 0) or y (axis 1). Output in qx,qy. */
static int clip_half(const double* px, const double* py, int n, int axis, double c, double s,
                     double* qx, double* qy) {
    int m = 0;
    for (int k = 0; k < n; ++k) {
        int l = (k + 1) % n;
        double ak = s * ((axis == 0 ? px[k] : py[k]) - c);
        double al = s * ((axis == 0 ? px[l] : py[l]) - c);
        int in_k = ak >= 0.0, in_l = al >= 0.0;
        if (in_k) { qx[m] = px[k]; qy[m] = py[k]; ++m; }
        if (in_k != in_l) {
            double f = ak / (ak - al);
            double ix = px[k] + f * (px[l] - px[k]);
            double iy = py[k] + f * (py[l] - py[k]);
            if (axis == 0) ix = c; else iy = c;
            qx[m] = ix; qy[m] = iy; ++m;
        }
    }
    return m;
}

static double poly_area(const double* px, const double* py, int n) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
        int l = (k + 1) % n;
        s += px[k] * py[l] - px[l] * py[k];
    }
    return 0.5 * s;
}

/* Rasterised piecewise-constant density (main text, section on previous
 * all-coordinates methods: a region's density is its value over its area; the
 * margin between the map and the box is filled with the mean density):
 *   d_i   = V_i / A_i,   d_out = sum(V)/sum(A)
 *   rho[j][i] = d_out + sum_rings (d_region - d_out) * area(ring  intersect  cell_ij)
 * where the area of the ring inside the unit cell is exact (polygon clipping),
 * signed by the ring's orientation. */
/* Add w * area(ring intersect cell) to rho[cell] for every cell the ring touches (the
 * ring clipped to each row strip, then to each cell of the strip). */
static void raster_ring(int Lx, int Ly, const double* xy, long long a, long long b, double w, double* rho) {
    int n = (int)(b - a);
    if (n < 3) return;
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (long long v = a; v < b; ++v) {
        x0 = fmin(x0, xy[2 * v]); x1 = fmax(x1, xy[2 * v]);
        y0 = fmin(y0, xy[2 * v + 1]); y1 = fmax(y1, xy[2 * v + 1]);
    }
    int cap = 16 * n + 64; /* each half-plane clip at most doubles the vertex count */
    double* rx = (double*)malloc(sizeof(double) * n);
    double* ry = (double*)malloc(sizeof(double) * n);
    double* b1x = (double*)malloc(sizeof(double) * cap);
    double* b1y = (double*)malloc(sizeof(double) * cap);
    double* b2x = (double*)malloc(sizeof(double) * cap);
    double* b2y = (double*)malloc(sizeof(double) * cap);
    double* b3x = (double*)malloc(sizeof(double) * cap);
    double* b3y = (double*)malloc(sizeof(double) * cap);
    double* b4x = (double*)malloc(sizeof(double) * cap);
    double* b4y = (double*)malloc(sizeof(double) * cap);
    for (int v = 0; v < n; ++v) { rx[v] = xy[2 * (a + v)]; ry[v] = xy[2 * (a + v) + 1]; }
    int j0 = (int)floor(y0), j1 = (int)ceil(y1);
    int i0 = (int)floor(x0), i1 = (int)ceil(x1);
    if (j0 < 0) j0 = 0;
    if (i0 < 0) i0 = 0;
    if (j1 > Ly) j1 = Ly;
    if (i1 > Lx) i1 = Lx;
    for (int j = j0; j < j1; ++j) {
        /* the ring restricted to the row strip j <= y <= j+1 */
        int m1 = clip_half(rx, ry, n, 1, (double)j, 1.0, b1x, b1y);
        int m2 = clip_half(b1x, b1y, m1, 1, (double)(j + 1), -1.0, b2x, b2y);
        if (m2 < 3) continue;
        for (int i = i0; i < i1; ++i) {
            int m3 = clip_half(b2x, b2y, m2, 0, (double)i, 1.0, b3x, b3y);
            int m4 = clip_half(b3x, b3y, m3, 0, (double)(i + 1), -1.0, b4x, b4y);
            if (m4 < 3) continue;
            double cov = poly_area(b4x, b4y, m4);
            if (cov != 0.0) {
#pragma omp atomic
                rho[(size_t)j * Lx + i] += w * cov;
            }
        }
    }
    free(rx); free(ry); free(b1x); free(b1y); free(b2x); free(b2y);
    free(b3x); free(b3y); free(b4x); free(b4y);
}

void orc_rasterize(int Lx, int Ly, int n_regions, const double* values, const double* areas,
                   long long n_rings, const long long* ring_offsets, const int* ring_region,
                   const double* xy, double* rho) {
    double sv = 0.0, sa = 0.0;
    for (int r = 0; r < n_regions; ++r) { sv += values[r]; sa += areas[r]; }
    const double d_out = sv / sa;
    for (size_t k = 0; k < (size_t)Lx * Ly; ++k) rho[k] = d_out;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long k = 0; k < n_rings; ++k) {
        int g = ring_region[k];
        raster_ring(Lx, Ly, xy, ring_offsets[k], ring_offsets[k + 1], values[g] / areas[g] - d_out, rho);
    }
}

/* Coverage of every cell by every region (signed sum of its rings' clipped areas),
 * cov[region][Ly][Lx]: the density is linear in the regions' densities through it. */
void orc_coverage(int Lx, int Ly, int n_regions, long long n_rings, const long long* ring_offsets,
                  const int* ring_region, const double* xy, double* cov) {
    memset(cov, 0, sizeof(double) * (size_t)n_regions * Lx * Ly);
#pragma omp parallel for schedule(dynamic, 1)
    for (long long k = 0; k < n_rings; ++k)
        raster_ring(Lx, Ly, xy, ring_offsets[k], ring_offsets[k + 1], 1.0,
                    cov + (size_t)ring_region[k] * Lx * Ly);
}

/* Map points through the projected grid (main text: the output of an integration
 * is the projected Lx*Ly grid; other points follow by interpolation). A point is
 * carried by bilinear interpolation of the projected cell centres (X, Y) over the
 * quad of cell centres that contains it; in the half-cell band along the walls the
 * nearest quad is extended linearly. */
void orc_map_points(int Lx, int Ly, const double* X, const double* Y, long long n,
                    const double* pin, double* pout) {
#pragma omp parallel for schedule(static)
    for (long long p = 0; p < n; ++p) {
        double u = pin[2 * p] - 0.5, w = pin[2 * p + 1] - 0.5;
        int i0 = (int)floor(u), j0 = (int)floor(w);
        if (i0 < 0) i0 = 0;
        if (i0 > Lx - 2) i0 = Lx - 2;
        if (j0 < 0) j0 = 0;
        if (j0 > Ly - 2) j0 = Ly - 2;
        double fx = u - i0, fy = w - j0;
        size_t k00 = (size_t)j0 * Lx + i0, k10 = k00 + 1, k01 = k00 + Lx, k11 = k01 + 1;
        double c00 = (1 - fx) * (1 - fy), c10 = fx * (1 - fy), c01 = (1 - fx) * fy, c11 = fx * fy;
        pout[2 * p] = c00 * X[k00] + c10 * X[k10] + c01 * X[k01] + c11 * X[k11];
        pout[2 * p + 1] = c00 * Y[k00] + c10 * Y[k10] + c01 * Y[k01] + c11 * Y[k11];
    }
}

/* The whole method (main text, section on benchmarking: rasterise, blur, integrate,
 * map, and repeat the integration on its own output until the maximum relative
 * area error is below area_tol):
 *   areas <- shoelace(xy); stop if max|err| < area_tol
 *   repeat up to max_iter times:
 *     rho <- rasterize(xy); spec <- forward(rho, blur); (X,Y) <- integrate(spec)
 *     (iteration it blurs with width blur * blur_decay^it)
 *     xy <- map(X, Y, xy); areas <- shoelace(xy); stop if max|err| < area_tol
 * xy (n_vertices*2) is updated in place. If grids is non-NULL it receives the
 * projected grid of every iteration, [iter][2][Ly][Lx] (X then Y), up to max_iter.
 * err_out (n_regions) receives the final signed area errors. */
int orc_cartogram(const orc_params* P, int n_regions, const double* values,
                  long long n_rings, const long long* ring_offsets, const int* ring_region,
                  long long n_vertices, double* xy, double* grids, double* err_out,
                  orc_stats* st) {
    const int Lx = P->Lx, Ly = P->Ly;
    const size_t N = (size_t)Lx * Ly;
    double* areas = (double*)malloc(sizeof(double) * n_regions);
    double* rho = (double*)malloc(sizeof(double) * N);
    double* spec = (double*)malloc(sizeof(double) * N);
    double* X = (double*)malloc(sizeof(double) * N);
    double* Y = (double*)malloc(sizeof(double) * N);
    double* out = (double*)malloc(sizeof(double) * 2 * (size_t)n_vertices);
    memset(st, 0, sizeof(*st));
    orc_region_areas(n_regions, n_rings, ring_offsets, ring_region, xy, areas);
    double mx = orc_area_errors(n_regions, values, areas, err_out);
    int status = 0;
    int it = 0;
    while (mx >= P->area_tol) {
        if (it >= P->max_iter) { status = -4; break; }
        orc_rasterize(Lx, Ly, n_regions, values, areas, n_rings, ring_offsets, ring_region, xy, rho);
        orc_forward(Lx, Ly, rho, P->blur * pow(P->blur_decay, (double)it), spec);
        long long a, r;
        double tend;
        int s = P->flow == 1 ? orc_integrate_linear(P, spec, X, Y, &a, &r, &tend)
                             : orc_integrate(P, spec, X, Y, &a, &r, &tend, NULL, NULL, 0);
        st->steps_accepted += a;
        st->steps_rejected += r;
        st->t_end_last = tend;
        if (s != 0) { status = s; break; }
        if (grids) {
            memcpy(grids + (size_t)it * 2 * N, X, sizeof(double) * N);
            memcpy(grids + (size_t)it * 2 * N + N, Y, sizeof(double) * N);
        }
        orc_map_points(Lx, Ly, X, Y, n_vertices, xy, out);
        memcpy(xy, out, sizeof(double) * 2 * (size_t)n_vertices);
        orc_region_areas(n_regions, n_rings, ring_offsets, ring_region, xy, areas);
        mx = orc_area_errors(n_regions, values, areas, err_out);
        ++it;
    }
    st->iterations = it;
    st->converged = mx < P->area_tol;
    st->status = status;
    st->max_area_error = mx;
    free(areas); free(rho); free(spec); free(X); free(Y); free(out);
    return status;
}

/* ---------------------------------------------------------------------------------
 * Diagnostics of the composed projection T = T_K o ... o T_1, where T_k is the map of
 * outer iteration k: bilinear interpolation of its projected grid (X_k, Y_k) over the
 * quads of cell centres, the nearest quad extended across the half-cell band along the
 * walls (the same map as orc_map_points).
 * ------------------------------------------------------------------------------- */

/* Quad of the cell-centre lattice that the map of a grid uses at (x, y), and the
 * fractional position in it. */
static void locate_quad(int Lx, int Ly, double x, double y, int* i0, int* j0, double* fx, double* fy) {
    double u = x - 0.5, w = y - 0.5;
    int i = (int)floor(u), j = (int)floor(w);
    if (i < 0) i = 0;
    if (i > Lx - 2) i = Lx - 2;
    if (j < 0) j = 0;
    if (j > Ly - 2) j = Ly - 2;
    *i0 = i;
    *j0 = j;
    *fx = u - i;
    *fy = w - j;
}

/* Angular distortion of the composed projection (SI section 3, the Tissot indicatrix):
 * at the centre of every quad of the original lattice, the Jacobian of T by the chain
 * rule through the K bilinear maps (each differentiated inside its quad), its singular
 * values a >= b, e = ln(a/b) and e~ = 2 asin((a - b)/(a + b)). grids: [K][2][Ly][Lx]
 * (X then Y). out: e_a (mean of e over the (Lx-1)(Ly-1) sample points), e_inf (max),
 * e~_a, e~_inf. Points where T folds (det J <= 0) count with their singular values. */
void orc_distortion(int Lx, int Ly, int K, const double* grids, double* out) {
    const size_t N = (size_t)Lx * Ly;
    double sum_e = 0.0, max_e = 0.0, sum_t = 0.0, max_t = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sum_e, sum_t) reduction(max : max_e, max_t)
    for (int j = 0; j < Ly - 1; ++j)
        for (int i = 0; i + 1 < Lx; ++i) {
            double x = i + 1.0, y = j + 1.0;
            double a = 1.0, b = 0.0, c = 0.0, d = 1.0; /* J = [[a, b], [c, d]] */
            for (int k = 0; k < K; ++k) {
                const double* X = grids + (size_t)k * 2 * N;
                const double* Y = X + N;
                int i0, j0;
                double fx, fy;
                locate_quad(Lx, Ly, x, y, &i0, &j0, &fx, &fy);
                size_t k00 = (size_t)j0 * Lx + i0, k10 = k00 + 1, k01 = k00 + Lx, k11 = k01 + 1;
                /* d T_k / d x and d T_k / d y of the bilinear map inside the quad */
                double txx = (1 - fy) * (X[k10] - X[k00]) + fy * (X[k11] - X[k01]);
                double tyx = (1 - fy) * (Y[k10] - Y[k00]) + fy * (Y[k11] - Y[k01]);
                double txy = (1 - fx) * (X[k01] - X[k00]) + fx * (X[k11] - X[k10]);
                double tyy = (1 - fx) * (Y[k01] - Y[k00]) + fx * (Y[k11] - Y[k10]);
                double na = txx * a + txy * c, nb = txx * b + txy * d;
                double nc = tyx * a + tyy * c, nd = tyx * b + tyy * d;
                a = na; b = nb; c = nc; d = nd;
                double c00 = (1 - fx) * (1 - fy), c10 = fx * (1 - fy), c01 = (1 - fx) * fy, c11 = fx * fy;
                double xn = c00 * X[k00] + c10 * X[k10] + c01 * X[k01] + c11 * X[k11];
                double yn = c00 * Y[k00] + c10 * Y[k10] + c01 * Y[k01] + c11 * Y[k11];
                x = xn;
                y = yn;
            }
            /* singular values of J from its conformal and anti-conformal parts,
             * p = |(a + d, c - b)| and q = |(a - d, c + b)|: s1 = (p + q)/2 and
             * s2 = |p - q|/2 (free of the cancellation of the characteristic
             * polynomial near a conformal J) */
            double pp = hypot(a + d, c - b), qq = hypot(a - d, c + b);
            double s1 = 0.5 * (pp + qq), s2 = 0.5 * fabs(pp - qq);
            double e = log(s1 / s2);
            double et = 2.0 * asin((s1 - s2) / (s1 + s2));
            sum_e += e;
            sum_t += et;
            if (e > max_e) max_e = e;
            if (et > max_t) max_t = et;
        }
    const double n = (double)(Lx - 1) * (Ly - 1);
    out[0] = sum_e / n;
    out[1] = max_e;
    out[2] = sum_t / n;
    out[3] = max_t;
}

/* Bilinear map of quad (i0, j0) at fractional position (u, v) (u, v outside [0, 1]
 * extend the quad linearly). */
static void quad_map(int Lx, const double* X, const double* Y, int i0, int j0, double u, double v,
                     double* x, double* y) {
    size_t k00 = (size_t)j0 * Lx + i0, k10 = k00 + 1, k01 = k00 + Lx, k11 = k01 + 1;
    *x = (1 - u) * (1 - v) * X[k00] + u * (1 - v) * X[k10] + (1 - u) * v * X[k01] + u * v * X[k11];
    *y = (1 - u) * (1 - v) * Y[k00] + u * (1 - v) * Y[k10] + (1 - u) * v * Y[k01] + u * v * Y[k11];
}

/* Preimage of q under one grid's map (the inverse of orc_map_points; the main text's
 * inverse graticule): every quad whose image could contain q is tried by Newton's
 * method on its bilinear map, from the quad's centre; the solution is kept when it
 * falls inside the quad's own domain, which for the quads along the walls extends to
 * the box edge. Returns 0 if no quad contains q. */
static int invert_one(int Lx, int Ly, const double* X, const double* Y, double qx, double qy, double* px,
                      double* py) {
    for (int j0 = 0; j0 + 1 < Ly; ++j0)
        for (int i0 = 0; i0 + 1 < Lx; ++i0) {
            /* domain of the quad in lattice units: [0,1]^2, extended to the box edge */
            const double ulo = i0 == 0 ? -0.5 : 0.0, uhi = i0 == Lx - 2 ? 1.5 : 1.0;
            const double vlo = j0 == 0 ? -0.5 : 0.0, vhi = j0 == Ly - 2 ? 1.5 : 1.0;
            /* bounding box of the image of the (extended) domain: a bilinear map sends
             * the rectangle into the hull of its corners' images */
            double xs[4], ys[4];
            quad_map(Lx, X, Y, i0, j0, ulo, vlo, &xs[0], &ys[0]);
            quad_map(Lx, X, Y, i0, j0, uhi, vlo, &xs[1], &ys[1]);
            quad_map(Lx, X, Y, i0, j0, ulo, vhi, &xs[2], &ys[2]);
            quad_map(Lx, X, Y, i0, j0, uhi, vhi, &xs[3], &ys[3]);
            double xmin = xs[0], xmax = xs[0], ymin = ys[0], ymax = ys[0];
            for (int t = 1; t < 4; ++t) {
                if (xs[t] < xmin) xmin = xs[t];
                if (xs[t] > xmax) xmax = xs[t];
                if (ys[t] < ymin) ymin = ys[t];
                if (ys[t] > ymax) ymax = ys[t];
            }
            const double eps = 1e-9;
            if (qx < xmin - eps || qx > xmax + eps || qy < ymin - eps || qy > ymax + eps) continue;
            size_t k00 = (size_t)j0 * Lx + i0, k10 = k00 + 1, k01 = k00 + Lx, k11 = k01 + 1;
            double u = 0.5, v = 0.5;
            for (int it = 0; it < 60; ++it) {
                double x, y;
                quad_map(Lx, X, Y, i0, j0, u, v, &x, &y);
                double rx = x - qx, ry = y - qy;
                double xu = (1 - v) * (X[k10] - X[k00]) + v * (X[k11] - X[k01]);
                double yu = (1 - v) * (Y[k10] - Y[k00]) + v * (Y[k11] - Y[k01]);
                double xv = (1 - u) * (X[k01] - X[k00]) + u * (X[k11] - X[k10]);
                double yv = (1 - u) * (Y[k01] - Y[k00]) + u * (Y[k11] - Y[k10]);
                double det = xu * yv - xv * yu;
                if (det == 0.0) break;
                double du = (rx * yv - ry * xv) / det, dv = (ry * xu - rx * yu) / det;
                u -= du;
                v -= dv;
                if (fabs(du) + fabs(dv) < 1e-15) break;
            }
            const double tol = 1e-10;
            if (u >= ulo - tol && u <= uhi + tol && v >= vlo - tol && v <= vhi + tol) {
                double x, y;
                quad_map(Lx, X, Y, i0, j0, u, v, &x, &y);
                if (fabs(x - qx) + fabs(y - qy) < 1e-9) {
                    *px = i0 + 0.5 + u;
                    *py = j0 + 0.5 + v;
                    return 1;
                }
            }
        }
    return 0;
}

/* Preimages of n points q under the composed projection: the grids' inverses applied
 * in reverse order. Points without a preimage get NaN. */
void orc_inverse_points(int Lx, int Ly, int K, const double* grids, long long n, const double* q, double* p) {
    const size_t N = (size_t)Lx * Ly;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long t = 0; t < n; ++t) {
        double x = q[2 * t], y = q[2 * t + 1];
        int ok = 1;
        for (int k = K - 1; k >= 0 && ok; --k) {
            const double* X = grids + (size_t)k * 2 * N;
            const double* Y = X + N;
            double px, py;
            ok = invert_one(Lx, Ly, X, Y, x, y, &px, &py);
            x = px;
            y = py;
        }
        p[2 * t] = ok ? x : NAN;
        p[2 * t + 1] = ok ? y : NAN;
    }
}

