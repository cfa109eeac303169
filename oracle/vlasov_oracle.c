/*
 * vlasov_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE; see vlasov_oracle.h).
 *
 * Written from the paper (arXiv:1206.3229), Sec. 2 (models) and Sec. 3 (algorithm), in the paper's
 * order: the second derivative array of a line is computed first (Eq. findif) and stored, then
 * each node takes the cubic-spline value at the foot of its characteristic (Eqs. splinegen,
 * splinecoeffs).  No blocking, no fusion, no FIR reformulation.  Sums use Neumaier compensation.
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *  - Eq. findif prints no 1/du^2 factor; it is required dimensionally and is applied here.
 *  - Eq. splinegen's f''_{i+i} is read as f''_{i+1}.
 *  - A line has n nodes u_k = umin + k*du, du = (umax-umin)/n (endpoint excluded).
 *  - Periodic axes wrap indices mod n.  Non-periodic axes extend f by zero outside the grid and
 *    also take f'' = 0 at nodes outside the grid.
 *  - The foot of node i is y = i - s (s = displacement in cells).  It is split once per line as
 *    n0 = floor(-s), beta = (-s) - n0, alpha = 1 - beta, so k = i + n0 and alpha equals
 *    (x_{k+1} - x)/(x_{k+1} - x_k) of Eq. splinecoeffs.
 *  - Global-spline variant (Eq. tridiagsys, used only for the comparison of Tables 1-2): the diagonal
 *    coefficient printed as 1/3 is read as 2/3, the value the first-derivative continuity the text
 *    derives it from gives (and the cited Numerical Recipes system, (x_{i+1}-x_{i-1})/3 = 2 du/3).
 *    Non-periodic lines solve it for the n grid nodes with f = f'' = 0 at the neighbours -1 and n.
 *  - The force is the rectangle rule of Eq. meanforce on the x nodes.  Ring: kernel
 *    V'(u) = sin u / (2 sqrt 2 (1 - cos u + eps)^{3/2}) at u = (i-k) dx.  Sheet: V = 2 pi G |x-x'|,
 *    so F_i = -2 pi G dx (sum_{k<i} rho_k - sum_{k>i} rho_k).
 */
#include "vlasov_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Eq. (findif) coefficients, |m| = 0..4 (Fornberg eighth-order central second difference). */
static const double FD_C[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

static const double VO_PI = 3.14159265358979323846;

/* ---------------------------------------------------------------- compensated summation */
typedef struct { double s, c; } nsum;
static void ns_add(nsum* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double ns_val(const nsum* a) { return a->s + a->c; }

/* Value of a line at integer index k with the axis' extension (periodic wrap or zero outside). */
static double at(const double* v, long n, int periodic, long k)
{
    if (periodic) {
        long r = k % n;
        if (r < 0) r += n;
        return v[r];
    }
    return (k >= 0 && k < n) ? v[k] : 0.0;
}

/* ---------------------------------------------------------------- Sec. 3, Eq. (findif) */
void vo_fd2(const double* f, long n, int periodic, double du, double* d2)
{
    const double inv = 1.0 / (du * du);
    for (long k = 0; k < n; ++k) {
        double acc = FD_C[0] * f[k];
        for (int m = 1; m <= 4; ++m)
            acc += FD_C[m] * (at(f, n, periodic, k - m) + at(f, n, periodic, k + m));
        d2[k] = acc * inv;
    }
}

/* ---------------------------------------------------------------- Sec. 3, Eq. (tridiagsys) */
/* Tridiagonal solve (sub a, diagonal b, super c, all constant) of n unknowns by elimination and
   back substitution; r is overwritten by the solution, w is n doubles of scratch. */
static void tridiag_const(double a, double b, double c, double* r, long n, double* w)
{
    double den = b;
    r[0] /= den;
    for (long k = 1; k < n; ++k) {
        w[k] = c / den;
        den = b - a * w[k];
        r[k] = (r[k] - a * r[k - 1]) / den;
    }
    for (long k = n - 2; k >= 0; --k) r[k] -= w[k + 1] * r[k + 1];
}

void vo_gs2(const double* f, long n, int periodic, double du, double* d2)
{
    const double a = 1.0 / 6.0, b = 2.0 / 3.0, c = 1.0 / 6.0;   /* times du^2 on the left */
    const double inv = 1.0 / (du * du);
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    for (long k = 0; k < n; ++k)
        d2[k] = (at(f, n, periodic, k + 1) - 2.0 * f[k] + at(f, n, periodic, k - 1)) * inv;
    if (!periodic) {
        tridiag_const(a, b, c, d2, n, w);
        free(w);
        return;
    }
    /* Cyclic system: corners A[0][n-1] = a, A[n-1][0] = c.  Sherman-Morrison: A = A' + u v^T with
       u = (g, 0, .., 0, c), v = (1, 0, .., 0, a/g), g = -b; A' is A without corners and with the
       diagonal ends b - g and b - c a / g (a general tridiagonal solve, written out here). */
    const double g = -b;
    double* y = d2;
    double* z = (double*)malloc(sizeof(double) * (size_t)n);
    double* diag = (double*)malloc(sizeof(double) * (size_t)n);
    for (long k = 0; k < n; ++k) {
        diag[k] = b;
        z[k] = 0.0;
    }
    diag[0] = b - g;
    diag[n - 1] = b - c * a / g;
    z[0] = g;
    z[n - 1] = c;
    /* forward elimination for both right-hand sides */
    double den = diag[0];
    y[0] /= den;
    z[0] /= den;
    for (long k = 1; k < n; ++k) {
        w[k] = c / den;
        den = diag[k] - a * w[k];
        y[k] = (y[k] - a * y[k - 1]) / den;
        z[k] = (z[k] - a * z[k - 1]) / den;
    }
    for (long k = n - 2; k >= 0; --k) {
        y[k] -= w[k + 1] * y[k + 1];
        z[k] -= w[k + 1] * z[k + 1];
    }
    const double fac = (y[0] + a / g * y[n - 1]) / (1.0 + z[0] + a / g * z[n - 1]);
    for (long k = 0; k < n; ++k) y[k] -= fac * z[k];
    free(z);
    free(diag);
    free(w);
}

/* ---------------------------------------------------------------- Sec. 3, Eqs. (splinegen, splinecoeffs) */
void vo_spline_shift(const double* f, const double* d2, long n, int periodic, double du,
                     double s, double* out)
{
    const double ms = -s;
    const double fl = floor(ms);
    const long n0 = (long)fl;
    const double beta = ms - fl;
    const double alpha = 1.0 - beta;
    const double h2 = du * du;
    const double gamma = (alpha * alpha * alpha - alpha) / 6.0 * h2;
    const double delta = (beta * beta * beta - beta) / 6.0 * h2;
    for (long i = 0; i < n; ++i) {
        const long k = i + n0;
        out[i] = alpha * at(f, n, periodic, k) + beta * at(f, n, periodic, k + 1)
               + gamma * at(d2, n, periodic, k) + delta * at(d2, n, periodic, k + 1);
    }
}

/* ---------------------------------------------------------------- Sec. 3 step 1 / step 4 */
void vo_advect_x(const vo_params* P, const double* f, const double* s_row, double* out)
{
    const long nx = P->nx, np = P->np;
    const double dx = (P->xmax - P->xmin) / (double)nx;
#pragma omp parallel
    {
        double* d2 = (double*)malloc(sizeof(double) * (size_t)nx);
#pragma omp for schedule(static)
        for (long j = 0; j < np; ++j) {
            const double* row = f + (size_t)j * nx;
            if (P->spline) vo_gs2(row, nx, P->x_periodic, dx, d2);
            else vo_fd2(row, nx, P->x_periodic, dx, d2);
            vo_spline_shift(row, d2, nx, P->x_periodic, dx, s_row[j], out + (size_t)j * nx);
        }
        free(d2);
    }
}

/* ---------------------------------------------------------------- Sec. 3 step 3 */
void vo_advect_p(const vo_params* P, const double* f, const double* s_col, double* out)
{
    const long nx = P->nx, np = P->np;
    const double dp = (P->pmax - P->pmin) / (double)np;
#pragma omp parallel
    {
        double* col = (double*)malloc(sizeof(double) * (size_t)np);
        double* d2 = (double*)malloc(sizeof(double) * (size_t)np);
        double* res = (double*)malloc(sizeof(double) * (size_t)np);
#pragma omp for schedule(static)
        for (long i = 0; i < nx; ++i) {
            for (long j = 0; j < np; ++j) col[j] = f[(size_t)j * nx + i];
            if (P->spline) vo_gs2(col, np, P->p_periodic, dp, d2);
            else vo_fd2(col, np, P->p_periodic, dp, d2);
            vo_spline_shift(col, d2, np, P->p_periodic, dp, s_col[i], res);
            for (long j = 0; j < np; ++j) out[(size_t)j * nx + i] = res[j];
        }
        free(col);
        free(d2);
        free(res);
    }
}

void vo_xshift_cells(const vo_params* P, double* s_row)
{
    const double dx = (P->xmax - P->xmin) / (double)P->nx;
    const double dp = (P->pmax - P->pmin) / (double)P->np;
    const double cx = (0.5 * P->dt) / dx;
    for (long j = 0; j < P->np; ++j) {
        const double p = P->pmin + (double)j * dp;
        s_row[j] = p * cx;
    }
}

/* ---------------------------------------------------------------- Sec. 2, density */
void vo_density(const vo_params* P, const double* f, double* rho)
{
    const long nx = P->nx, np = P->np;
    const double dp = (P->pmax - P->pmin) / (double)np;
    for (long i = 0; i < nx; ++i) {
        nsum a = {0.0, 0.0};
        for (long j = 0; j < np; ++j) ns_add(&a, f[(size_t)j * nx + i]);
        rho[i] = dp * ns_val(&a);
    }
}

/* Eq. (ringpot) derivative: V'(u) = sin u / (2 sqrt2 (1 - cos u + eps)^{3/2}). */
static double ring_dV(double u, double eps)
{
    const double q = 1.0 - cos(u) + eps;
    return sin(u) / (2.0 * sqrt(2.0) * q * sqrt(q));
}
/* Eq. (ringpot): V(u) = -1 / (sqrt2 sqrt(1 - cos u + eps)). */
static double ring_V(double u, double eps)
{
    return -1.0 / (sqrt(2.0) * sqrt(1.0 - cos(u) + eps));
}

/* ---------------------------------------------------------------- Sec. 2, Eqs. (meanforce, hmfmeanforce, mxmydef) */
void vo_force(const vo_params* P, const double* rho, double* F)
{
    const long nx = P->nx;
    const double dx = (P->xmax - P->xmin) / (double)nx;
    if (P->model == VO_HMF) {
        /* Eq. (mxmydef) then Eq. (hmfmeanforce). */
        nsum mx = {0.0, 0.0}, my = {0.0, 0.0};
        for (long i = 0; i < nx; ++i) {
            const double th = P->xmin + (double)i * dx;
            ns_add(&mx, cos(th) * rho[i]);
            ns_add(&my, sin(th) * rho[i]);
        }
        const double Mx = dx * ns_val(&mx), My = dx * ns_val(&my);
        for (long i = 0; i < nx; ++i) {
            const double th = P->xmin + (double)i * dx;
            F[i] = -Mx * sin(th) + My * cos(th);
        }
    } else if (P->model == VO_RING) {
        /* Eq. (meanforce) with Eq. (ringpot): F_i = -dx sum_k V'((i-k) dx) rho_k.  V' depends only
           on the index difference m = i - k, so it is tabulated once for |m| < nx. */
        double* dV = (double*)malloc(sizeof(double) * (size_t)(2 * nx - 1));
        for (long mm = -(nx - 1); mm <= nx - 1; ++mm) dV[mm + nx - 1] = ring_dV((double)mm * dx, P->eps);
        for (long i = 0; i < nx; ++i) {
            nsum a = {0.0, 0.0};
            for (long k = 0; k < nx; ++k) ns_add(&a, dV[i - k + nx - 1] * rho[k]);
            F[i] = -dx * ns_val(&a);
        }
        free(dV);
    } else if (P->model == VO_SHEET) {
        /* Eq. (meanforce) with V = 2 pi G |x - x'|: F_i = -2 pi G dx sum_k sign(i-k) rho_k. */
        for (long i = 0; i < nx; ++i) {
            nsum a = {0.0, 0.0};
            for (long k = 0; k < nx; ++k) {
                if (k < i) ns_add(&a, rho[k]);
                else if (k > i) ns_add(&a, -rho[k]);
            }
            F[i] = -2.0 * VO_PI * P->G * dx * ns_val(&a);
        }
    } else {
        for (long i = 0; i < nx; ++i) F[i] = 0.0;
    }
}

void vo_pshift_cells(const vo_params* P, const double* F, double* s_col)
{
    const double dp = (P->pmax - P->pmin) / (double)P->np;
    const double cp = P->dt / dp;
    for (long i = 0; i < P->nx; ++i) s_col[i] = F[i] * cp;
}

/* ---------------------------------------------------------------- diagnostics (Sec. 4: energy, norm, Casimirs) */
/* Eq. (casimirs) with s(f) = -f log f, the entropy of Secs. 4.1-4.2, by the rectangle rule on the
   grid nodes; nodes where f <= 0 (spline undershoot) contribute nothing (f log f -> 0 as f -> 0+). */
double vo_entropy(const vo_params* P, const double* f)
{
    const long nx = P->nx, np = P->np;
    const double dx = (P->xmax - P->xmin) / (double)nx;
    const double dp = (P->pmax - P->pmin) / (double)np;
    nsum s = {0, 0};
    for (size_t k = 0; k < (size_t)nx * (size_t)np; ++k)
        if (f[k] > 0.0) ns_add(&s, -f[k] * log(f[k]));
    return dx * dp * ns_val(&s);
}

void vo_moments_of(const vo_params* P, const double* f, vo_moments* out)
{
    const long nx = P->nx, np = P->np;
    const double dx = (P->xmax - P->xmin) / (double)nx;
    const double dp = (P->pmax - P->pmin) / (double)np;
    double* rho = (double*)malloc(sizeof(double) * (size_t)nx);
    vo_density(P, f, rho);

    nsum m = {0, 0}, cx = {0, 0}, sx = {0, 0}, kin = {0, 0}, l2 = {0, 0};
    for (long i = 0; i < nx; ++i) {
        const double th = P->xmin + (double)i * dx;
        ns_add(&m, rho[i]);
        ns_add(&cx, cos(th) * rho[i]);
        ns_add(&sx, sin(th) * rho[i]);
    }
    for (long j = 0; j < np; ++j) {
        const double p = P->pmin + (double)j * dp;
        nsum row = {0, 0};
        for (long i = 0; i < nx; ++i) {
            const double v = f[(size_t)j * nx + i];
            ns_add(&row, v);
            ns_add(&l2, v * v);
        }
        ns_add(&kin, 0.5 * p * p * ns_val(&row));
    }
    out->mass = dx * ns_val(&m);
    out->Mx = dx * ns_val(&cx);
    out->My = dx * ns_val(&sx);
    out->kinetic = dx * dp * ns_val(&kin);
    out->l2 = dx * dp * ns_val(&l2);

    /* Potential energy: U = 1/2 dx^2 sum_i sum_k V(x_i - x_k) rho_i rho_k (Eq. hamgen, mean field). */
    nsum u = {0, 0};
    if (P->model == VO_HMF || P->model == VO_RING || P->model == VO_SHEET) {
        /* Kernel as a function of the index difference m = i - k, tabulated for |m| < nx. */
        double* V = (double*)malloc(sizeof(double) * (size_t)(2 * nx - 1));
        for (long mm = -(nx - 1); mm <= nx - 1; ++mm) {
            const double d = (double)mm * dx;
            double v;
            if (P->model == VO_HMF) v = 1.0 - cos(d);                       /* Eq. (hmfpot) */
            else if (P->model == VO_RING) v = ring_V(d, P->eps);            /* Eq. (ringpot) */
            else v = 2.0 * VO_PI * P->G * fabs(d);                          /* Eq. (sheetpot) */
            V[mm + nx - 1] = v;
        }
        for (long i = 0; i < nx; ++i)
            for (long k = 0; k < nx; ++k) ns_add(&u, V[i - k + nx - 1] * rho[i] * rho[k]);
        free(V);
    }
    out->potential = 0.5 * dx * dx * ns_val(&u);
    out->energy = out->kinetic + out->potential;
    free(rho);
}

/* ---------------------------------------------------------------- Sec. 3 steps 1-4 */
int vo_step_parts(const vo_params* P, const double* f, double* f1, double* F, double* f2,
                  double* out)
{
    const long nx = P->nx, np = P->np;
    const size_t cells = (size_t)nx * (size_t)np;
    double* s_row = (double*)malloc(sizeof(double) * (size_t)np);
    double* s_col = (double*)malloc(sizeof(double) * (size_t)nx);
    double* rho = (double*)malloc(sizeof(double) * (size_t)nx);
    double* Fl = (double*)malloc(sizeof(double) * (size_t)nx);
    double* a = (double*)malloc(sizeof(double) * cells);
    double* b = (double*)malloc(sizeof(double) * cells);
    if (!s_row || !s_col || !rho || !Fl || !a || !b) {
        free(s_row); free(s_col); free(rho); free(Fl); free(a); free(b);
        return -1;
    }
    vo_xshift_cells(P, s_row);
    vo_advect_x(P, f, s_row, a);                 /* Eq. (step1) */
    vo_density(P, a, rho);
    vo_force(P, rho, Fl);                        /* Eq. (step2) */
    vo_pshift_cells(P, Fl, s_col);
    vo_advect_p(P, a, s_col, b);                 /* Eq. (step3) */
    if (f1) memcpy(f1, a, sizeof(double) * cells);
    if (F) memcpy(F, Fl, sizeof(double) * (size_t)nx);
    if (f2) memcpy(f2, b, sizeof(double) * cells);
    if (out) vo_advect_x(P, b, s_row, out);      /* Eq. (step4) */
    free(s_row); free(s_col); free(rho); free(Fl); free(a); free(b);
    return 0;
}

int vo_run(const vo_params* P, double* f, long nsteps, vo_moments* hist)
{
    if (!P || !f || P->nx < 1 || P->np < 1 || nsteps < 0) return -1;
    const long nx = P->nx, np = P->np;
    const size_t cells = (size_t)nx * (size_t)np;
    double* s_row = (double*)malloc(sizeof(double) * (size_t)np);
    double* s_col = (double*)malloc(sizeof(double) * (size_t)nx);
    double* rho = (double*)malloc(sizeof(double) * (size_t)nx);
    double* F = (double*)malloc(sizeof(double) * (size_t)nx);
    double* a = (double*)malloc(sizeof(double) * cells);
    double* b = (double*)malloc(sizeof(double) * cells);
    if (!s_row || !s_col || !rho || !F || !a || !b) {
        free(s_row); free(s_col); free(rho); free(F); free(a); free(b);
        return -1;
    }
    vo_xshift_cells(P, s_row);
    for (long n = 0; n < nsteps; ++n) {
        vo_advect_x(P, f, s_row, a);             /* step 1: f^(I) = f(x - p dt/2, p) */
        vo_density(P, a, rho);                   /* step 2: F^(I) from f^(I) */
        vo_force(P, rho, F);
        vo_pshift_cells(P, F, s_col);
        vo_advect_p(P, a, s_col, b);             /* step 3: f^(II) = f^(I)(x, p - F dt) */
        vo_advect_x(P, b, s_row, f);             /* step 4: f(t+dt) = f^(II)(x - p dt/2, p) */
        if (hist) {
            vo_moments_of(P, f, &hist[n]);
            hist[n].t = (double)(n + 1) * P->dt;
        }
    }
    free(s_row); free(s_col); free(rho); free(F); free(a); free(b);
    return 0;
}

int vo_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
