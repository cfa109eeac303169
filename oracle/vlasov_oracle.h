/*
 * vlasov_oracle.h -- plain FP64 CPU oracle for the Strang-split semi-Lagrangian Vlasov step.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent reference that the CUDA path is
 * checked against.  It shares no code, header, table or helper with the CUDA library; only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may load it.
 *
 * Paper: T. M. Rocha Filho, "Solving the Vlasov equation for one-dimensional models with long
 * range interactions on a GPU" (arXiv:1206.3229).  Each function cites the section / equation it
 * follows.  Storage follows Sec. 3: f[j*nx + i] with x (or theta) fastest and p rows.
 */
#ifndef VLASOV_ORACLE_H
#define VLASOV_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { VO_HMF = 0, VO_RING = 1, VO_SHEET = 2, VO_FREE = 3 };

typedef struct {
    int model;                 /* VO_HMF / VO_RING / VO_SHEET / VO_FREE (F = 0) */
    long nx, np;               /* grid points along x (theta) and p */
    double xmin, xmax;         /* x nodes: x_i = xmin + i*dx, dx = (xmax-xmin)/nx */
    double pmin, pmax;         /* p nodes: p_j = pmin + j*dp, dp = (pmax-pmin)/np */
    int x_periodic, p_periodic;/* 1: wrap; 0: f = 0 (and f'' = 0) outside the grid */
    double eps;                /* ring softening, Eq. (ringpot) */
    double G;                  /* sheet coupling: V = 2*pi*G*|x - x'| */
    double dt;                 /* time step */
    int spline;                /* 0: f'' by Eq. (findif) (the paper's method); 1: global spline,
                                  f'' from the tridiagonal system of Eq. (tridiagsys) */
} vo_params;

typedef struct {
    double t, mass, Mx, My, kinetic, potential, energy, l2;
} vo_moments;

/* Eq. (findif): f''_k = (1/du^2) sum_{m=-4..4} c_|m| f_{k+m} along one line of n points. */
void vo_fd2(const double* f, long n, int periodic, double du, double* d2);

/* Eq. (tridiagsys), the global cubic spline the paper compares against (Tables 1-2): f'' of the
   n nodes from (f''_{k-1}/6 + 2 f''_k/3 + f''_{k+1}/6) du^2 = f_{k+1} - 2 f_k + f_{k-1}.
   Periodic lines: the cyclic system.  Non-periodic lines: f = 0 and f'' = 0 at the nodes -1 and n
   next to the grid (a natural spline through the zero-extended data), f'' = 0 further out. */
void vo_gs2(const double* f, long n, int periodic, double du, double* d2);

/* Eqs. (splinegen, splinecoeffs): value at the foot y_i = i - s (s in cells) of every node i. */
void vo_spline_shift(const double* f, const double* d2, long n, int periodic, double du,
                     double s, double* out);

/* Eq. (step1)/(step4): every row j moved by s_row[j] cells along x. */
void vo_advect_x(const vo_params* P, const double* f, const double* s_row, double* out);
/* Eq. (step3): every column i moved by s_col[i] cells along p. */
void vo_advect_p(const vo_params* P, const double* f, const double* s_col, double* out);

/* Row displacement of the half free-streaming step, in cells: s_j = p_j * ((dt/2)/dx). */
void vo_xshift_cells(const vo_params* P, double* s_row);

/* rho_i = dp * sum_j f[j, i]. */
void vo_density(const vo_params* P, const double* f, double* rho);
/* Eq. (meanforce) / (hmfmeanforce) discretised by the rectangle rule on the x nodes. */
void vo_force(const vo_params* P, const double* rho, double* F);
/* p-displacement in cells of every column: s_i = F_i * (dt/dp). */
void vo_pshift_cells(const vo_params* P, const double* F, double* s_col);

/* Entropy Casimir of Eq. (casimirs), s(f) = -f log f: -dx dp sum over nodes with f > 0 of f ln f. */
double vo_entropy(const vo_params* P, const double* f);

/* mass, magnetisation, kinetic, potential, total energy and the L2 Casimir of f. */
void vo_moments_of(const vo_params* P, const double* f, vo_moments* out);

/* Sec. 3 steps 1-4, nsteps times, in place on f (np*nx doubles).  hist (may be NULL) receives
   the moments of f after every step.  Returns 0, or -1 on bad arguments / allocation failure. */
int vo_run(const vo_params* P, double* f, long nsteps, vo_moments* hist);

/* One Strang step split into its pieces (for tests): f1 = x-half-shift(f), F = force(f1),
   f2 = p-shift(f1), out = x-half-shift(f2).  Any of f1/F/f2 may be NULL. */
int vo_step_parts(const vo_params* P, const double* f, double* f1, double* F, double* f2,
                  double* out);

/* OpenMP threads used by the line sweeps (0 = library default).  Returns the count in use. */
int vo_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
