/*
 * osbli_oracle.c -- plain, slow, FP64 CPU oracle of the OpenSBLI residual / RK-stage path
 * (Lusher, Jammy & Sandham, "OpenSBLI: Automated code-generation for heterogeneous computing
 * architectures applied to compressible fluid dynamics on structured grids", arXiv:2007.14933).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's CPU
 * baseline load this library.  It shares no code, header, table or constant with the CUDA
 * path, and it never calls it.
 *
 * Every function states the passage of the paper it restates.  Where the paper is silent or
 * garbled the reading taken is stated at the place it is used; the same list is kept in the
 * design notes.  No blocking, fusion or reordering beyond what the definitions state: each
 * grid point's residual is evaluated on its own from the ghosted state (interface fluxes and
 * viscous fluxes are recomputed wherever they are needed).
 *
 * Conventions
 *   - State U: five conserved variables (rho, rho*u, rho*v, rho*w, rho*E), structure of arrays
 *     [5][nz][ny][nx], x fastest.  A direction with n = 1 is inactive (no ghosts, no flux).
 *   - Computational coordinates xi_d have unit spacing; physical coordinates x(xi) are given
 *     per interior node (or i*h_d on a uniform grid).
 *   - Curvilinear form (Sec. 2.7 gives no equations; reading): strong conservation form
 *       dU/dt = -(1/Jinv) sum_d d/dxi_d ( S_d . F_cart(U) ) + viscous terms,
 *     with S_d = Jinv grad(xi_d) (cross products of the coordinate derivatives) and
 *     Jinv = det(dx/dxi).  S_d is normalised by s_d = max over the interior of |S_d|, so that
 *     on a uniform Cartesian grid the reconstructed flux is the physical flux itself.
 *   - Ghost width 3 (the WENO5/TENO5/TENO6 stencil i-2..i+3 of Sec. 2.2-2.5).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no contraction: every product and
 * sum is rounded as written).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 5
#define GH 3

enum { ORC_CENTRAL4 = 0, ORC_WENO5JS = 1, ORC_TENO5 = 2, ORC_WENO5Z = 3, ORC_TENO6 = 4 };
enum { ORC_PERIODIC = 0, ORC_ZEROGRAD = 1, ORC_WALL = 2, ORC_DIRICHLET = 3, ORC_INFLOW = 4, ORC_ADIABATIC = 5 };

typedef struct {
    int n[3];              /* interior points per direction, 1 = inactive */
    double gamma, Re, Pr, Ma;  /* Re <= 0: inviscid */
    double dt;
    int scheme;            /* ORC_CENTRAL4 | ORC_WENO5JS | ORC_TENO5 | ORC_WENO5Z | ORC_TENO6 */
    double teno_ct;        /* TENO cut-off C_T */
    int bc[3][2];          /* per direction, side */
    double T_wall;         /* isothermal wall temperature */
    double suth;           /* T_s/T_ref for Sutherland's law; <= 0: mu = 1 */
    double h[3];           /* uniform spacing when coords == NULL */
    double L[3];           /* period of each periodic direction for given coords (uniform grid: n*h) */
    const double *coords;  /* [3][nz][ny][nx] physical coordinates or NULL */
    const double *bdata[6];/* face 2*d+s: [5][plane] Dirichlet (rho,u,v,w,p) or inflow (-,u,v,w,T) */
    int rk;                /* 0: 3-stage RK3, 1: 5-stage RK4 (both low-storage 2N) */
    double force[3];       /* body force per unit volume (momentum) and its work f.u (energy) */
} orc_params;

typedef struct {
    orc_params p;
    int g[3], np[3];
    long st[3];
    long ntot;
    double *U;      /* [5][ntot] ghosted state */
    double *dU;     /* [5][ntot] RK register */
    double *Rw;     /* [5][ntot] residual work */
    double *S;      /* [3 dir][3 comp][ntot] normalised contravariant metric S~_d */
    double *Jr;     /* [ntot] 1/Jinv */
    double shat[3];
    int active[3];
    double margin_min;  /* smallest TENO |chi - C_T|/C_T seen by the last residual */
    double *Vn;         /* [3 dir][4 comp][nz][ny][nx] viscous flux of every interior node of the
                           current state (filled before each residual; each value is computed
                           once and read by the divergences that need it) */
    int vn_valid;       /* Vn holds the current state's fluxes */
    unsigned char *gate;/* cell gate of the gated convective form ([nz][ny][nx]) or NULL */
    double jump;        /* strong-jump ratio of the gated form */
} orc_ctx;

/* ------------------------------------------------------------------------------------------
 * ENO candidate coefficients c_rj and optimal weights d_r (Eqs. 14-15, Sec. 2.3).
 * The paper cites them "from Shu 1997" without printing them.  They are derived here from their
 * definition: the candidate f^(r)_{i+1/2} is the derivative at x_{i+1/2} of the degree-k
 * polynomial that interpolates the primitive function H(x_{j+1/2}) = sum_{l<=j} f_l on the k+1
 * cell edges of the stencil {i-r, ..., i-r+k-1} (unit spacing, cell averages f).
 * ------------------------------------------------------------------------------------------ */
static double lagrange_deriv_at0(const double *t, int npts, int m)
{
    /* d/dx of the m-th Lagrange basis polynomial on nodes t[0..npts-1], evaluated at x = 0 */
    double sum = 0.0;
    for (int q = 0; q < npts; q++) {
        if (q == m) continue;
        double prod = 1.0 / (t[m] - t[q]);
        for (int s = 0; s < npts; s++) {
            if (s == m || s == q) continue;
            prod *= (0.0 - t[s]) / (t[m] - t[s]);
        }
        sum += prod;
    }
    return sum;
}

/* c[r*k + j] for r, j in [0, k): reconstruction at x_{i+1/2} from f_{i-r+j} */
void orc_eno_coeffs(int k, double *c)
{
    double t[16];
    for (int r = 0; r < k; r++) {
        /* edges x_{i-r-1/2+m}, m = 0..k, measured from x_{i+1/2}: m - r - 1 */
        for (int m = 0; m <= k; m++) t[m] = (double)(m - r - 1);
        for (int j = 0; j < k; j++) {
            double s = 0.0;
            for (int m = j + 1; m <= k; m++) s += lagrange_deriv_at0(t, k + 1, m);
            c[r * k + j] = s;
        }
    }
}

static double C3[3][3];   /* c_rj, k = 3 */
static double D3[3];      /* d_r, 5th order */
static int coeffs_ready = 0;

/* Optimal weights: the unique d_r with sum_r d_r f^(r) equal to the 5-point (2k-1 = 5)
 * reconstruction on {i-2..i+2} (Eq. 15 with linear weights).  Solved from the two end
 * coefficients (each touched by one candidate only) and consistency sum d_r = 1. */
void orc_linear_weights(double d[3])
{
    double c5[25];
    orc_eno_coeffs(5, c5);          /* row r = 2: stencil i-2..i+2 */
    const double *big = &c5[2 * 5]; /* coefficient of f_{i-2+j} */
    double c[9];
    orc_eno_coeffs(3, c);
    /* f_{i-2} appears only in candidate r=2 (j=0); f_{i+2} only in r=0 (j=2) */
    d[2] = big[0] / c[2 * 3 + 0];
    d[0] = big[4] / c[0 * 3 + 2];
    d[1] = 1.0 - d[0] - d[2];
}

static double C4[4];      /* TENO6 fourth candidate: reconstruction at x_{i+1/2} from f_{i..i+3} */
static double D6[4];      /* d_r, TENO6 */

/* TENO6 linear weights (Sec. 2.5; the values are not printed).  Reading: the unique d_r with
 * sum_r d_r f^(r) equal to the 6-point reconstruction on {i-2..i+3}, the candidates being the
 * three 3-point stencils of the 5th-order schemes (r = 0: {i..i+2}, 1: {i-1..i+1}, 2:
 * {i-2..i}) and the 4-point stencil r = 3: {i..i+3}.  Solved coefficient by coefficient:
 * f_{i-2} only in r = 2, f_{i+3} only in r = 3, f_{i-1} in r = 1 and 2, then sum d_r = 1. */
void orc_teno6_linear_weights(double d[4])
{
    double c6[36], c3[9], c4[16];
    orc_eno_coeffs(6, c6);
    orc_eno_coeffs(3, c3);
    orc_eno_coeffs(4, c4);
    const double *big = &c6[2 * 6];      /* coefficient of f_{i-2+j}, j = 0..5 */
    d[2] = big[0] / c3[2 * 3 + 0];
    d[3] = big[5] / c4[0 * 4 + 3];
    d[1] = (big[1] - d[2] * c3[2 * 3 + 1]) / c3[1 * 3 + 0];
    d[0] = 1.0 - d[1] - d[2] - d[3];
}

static void init_coeffs(void)
{
    if (coeffs_ready) return;
    double c[9], c4[16];
    orc_eno_coeffs(3, c);
    for (int r = 0; r < 3; r++)
        for (int j = 0; j < 3; j++) C3[r][j] = c[r * 3 + j];
    orc_linear_weights(D3);
    orc_eno_coeffs(4, c4);
    for (int j = 0; j < 4; j++) C4[j] = c4[j];
    orc_teno6_linear_weights(D6);
    coeffs_ready = 1;
}

/* ------------------------------------------------------------------------------------------
 * Smoothness indicators, Eqs. 17-19 (Sec. 2.3), as printed.  f[0..4] = f_{i-2..i+2}.
 * ------------------------------------------------------------------------------------------ */
void orc_smoothness5(const double *f, double *beta)
{
    double a, b;
    a = f[2] - 2.0 * f[3] + f[4];
    b = 3.0 * f[2] - 4.0 * f[3] + f[4];
    beta[0] = (13.0 / 12.0) * a * a + 0.25 * b * b;
    a = f[1] - 2.0 * f[2] + f[3];
    b = f[1] - f[3];
    beta[1] = (13.0 / 12.0) * a * a + 0.25 * b * b;
    a = f[0] - 2.0 * f[1] + f[2];
    b = f[0] - 4.0 * f[1] + 3.0 * f[2];
    beta[2] = (13.0 / 12.0) * a * a + 0.25 * b * b;
}

/* Nonlinear weights.  WENO-JS: Eqs. 20-21 (p = 2, eps = 1e-6).  WENO-Z: Eq. 22 with
 * sigma_r = beta_r, tau = |beta_0 - beta_2|, eps = 1e-16, alpha_r = d_r (1 + (tau / (beta_r +
 * eps))^2).  TENO5: Eqs. 23-27
 * (C = 1, q = 6, eps = 1e-16, tau_5 = |beta_0 - beta_2|, cut-off C_T).  Returns in *margin the
 * smallest |chi_r - C_T|/C_T (TENO only; used to recognise cut-off decisions that sit on the
 * threshold within rounding). */
void orc_weights5(const double *beta, int scheme, double ct, double *w, double *margin)
{
    init_coeffs();
    if (scheme == ORC_WENO5Z) {
        const double eps = 1e-16;
        const double tau = fabs(beta[0] - beta[2]);
        double a[3], s = 0.0;
        for (int r = 0; r < 3; r++) {
            const double x = tau / (beta[r] + eps);
            a[r] = D3[r] * (1.0 + x * x);
            s += a[r];
        }
        for (int r = 0; r < 3; r++) w[r] = a[r] / s;
        if (margin) *margin = INFINITY;
    } else if (scheme == ORC_WENO5JS) {
        const double eps = 1e-6;
        double a[3], s = 0.0;
        for (int r = 0; r < 3; r++) {
            double e = eps + beta[r];
            a[r] = D3[r] / (e * e);
            s += a[r];
        }
        for (int r = 0; r < 3; r++) w[r] = a[r] / s;
        if (margin) *margin = INFINITY;
    } else {
        const double eps = 1e-16;
        double tau = fabs(beta[0] - beta[2]);
        double gam[3], sg = 0.0;
        for (int r = 0; r < 3; r++) {
            double t = 1.0 + tau / (beta[r] + eps);
            double t2 = t * t;
            gam[r] = t2 * t2 * t2;
            sg += gam[r];
        }
        double dsum = 0.0, dl[3], mg = INFINITY;
        for (int r = 0; r < 3; r++) {
            double chi = gam[r] / sg;
            int delta = (chi < ct) ? 0 : 1;
            double m = fabs(chi - ct) / ct;
            if (m < mg) mg = m;
            dl[r] = D3[r] * (double)delta;
            dsum += dl[r];
        }
        for (int r = 0; r < 3; r++) w[r] = dl[r] / dsum;
        if (margin) *margin = mg;
    }
}

/* Smoothness indicator of the 4-point TENO6 stencil {i..i+3} (g[0..3] = f_{i..i+3}): the
 * Jiang-Shu measure of Eq. 16 for k = 4 (sum over l = 1..3 of dx^(2l-1) times the integral over
 * cell i of the squared l-th derivative of the cubic whose cell averages are g), written out. */
double orc_smoothness_cubic(const double *g)
{
    const double a = -11.0 * g[0] + 18.0 * g[1] - 9.0 * g[2] + 2.0 * g[3];
    const double b = 2.0 * g[0] - 5.0 * g[1] + 4.0 * g[2] - g[3];
    const double c = -g[0] + 3.0 * g[1] - 3.0 * g[2] + g[3];
    return a * a / 36.0 + (13.0 / 12.0) * b * b + (781.0 / 720.0) * c * c;
}

/* TENO6 weights (Eqs. 23-27 with K = 6): gamma_r = (1 + tau_6 / (beta_r + eps))^6, r = 0..3,
 * tau_6 = |beta_3 - (beta_0 + beta_2 + 4 beta_1) / 6| as printed, eps = 1e-16, chi_r =
 * gamma_r / sum gamma, delta_r = [chi_r >= C_T], omega_r = d_r delta_r / sum d delta.  *margin
 * as for TENO5. */
void orc_weights6(const double *beta, double ct, double *w, double *margin)
{
    init_coeffs();
    const double eps = 1e-16;
    const double tau = fabs(beta[3] - (beta[0] + beta[2] + 4.0 * beta[1]) / 6.0);
    double gam[4], sg = 0.0;
    for (int r = 0; r < 4; r++) {
        double t = 1.0 + tau / (beta[r] + eps);
        double t2 = t * t;
        gam[r] = t2 * t2 * t2;
        sg += gam[r];
    }
    double dsum = 0.0, dl[4], mg = INFINITY;
    for (int r = 0; r < 4; r++) {
        double chi = gam[r] / sg;
        int delta = (chi < ct) ? 0 : 1;
        double m = fabs(chi - ct) / ct;
        if (m < mg) mg = m;
        dl[r] = D6[r] * (double)delta;
        dsum += dl[r];
    }
    for (int r = 0; r < 4; r++) w[r] = dl[r] / dsum;
    if (margin) *margin = mg;
}

/* TENO6 reconstruction of the value at x_{i+1/2} from f[0..5] = f_{i-2..i+3}. */
double orc_recon6(const double *f, double ct, double *wout, double *margin)
{
    init_coeffs();
    double beta[4], w[4], fr[4];
    orc_smoothness5(f, beta);
    beta[3] = orc_smoothness_cubic(f + 2);
    orc_weights6(beta, ct, w, margin);
    for (int r = 0; r < 3; r++) {
        double s = 0.0;
        for (int j = 0; j < 3; j++) s += C3[r][j] * f[2 - r + j];
        fr[r] = s;
    }
    fr[3] = 0.0;
    for (int j = 0; j < 4; j++) fr[3] += C4[j] * f[2 + j];
    if (wout)
        for (int r = 0; r < 4; r++) wout[r] = w[r];
    return w[0] * fr[0] + w[1] * fr[1] + w[2] * fr[2] + w[3] * fr[3];
}

/* Reconstruction of the value at x_{i+1/2} from f[0..4] = f_{i-2..i+2} (Eqs. 14-15). */
double orc_recon5(const double *f, int scheme, double ct, double *wout, double *margin)
{
    init_coeffs();
    double beta[3], w[3];
    orc_smoothness5(f, beta);
    orc_weights5(beta, scheme, ct, w, margin);
    double fr[3];
    for (int r = 0; r < 3; r++) {
        double s = 0.0;
        for (int j = 0; j < 3; j++) s += C3[r][j] * f[2 - r + j];
        fr[r] = s;
    }
    if (wout) { wout[0] = w[0]; wout[1] = w[1]; wout[2] = w[2]; }
    return w[0] * fr[0] + w[1] * fr[1] + w[2] * fr[2];
}

/* ------------------------------------------------------------------------------------------
 * Thermodynamics (Eqs. 4-7).
 * ------------------------------------------------------------------------------------------ */
typedef struct { double rho, u[3], p, T, a, H; } prim_t;

static void primitives(const orc_params *P, const double *U, prim_t *w)
{
    double g = P->gamma;
    w->rho = U[0];
    for (int c = 0; c < 3; c++) w->u[c] = U[1 + c] / U[0];
    double q2 = w->u[0] * w->u[0] + w->u[1] * w->u[1] + w->u[2] * w->u[2];
    w->p = (g - 1.0) * (U[4] - 0.5 * U[0] * q2);                /* Eq. 7 */
    w->T = g * P->Ma * P->Ma * w->p / U[0];                     /* p = rho T/(gamma M^2) */
    w->a = sqrt(g * w->p / U[0]);
    w->H = (U[4] + w->p) / U[0];
}

static double viscosity(const orc_params *P, double T)
{
    if (P->suth <= 0.0) return 1.0;
    return pow(T, 1.5) * (1.0 + P->suth) / (T + P->suth);      /* Eq. 6 */
}

double orc_sutherland(double T, double suth)
{
    orc_params P;
    memset(&P, 0, sizeof P);
    P.suth = suth;
    return viscosity(&P, T);
}

/* Convective flux along the (unnormalised) metric vector S: S . (F, G, H)  (Eqs. 1-3). */
void orc_flux(double gamma, const double *U, const double *S, double *F)
{
    double rho = U[0], u = U[1] / rho, v = U[2] / rho, w = U[3] / rho;
    double p = (gamma - 1.0) * (U[4] - 0.5 * rho * (u * u + v * v + w * w));
    double Un = S[0] * u + S[1] * v + S[2] * w;
    F[0] = rho * Un;
    F[1] = U[1] * Un + S[0] * p;
    F[2] = U[2] * Un + S[1] * p;
    F[3] = U[3] * Un + S[2] * p;
    F[4] = (U[4] + p) * Un;
}

/* ------------------------------------------------------------------------------------------
 * Roe-averaged eigensystem (Sec. 2.2 steps (a)-(b)).  The paper prints no eigenvectors; the
 * textbook Euler eigenvectors along a unit normal n are used, ordered by eigenvalue
 * (u_n - a, u_n, u_n, u_n, u_n + a).  The three u_n fields are the entropy wave and two shear
 * waves along tangents t1, t2:  t1 = normalise(z x n) if |n_z| < 0.9 else normalise(n x x),
 * t2 = n x t1.  R holds the right eigenvectors as columns (R[row*5+col]); L = R^-1.
 * ------------------------------------------------------------------------------------------ */
static void tangents(const double *n, double *t1, double *t2)
{
    if (fabs(n[2]) < 0.9) {
        double m = sqrt(n[0] * n[0] + n[1] * n[1]);
        t1[0] = -n[1] / m; t1[1] = n[0] / m; t1[2] = 0.0;
    } else {
        double m = sqrt(n[2] * n[2] + n[1] * n[1]);
        t1[0] = 0.0; t1[1] = n[2] / m; t1[2] = -n[1] / m;
    }
    t2[0] = n[1] * t1[2] - n[2] * t1[1];
    t2[1] = n[2] * t1[0] - n[0] * t1[2];
    t2[2] = n[0] * t1[1] - n[1] * t1[0];
}

static void eigensystem(double g, const double *u, double H, double a, const double *n,
                        double *R, double *L)
{
    double t1[3], t2[3];
    tangents(n, t1, t2);
    double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    double ut1 = u[0] * t1[0] + u[1] * t1[1] + u[2] * t1[2];
    double ut2 = u[0] * t2[0] + u[1] * t2[1] + u[2] * t2[2];
    /* right eigenvectors (columns) */
    double col[5][5];
    col[0][0] = 1.0; col[1][0] = 1.0; col[2][0] = 0.0; col[3][0] = 0.0; col[4][0] = 1.0;
    for (int c = 0; c < 3; c++) {
        col[0][1 + c] = u[c] - a * n[c];
        col[1][1 + c] = u[c];
        col[2][1 + c] = t1[c];
        col[3][1 + c] = t2[c];
        col[4][1 + c] = u[c] + a * n[c];
    }
    col[0][4] = H - a * un;
    col[1][4] = 0.5 * q2;
    col[2][4] = ut1;
    col[3][4] = ut2;
    col[4][4] = H + a * un;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j < 5; j++) R[i * 5 + j] = col[j][i];
    /* left eigenvectors (rows) */
    double b1 = (g - 1.0) / (a * a);
    double b2 = 0.5 * b1 * q2;
    L[0 * 5 + 0] = 0.5 * (b2 + un / a);
    L[4 * 5 + 0] = 0.5 * (b2 - un / a);
    L[1 * 5 + 0] = 1.0 - b2;
    L[2 * 5 + 0] = -ut1;
    L[3 * 5 + 0] = -ut2;
    for (int c = 0; c < 3; c++) {
        L[0 * 5 + 1 + c] = -0.5 * (b1 * u[c] + n[c] / a);
        L[4 * 5 + 1 + c] = -0.5 * (b1 * u[c] - n[c] / a);
        L[1 * 5 + 1 + c] = b1 * u[c];
        L[2 * 5 + 1 + c] = t1[c];
        L[3 * 5 + 1 + c] = t2[c];
    }
    L[0 * 5 + 4] = 0.5 * b1;
    L[4 * 5 + 4] = 0.5 * b1;
    L[1 * 5 + 4] = -b1;
    L[2 * 5 + 4] = 0.0;
    L[3 * 5 + 4] = 0.0;
}

/* Roe average of two states (Sec. 2.2 step (a), averaging = Roe). */
static void roe_average(const orc_params *P, const double *UL, const double *UR,
                        double *u, double *H, double *a)
{
    prim_t wl, wr;
    primitives(P, UL, &wl);
    primitives(P, UR, &wr);
    double rl = sqrt(wl.rho), rr = sqrt(wr.rho);
    double inv = 1.0 / (rl + rr);
    for (int c = 0; c < 3; c++) u[c] = (rl * wl.u[c] + rr * wr.u[c]) * inv;
    *H = (rl * wl.H + rr * wr.H) * inv;
    double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    *a = sqrt((P->gamma - 1.0) * (*H - 0.5 * q2));
}

/* Exposed for the eigensystem pins. */
void orc_eigensystem(double gamma, const double *UL, const double *UR, const double *n,
                     double *R, double *L, double *lam)
{
    orc_params P;
    memset(&P, 0, sizeof P);
    P.gamma = gamma;
    P.Ma = 1.0;
    double u[3], H, a;
    roe_average(&P, UL, UR, u, &H, &a);
    eigensystem(gamma, u, H, a, n, R, L);
    double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    lam[0] = un - a; lam[1] = un; lam[2] = un; lam[3] = un; lam[4] = un + a;
}

/* ------------------------------------------------------------------------------------------
 * Grid / ghost bookkeeping.
 * ------------------------------------------------------------------------------------------ */
static inline long IDX(const orc_ctx *c, int i, int j, int k)
{
    return ((long)(k + c->g[2]) * c->np[1] + (j + c->g[1])) * c->np[0] + (i + c->g[0]);
}

static inline int wrapi(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* physical coordinate component cc of interior node (i,j,k), with periodic unwrapping for
 * indices outside [0, n) of a periodic direction (shift L_d along Cartesian axis d) */
static double coord(const orc_ctx *c, int cc, int i, int j, int k)
{
    const orc_params *P = &c->p;
    int ii[3] = {i, j, k};
    double shift = 0.0;
    for (int d = 0; d < 3; d++) {
        int n = P->n[d];
        if (ii[d] < 0 || ii[d] >= n) {
            int w = wrapi(ii[d], n);
            int periods = (ii[d] - w) / n;
            /* period of the direction: L_d for given coordinates, n_d h_d on a uniform grid */
            double period = P->coords ? P->L[d] : n * P->h[d];
            if (cc == d) shift += periods * period;
            ii[d] = w;
        }
    }
    if (!P->coords) return ii[cc] * P->h[cc] + shift;
    long plane = (long)P->n[0] * P->n[1] * P->n[2];
    long id = ((long)ii[2] * P->n[1] + ii[1]) * P->n[0] + ii[0];
    return P->coords[cc * plane + id] + shift;
}

/* 4th-order first derivative along a line of values f(s) for s = 0..N-1 (Sec. 2.6):
 * central interior formula (sign as in the generated kernel of Sec. 4; the printed Eq. 28 has
 * it reversed), Ekaterinaris one-sided closures (Eqs. 30-33) at 0, 1, N-2, N-1 of a
 * non-periodic line.  fetch(s) returns f at line index s (callers wrap periodic indices). */
typedef double (*fetch_fn)(const void *ud, int s);

static double deriv4(fetch_fn f, const void *ud, int i, int N, int periodic)
{
    if (periodic || (i >= 2 && i <= N - 3))
        return (f(ud, i - 2) - 8.0 * f(ud, i - 1) + 8.0 * f(ud, i + 1) - f(ud, i + 2)) / 12.0;
    if (i == 0)
        return (-25.0 * f(ud, 0) + 48.0 * f(ud, 1) - 36.0 * f(ud, 2) + 16.0 * f(ud, 3) - 3.0 * f(ud, 4)) / 12.0;
    if (i == 1)
        return (-3.0 * f(ud, 0) - 10.0 * f(ud, 1) + 18.0 * f(ud, 2) - 6.0 * f(ud, 3) + f(ud, 4)) / 12.0;
    if (i == N - 2)
        return (-f(ud, N - 5) + 6.0 * f(ud, N - 4) - 18.0 * f(ud, N - 3) + 10.0 * f(ud, N - 2) + 3.0 * f(ud, N - 1)) / 12.0;
    /* i == N - 1 */
    return (3.0 * f(ud, N - 5) - 16.0 * f(ud, N - 4) + 36.0 * f(ud, N - 3) - 48.0 * f(ud, N - 2) + 25.0 * f(ud, N - 1)) / 12.0;
}

/* exposed for the operator pins: derivative of samples v[0..N-1] at index i */
typedef struct { const double *v; int N; int periodic; } arr_ud;
static double arr_fetch(const void *ud, int s)
{
    const arr_ud *a = (const arr_ud *)ud;
    int t = a->periodic ? wrapi(s, a->N) : s;
    return a->v[t];
}
double orc_deriv4(const double *v, int N, int i, int periodic)
{
    arr_ud a = {v, N, periodic};
    return deriv4(arr_fetch, &a, i, N, periodic);
}

/* coordinate fetch along direction d for the metric derivatives */
typedef struct { const orc_ctx *c; int cc, d, i, j, k; } crd_ud;
/* Coordinate at line index s relative to the stencil's centre node.  The difference operator
 * annihilates constants (its coefficients sum to zero), so this changes nothing but rounding;
 * on a uniform grid the offsets (s - centre) h are exact and so are the metrics. */
static double crd_fetch(const void *ud, int s)
{
    const crd_ud *a = (const crd_ud *)ud;
    const orc_ctx *c = a->c;
    int ii[3] = {a->i, a->j, a->k};
    int centre = ii[a->d];
    if (!c->p.coords) {
        /* uniform grid: x_cc depends on index cc only */
        return a->cc == a->d ? (double)(s - centre) * c->p.h[a->cc] : 0.0;
    }
    double x0 = coord(c, a->cc, ii[0], ii[1], ii[2]);
    ii[a->d] = s;
    return coord(c, a->cc, ii[0], ii[1], ii[2]) - x0;
}

static void cross(const double *a, const double *b, double *r)
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

/* Metric terms (Sec. 2.7: computed once, with the same central/one-sided schemes).
 * X[d][cc] = d x_cc / d xi_d; inactive direction: unit vector.  S_0 = X_1 x X_2,
 * S_1 = X_2 x X_0, S_2 = X_0 x X_1, Jinv = X_0 . S_0. */
static void metric_at(const orc_ctx *c, int i, int j, int k, double S[3][3], double *Jinv)
{
    const orc_params *P = &c->p;
    double X[3][3];
    int ii[3] = {i, j, k};
    for (int d = 0; d < 3; d++) {
        for (int cc = 0; cc < 3; cc++) {
            if (!c->active[d]) { X[d][cc] = (cc == d) ? 1.0 : 0.0; continue; }
            crd_ud ud = {c, cc, d, i, j, k};
            int per = P->bc[d][0] == ORC_PERIODIC;
            X[d][cc] = deriv4(crd_fetch, &ud, ii[d], P->n[d], per);
        }
    }
    cross(X[1], X[2], S[0]);
    cross(X[2], X[0], S[1]);
    cross(X[0], X[1], S[2]);
    *Jinv = X[0][0] * S[0][0] + X[0][1] * S[0][1] + X[0][2] * S[0][2];
}

/* map a (possibly ghost) index to the interior node whose metric it takes: periodic wrap,
 * non-periodic mirror about the boundary node (reading: the paper does not define ghost-node
 * metrics; mirrored coordinates x_{-i} = 2 x_0 - x_i give the mirrored derivative). */
static int metric_src(const orc_ctx *c, int d, int i)
{
    int n = c->p.n[d];
    if (i >= 0 && i < n) return i;
    if (c->p.bc[d][0] == ORC_PERIODIC) return wrapi(i, n);
    if (i < 0) return -i;
    return 2 * (n - 1) - i;
}

static void compute_metrics(orc_ctx *c)
{
    const orc_params *P = &c->p;
    long nt = c->ntot;
    /* interior first */
    double *Sraw = (double *)malloc(sizeof(double) * 9 * nt);
    double *Jv = (double *)malloc(sizeof(double) * nt);
    for (int k = 0; k < P->n[2]; k++)
        for (int j = 0; j < P->n[1]; j++)
            for (int i = 0; i < P->n[0]; i++) {
                double S[3][3], J;
                metric_at(c, i, j, k, S, &J);
                long id = IDX(c, i, j, k);
                for (int d = 0; d < 3; d++)
                    for (int cc = 0; cc < 3; cc++) Sraw[(d * 3 + cc) * nt + id] = S[d][cc];
                Jv[id] = J;
            }
    for (int d = 0; d < 3; d++) {
        double mx = 0.0;
        for (int k = 0; k < P->n[2]; k++)
            for (int j = 0; j < P->n[1]; j++)
                for (int i = 0; i < P->n[0]; i++) {
                    long id = IDX(c, i, j, k);
                    double s0 = Sraw[(d * 3 + 0) * nt + id], s1 = Sraw[(d * 3 + 1) * nt + id],
                           s2 = Sraw[(d * 3 + 2) * nt + id];
                    double m = sqrt(s0 * s0 + s1 * s1 + s2 * s2);
                    if (m > mx) mx = m;
                }
        c->shat[d] = mx;
    }
    /* all nodes incl. ghosts from their source interior node */
    for (int k = -c->g[2]; k < P->n[2] + c->g[2]; k++)
        for (int j = -c->g[1]; j < P->n[1] + c->g[1]; j++)
            for (int i = -c->g[0]; i < P->n[0] + c->g[0]; i++) {
                long id = IDX(c, i, j, k);
                long src = IDX(c, metric_src(c, 0, i), metric_src(c, 1, j), metric_src(c, 2, k));
                for (int d = 0; d < 3; d++)
                    for (int cc = 0; cc < 3; cc++)
                        c->S[(d * 3 + cc) * nt + id] = Sraw[(d * 3 + cc) * nt + src] / c->shat[d];
                c->Jr[id] = 1.0 / Jv[src];
            }
    free(Sraw);
    free(Jv);
}

/* ------------------------------------------------------------------------------------------
 * Boundary conditions (Sec. 3.1.3 and Sec. 5-6 problem set-ups).
 *   PERIODIC   ghost = wrapped interior value.
 *   ZEROGRAD   ghost = copy of the boundary node (zero-order extrapolation; Sod ends, outlet).
 *   WALL       isothermal no-slip wall on the boundary node (Eqs. 40-46): ghost temperature
 *              T_{-i} = (i+1) T_w - i T_1, ghost density rho = M^2 gamma p_w / T_{-i}
 *              (the printed rho_{-1} read as rho_{-i}), momentum reflected
 *              rho u_{-i} = -rho_{-i} u_i, ghost pressure = p_w, the wall node's pressure.
 *              After each stage the wall node gets rho u_i = 0 and rho E = rho_w T_w /
 *              (M^2 gamma (gamma-1)) (Eq. 41); its density floats.
 *   DIRICHLET  ghosts and boundary node = the given primitive plane (rho,u,v,w,p).
 *   INFLOW     velocity and temperature from the given plane, pressure extrapolated from the
 *              first interior node (zero order), rho = gamma M^2 p / T; ghosts and node.
 *   ADIABATIC  no-slip wall with zero heat flux (the laminar channel of Sec. 5.4; the paper
 *              prints no discretisation): as WALL but the ghost temperature mirrors the interior,
 *              T_{-i} = T_i; after each stage the wall node gets rho u_i = 0 and the temperature
 *              that makes the one-sided 4th-order derivative (Eq. 30) vanish,
 *              T_w = (48 T_1 - 36 T_2 + 16 T_3 - 3 T_4) / 25, rho E = rho_w T_w / (M^2 gamma (gamma-1)).
 * The plane of a face lists the interior nodes of the two other directions (lower first
 * direction fastest); ghost lines of those directions clamp to the nearest interior line.
 * ------------------------------------------------------------------------------------------ */
static void set_from_prim(const orc_params *P, double *U, long id, long nt,
                          double rho, const double *u, double p)
{
    U[0 * nt + id] = rho;
    U[1 * nt + id] = rho * u[0];
    U[2 * nt + id] = rho * u[1];
    U[3 * nt + id] = rho * u[2];
    U[4 * nt + id] = p / (P->gamma - 1.0) + 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

static void load_state(const double *U, long id, long nt, double *u5)
{
    for (int v = 0; v < NV; v++) u5[v] = U[v * nt + id];
}

/* face plane index for a line at other-direction indices (a, b) */
static long plane_index(const orc_ctx *c, int d, int ia, int ib)
{
    int da = (d == 0) ? 1 : 0, db = (d == 2) ? 1 : 2;
    int na = c->p.n[da], nb = c->p.n[db];
    if (ia < 0) ia = 0;
    if (ia >= na) ia = na - 1;
    if (ib < 0) ib = 0;
    if (ib >= nb) ib = nb - 1;
    return (long)ib * na + ia;
}

static void face_prim(const orc_ctx *c, int d, int s, long pid, double *rho, double *u, double *x4)
{
    int da = (d == 0) ? 1 : 0, db = (d == 2) ? 1 : 2;
    long plane = (long)c->p.n[da] * c->p.n[db];
    const double *b = c->p.bdata[2 * d + s];
    *rho = b[0 * plane + pid];
    u[0] = b[1 * plane + pid];
    u[1] = b[2 * plane + pid];
    u[2] = b[3 * plane + pid];
    *x4 = b[4 * plane + pid];
}

static void ghost_fill(orc_ctx *c)
{
    const orc_params *P = &c->p;
    long nt = c->ntot;
    double *U = c->U;
    for (int d = 0; d < 3; d++) {
        if (!c->active[d]) continue;
        int n = P->n[d];
        int da = (d == 0) ? 1 : 0, db = (d == 2) ? 1 : 2;
        for (int s = 0; s < 2; s++) {
            int bc = P->bc[d][s];
            for (int ib = -c->g[db]; ib < P->n[db] + c->g[db]; ib++)
                for (int ia = -c->g[da]; ia < P->n[da] + c->g[da]; ia++) {
                    int ii[3];
                    ii[da] = ia; ii[db] = ib;
                    /* boundary node and first interior node of this line */
                    int nb_ = s == 0 ? 0 : n - 1, n1 = s == 0 ? 1 : n - 2;
                    ii[d] = nb_;
                    long idb = IDX(c, ii[0], ii[1], ii[2]);
                    ii[d] = n1;
                    long id1 = IDX(c, ii[0], ii[1], ii[2]);
                    prim_t wb, w1;
                    double ub[5], u1[5];
                    load_state(U, idb, nt, ub);
                    load_state(U, id1, nt, u1);
                    for (int gi = 1; gi <= GH; gi++) {
                        int gidx = s == 0 ? -gi : n - 1 + gi;
                        ii[d] = gidx;
                        long idg = IDX(c, ii[0], ii[1], ii[2]);
                        if (bc == ORC_PERIODIC) {
                            ii[d] = wrapi(gidx, n);
                            long src = IDX(c, ii[0], ii[1], ii[2]);
                            for (int v = 0; v < NV; v++) U[v * nt + idg] = U[v * nt + src];
                        } else if (bc == ORC_ZEROGRAD) {
                            for (int v = 0; v < NV; v++) U[v * nt + idg] = ub[v];
                        } else if (bc == ORC_WALL || bc == ORC_ADIABATIC) {
                            primitives(P, ub, &wb);
                            primitives(P, u1, &w1);
                            int mi = s == 0 ? gi : n - 1 - gi;   /* mirrored interior node */
                            ii[d] = mi;
                            long idm = IDX(c, ii[0], ii[1], ii[2]);
                            double um[5];
                            prim_t wm;
                            load_state(U, idm, nt, um);
                            primitives(P, um, &wm);
                            double Tg = bc == ORC_ADIABATIC ? wm.T : (gi + 1) * P->T_wall - gi * w1.T;
                            double rg = P->Ma * P->Ma * P->gamma * wb.p / Tg;
                            double ug[3] = {-wm.u[0], -wm.u[1], -wm.u[2]};
                            set_from_prim(P, U, idg, nt, rg, ug, wb.p);
                        } else if (bc == ORC_DIRICHLET) {
                            double r, u[3], p;
                            face_prim(c, d, s, plane_index(c, d, ia, ib), &r, u, &p);
                            set_from_prim(P, U, idg, nt, r, u, p);
                        } else if (bc == ORC_INFLOW) {
                            double r, u[3], T;
                            face_prim(c, d, s, plane_index(c, d, ia, ib), &r, u, &T);
                            primitives(P, u1, &w1);
                            double rr = P->gamma * P->Ma * P->Ma * w1.p / T;
                            set_from_prim(P, U, idg, nt, rr, u, w1.p);
                        }
                    }
                }
        }
    }
}

/* After-stage conditions on boundary nodes (walls, Dirichlet and inflow nodes). */
static void impose_boundary_nodes(orc_ctx *c)
{
    const orc_params *P = &c->p;
    long nt = c->ntot;
    double *U = c->U;
    for (int d = 0; d < 3; d++) {
        if (!c->active[d]) continue;
        int n = P->n[d];
        int da = (d == 0) ? 1 : 0, db = (d == 2) ? 1 : 2;
        for (int s = 0; s < 2; s++) {
            int bc = P->bc[d][s];
            if (bc != ORC_WALL && bc != ORC_DIRICHLET && bc != ORC_INFLOW && bc != ORC_ADIABATIC) continue;
            for (int ib = 0; ib < P->n[db]; ib++)
                for (int ia = 0; ia < P->n[da]; ia++) {
                    int ii[3];
                    ii[da] = ia; ii[db] = ib;
                    ii[d] = s == 0 ? 0 : n - 1;
                    long idb = IDX(c, ii[0], ii[1], ii[2]);
                    ii[d] = s == 0 ? 1 : n - 2;
                    long id1 = IDX(c, ii[0], ii[1], ii[2]);
                    if (bc == ORC_ADIABATIC) {
                        double Tn[5];
                        for (int q = 1; q <= 4; q++) {
                            ii[d] = s == 0 ? q : n - 1 - q;
                            double uq[5];
                            prim_t wq;
                            load_state(U, IDX(c, ii[0], ii[1], ii[2]), nt, uq);
                            primitives(P, uq, &wq);
                            Tn[q] = wq.T;
                        }
                        double Tw = (48.0 * Tn[1] - 36.0 * Tn[2] + 16.0 * Tn[3] - 3.0 * Tn[4]) / 25.0;
                        double rw = U[0 * nt + idb];
                        U[1 * nt + idb] = 0.0;
                        U[2 * nt + idb] = 0.0;
                        U[3 * nt + idb] = 0.0;
                        U[4 * nt + idb] = rw * Tw / (P->Ma * P->Ma * P->gamma * (P->gamma - 1.0));
                    } else if (bc == ORC_WALL) {
                        double rw = U[0 * nt + idb];
                        U[1 * nt + idb] = 0.0;
                        U[2 * nt + idb] = 0.0;
                        U[3 * nt + idb] = 0.0;
                        U[4 * nt + idb] = rw * P->T_wall /
                                          (P->Ma * P->Ma * P->gamma * (P->gamma - 1.0));
                    } else if (bc == ORC_DIRICHLET) {
                        double r, u[3], p;
                        face_prim(c, d, s, plane_index(c, d, ia, ib), &r, u, &p);
                        set_from_prim(P, U, idb, nt, r, u, p);
                    } else {
                        double r, u[3], T, u1[5];
                        prim_t w1;
                        face_prim(c, d, s, plane_index(c, d, ia, ib), &r, u, &T);
                        load_state(U, id1, nt, u1);
                        primitives(P, u1, &w1);
                        double rr = P->gamma * P->Ma * P->Ma * w1.p / T;
                        set_from_prim(P, U, idb, nt, rr, u, w1.p);
                    }
                }
        }
    }
}

/* ------------------------------------------------------------------------------------------
 * Characteristic WENO/TENO interface flux (Sec. 2.2 algorithm, steps 2(a)-(f)) at the
 * half-node between node m and node m + st along direction d.  Stencil nodes
 * k = m-2st .. m+3st.  Reading of step (d): alpha_j = max over those six nodes of
 * |lambda_j| evaluated from each node's own state and metric.
 * ------------------------------------------------------------------------------------------ */
/* Sensor label of one reconstruction (no counterpart in the paper): a TENO cut-off (some
 * omega_r = 0) that moves the reconstructed value away from the linear 5th-order value
 * (2, -13, 47, 27, -3)/60 by more than 5 % of the range of the five stencil values and by more
 * than `noise` (1e-5 of the interface's mean density times its largest acoustic speed), so that
 * cut-offs decided by rounding noise in near-uniform flow do not count. */
static int cut_matters(const double *f, double h, const double *w, double noise)
{
    if (w[0] != 0.0 && w[1] != 0.0 && w[2] != 0.0) return 0;
    double lin = (2.0 * f[0] - 13.0 * f[1] + 47.0 * f[2] + 27.0 * f[3] - 3.0 * f[4]) / 60.0;
    double lo = f[0], hi = f[0];
    for (int k = 1; k < 5; k++) {
        if (f[k] < lo) lo = f[k];
        if (f[k] > hi) hi = f[k];
    }
    double dev = fabs(h - lin);
    return dev > 0.05 * (hi - lo) && dev > noise;
}

static void interface_flux(const orc_ctx *c, int d, long m, double *Fh, double *margin, int *cut)
{
    const orc_params *P = &c->p;
    long nt = c->ntot, st = c->st[d];
    double Uk[6][NV], Fk[6][NV], lam[6][3];
    for (int s = 0; s < 6; s++) {
        long id = m + (long)(s - 2) * st;
        double S[3];
        for (int cc = 0; cc < 3; cc++) S[cc] = c->S[(d * 3 + cc) * nt + id];
        load_state(c->U, id, nt, Uk[s]);
        orc_flux(P->gamma, Uk[s], S, Fk[s]);
        prim_t w;
        primitives(P, Uk[s], &w);
        double un = S[0] * w.u[0] + S[1] * w.u[1] + S[2] * w.u[2];
        double sm = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
        lam[s][0] = un - sm * w.a;
        lam[s][1] = un;
        lam[s][2] = un + sm * w.a;
    }
    /* (a) Roe average between nodes m and m+1; interface normal = normalised mean metric */
    double u[3], H, a;
    roe_average(P, Uk[2], Uk[3], u, &H, &a);
    double nv[3], nm = 0.0;
    for (int cc = 0; cc < 3; cc++) {
        nv[cc] = 0.5 * (c->S[(d * 3 + cc) * nt + m] + c->S[(d * 3 + cc) * nt + m + st]);
        nm += nv[cc] * nv[cc];
    }
    nm = sqrt(nm);
    for (int cc = 0; cc < 3; cc++) nv[cc] /= nm;
    /* (b) eigensystem */
    double R[25], L[25];
    eigensystem(P->gamma, u, H, a, nv, R, L);
    double gh[NV];
    double mg = INFINITY;
    double acoustic = 0.0;
    for (int s = 0; s < 6; s++) {
        if (fabs(lam[s][0]) > acoustic) acoustic = fabs(lam[s][0]);
        if (fabs(lam[s][2]) > acoustic) acoustic = fabs(lam[s][2]);
    }
    const double floor_ = 1e-5 * 0.5 * (Uk[2][0] + Uk[3][0]) * acoustic;
    for (int j = 0; j < NV; j++) {
        int lj = (j == 0) ? 0 : (j == 4 ? 2 : 1);
        double alpha = 0.0;
        for (int s = 0; s < 6; s++) {
            double al = fabs(lam[s][lj]);
            if (al > alpha) alpha = al;
        }
        /* (c) project, (d) split */
        double gp[6], gm[6];
        for (int s = 0; s < 6; s++) {
            double V = 0.0, gg = 0.0;
            for (int v = 0; v < NV; v++) {
                V += L[j * 5 + v] * Uk[s][v];
                gg += L[j * 5 + v] * Fk[s][v];
            }
            gp[s] = 0.5 * (gg + alpha * V);
            gm[s] = 0.5 * (gg - alpha * V);
        }
        /* (e) reconstruct g+ from nodes m-2..m+2 and g- mirrored from m+3..m-1 (TENO6: g+ from
         * m-2..m+3 and g- mirrored from m+3..m-2) */
        double fm[6] = {gm[5], gm[4], gm[3], gm[2], gm[1], gm[0]};
        double m1 = INFINITY, m2 = INFINITY, w1[4], w2[4], hp, hm;
        if (P->scheme == ORC_TENO6) {
            hp = orc_recon6(gp, P->teno_ct, w1, &m1);
            hm = orc_recon6(fm, P->teno_ct, w2, &m2);
        } else {
            hp = orc_recon5(gp, P->scheme, P->teno_ct, w1, &m1);
            hm = orc_recon5(fm, P->scheme, P->teno_ct, w2, &m2);
        }
        if (cut && P->scheme == ORC_TENO5) {
            if (cut_matters(gp, hp, w1, floor_) || cut_matters(fm, hm, w2, floor_)) *cut = 1;
        }
        if (m1 < mg) mg = m1;
        if (m2 < mg) mg = m2;
        gh[j] = hp + hm;
    }
    /* (f) back to physical space */
    for (int v = 0; v < NV; v++) {
        double s = 0.0;
        for (int j = 0; j < NV; j++) s += R[v * 5 + j] * gh[j];
        Fh[v] = s;
    }
    if (margin && mg < *margin) *margin = mg;
}

/* exposed: the characteristic interface flux of a 1D stencil (six states, unit metric along
 * direction vector S for every node), for the unit pins */
void orc_char_flux_1d(double gamma, int scheme, double ct, const double *U6 /* [6][5] */,
                      const double *S, double *Fh)
{
    orc_ctx c;
    memset(&c, 0, sizeof c);
    c.p.gamma = gamma;
    c.p.Ma = 1.0;
    c.p.scheme = scheme;
    c.p.teno_ct = ct;
    c.ntot = 6;
    c.st[0] = 1;
    double Ubuf[30], Sbuf[54];
    for (int s = 0; s < 6; s++)
        for (int v = 0; v < 5; v++) Ubuf[v * 6 + s] = U6[s * 5 + v];
    for (int i = 0; i < 54; i++) Sbuf[i] = 0.0;
    for (int s = 0; s < 6; s++)
        for (int cc = 0; cc < 3; cc++) Sbuf[(0 * 3 + cc) * 6 + s] = S[cc];
    c.U = Ubuf;
    c.S = Sbuf;
    interface_flux(&c, 0, 2, Fh, NULL, NULL);
}

/* ------------------------------------------------------------------------------------------
 * Gated convective form (the learned-sensor extension; the paper has no sensor and runs one
 * scheme everywhere).  A cell gate g (one byte per interior node, an input) chooses, per
 * interface i+1/2 of direction d:
 *   - the characteristic WENO/TENO flux above (Sec. 2.2) when g_i or g_{i+1} is set, or when
 *     the interface's six-node stencil i-2..i+3 holds two adjacent nodes whose pressure ratio
 *     or density ratio (larger over smaller) exceeds `jump` (a strong jump);
 *   - otherwise the central 4th-order interface flux
 *         F^_{i+1/2} = [7 (F_i + F_{i+1}) - (F_{i-1} + F_{i+2})] / 12
 *     of each node's contravariant flux: the flux form of the first-derivative operator of
 *     Sec. 2.6 (Eq. 28 with the sign of the generated kernel of Sec. 4), since
 *     F^_{i+1/2} - F^_{i-1/2} = (F_{i-2} - 8 F_{i-1} + 8 F_{i+1} - F_{i+2}) / 12.
 * Reading for ghost nodes (non-periodic ends): the central flux reads the ghost values like the
 * characteristic one (no one-sided closure), and a ghost node takes the gate of the node its
 * value comes from -- the periodic image, else the nearest interior node of the line.
 * ------------------------------------------------------------------------------------------ */
static int gate_at(const orc_ctx *c, const int *ii)
{
    int x[3];
    for (int d = 0; d < 3; d++) {
        int n = c->p.n[d], y = ii[d];
        if (y < 0 || y >= n) {
            if (c->p.bc[d][0] == ORC_PERIODIC) y = wrapi(y, n);
            else y = y < 0 ? 0 : n - 1;
        }
        x[d] = y;
    }
    return c->gate[((long)x[2] * c->p.n[1] + x[1]) * c->p.n[0] + x[0]] != 0;
}

/* Strong-jump test of the interface between line index ii[d] and ii[d] + 1; *jm receives the
 * smallest |ratio / jump - 1| over the five adjacent pairs (how close the decision came). */
static int strong_jump(const orc_ctx *c, int d, const int *ii, double *jm)
{
    const orc_params *P = &c->p;
    double pr[6], rh[6];
    int jj[3] = {ii[0], ii[1], ii[2]};
    for (int s = 0; s < 6; s++) {
        jj[d] = ii[d] + s - 2;
        double u5[5];
        prim_t w;
        load_state(c->U, IDX(c, jj[0], jj[1], jj[2]), c->ntot, u5);
        primitives(P, u5, &w);
        pr[s] = w.p;
        rh[s] = w.rho;
    }
    int strong = 0;
    for (int s = 1; s < 6; s++) {
        double qa = pr[s] > pr[s - 1] ? pr[s] / pr[s - 1] : pr[s - 1] / pr[s];
        double qb = rh[s] > rh[s - 1] ? rh[s] / rh[s - 1] : rh[s - 1] / rh[s];
        if (qa > c->jump || qb > c->jump) strong = 1;
        double ma = fabs(qa / c->jump - 1.0), mb = fabs(qb / c->jump - 1.0);
        if (ma < *jm) *jm = ma;
        if (mb < *jm) *jm = mb;
    }
    return strong;
}

/* Interface flux of the gated form between line index ii[d] and ii[d] + 1 (node id m). */
static void gated_flux(const orc_ctx *c, int d, const int *ii, double *Fh, double *margin, double *jm)
{
    long st = c->st[d];
    long m = IDX(c, ii[0], ii[1], ii[2]);
    int ir[3] = {ii[0], ii[1], ii[2]};
    ir[d] = ii[d] + 1;
    int strong = strong_jump(c, d, ii, jm);
    if (strong || gate_at(c, ii) || gate_at(c, ir)) {
        interface_flux(c, d, m, Fh, margin, NULL);
        return;
    }
    double F[4][NV];
    for (int s = 0; s < 4; s++) {
        long id = m + (long)(s - 1) * st;
        double u5[5], S[3];
        load_state(c->U, id, c->ntot, u5);
        for (int cc = 0; cc < 3; cc++) S[cc] = c->S[(d * 3 + cc) * c->ntot + id];
        orc_flux(c->p.gamma, u5, S, F[s]);
    }
    for (int v = 0; v < NV; v++)
        Fh[v] = (7.0 * (F[1][v] + F[2][v]) - (F[0][v] + F[3][v])) / 12.0;
}

/* ------------------------------------------------------------------------------------------
 * Viscous and heat-flux terms (Eqs. 2-5, central 4th order of Sec. 2.6 with the metric chain
 * rule d/dx_j = sum_d (s_d/Jinv) S~_{d,j} d/dxi_d).  Reading: the viscous terms are written
 * in flux form, d/dxi_d( S~_d . tau ) etc., with the same first-derivative operator for the
 * velocity/temperature gradients and for the divergence (discretely conservative on periodic
 * grids).  Gradients are evaluated on interior nodes only (periodic indices wrap, non-periodic
 * ends use the one-sided closures), so no ghost values enter the viscous terms.
 * ------------------------------------------------------------------------------------------ */
typedef struct { const orc_ctx *c; int d, var, i, j, k; } prm_ud;

/* primitive value var (0,1,2: u,v,w; 3: T) at interior node along direction d, index s */
static double prim_fetch(const void *ud, int s)
{
    const prm_ud *a = (const prm_ud *)ud;
    const orc_ctx *c = a->c;
    int ii[3] = {a->i, a->j, a->k};
    ii[a->d] = (c->p.bc[a->d][0] == ORC_PERIODIC) ? wrapi(s, c->p.n[a->d]) : s;
    long id = IDX(c, ii[0], ii[1], ii[2]);
    double u5[5];
    load_state(c->U, id, c->ntot, u5);
    prim_t w;
    primitives(&c->p, u5, &w);
    return a->var < 3 ? w.u[a->var] : w.T;
}

/* viscous flux vector along computational direction d at interior node (i,j,k):
 * out[0..2] = S~_d . tau_{i.}, out[3] = S~_d . (u_i tau_{i.} - q) */
static void viscous_flux(const orc_ctx *c, int d, int i, int j, int k, double *out)
{
    const orc_params *P = &c->p;
    long nt = c->ntot;
    long id = IDX(c, i, j, k);
    int ii[3] = {i, j, k};
    /* computational derivatives of u, v, w, T */
    double dxi[3][4];
    for (int e = 0; e < 3; e++)
        for (int v = 0; v < 4; v++) {
            if (!c->active[e]) { dxi[e][v] = 0.0; continue; }
            prm_ud ud = {c, e, v, i, j, k};
            dxi[e][v] = deriv4(prim_fetch, &ud, ii[e], P->n[e], P->bc[e][0] == ORC_PERIODIC);
        }
    /* physical gradients grad[v][jc] = d(var v)/dx_jc */
    double grad[4][3];
    for (int v = 0; v < 4; v++)
        for (int jc = 0; jc < 3; jc++) {
            double s = 0.0;
            for (int e = 0; e < 3; e++)
                s += c->shat[e] * c->Jr[id] * c->S[(e * 3 + jc) * nt + id] * dxi[e][v];
            grad[v][jc] = s;
        }
    double u5[5];
    load_state(c->U, id, nt, u5);
    prim_t w;
    primitives(P, u5, &w);
    double mu = viscosity(P, w.T);
    double div = grad[0][0] + grad[1][1] + grad[2][2];
    double tau[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            tau[a][b] = (mu / P->Re) * (grad[a][b] + grad[b][a] - (a == b ? (2.0 / 3.0) * div : 0.0));
    double kq = -mu / ((P->gamma - 1.0) * P->Ma * P->Ma * P->Pr * P->Re);   /* Eq. 4 */
    double q[3];
    for (int b = 0; b < 3; b++) q[b] = kq * grad[3][b];
    double Sd[3];
    for (int cc = 0; cc < 3; cc++) Sd[cc] = c->S[(d * 3 + cc) * nt + id];
    for (int a = 0; a < 3; a++) out[a] = Sd[0] * tau[a][0] + Sd[1] * tau[a][1] + Sd[2] * tau[a][2];
    double e[3];
    for (int b = 0; b < 3; b++)
        e[b] = w.u[0] * tau[0][b] + w.u[1] * tau[1][b] + w.u[2] * tau[2][b] - q[b];
    out[3] = Sd[0] * e[0] + Sd[1] * e[1] + Sd[2] * e[2];
}

typedef struct { const orc_ctx *c; int d, comp, i, j, k; } vf_ud;
static double vflux_fetch(const void *ud, int s)
{
    const vf_ud *a = (const vf_ud *)ud;
    const orc_ctx *c = a->c;
    const orc_params *P = &c->p;
    int ii[3] = {a->i, a->j, a->k};
    ii[a->d] = (P->bc[a->d][0] == ORC_PERIODIC) ? wrapi(s, P->n[a->d]) : s;
    if (!c->vn_valid) {   /* sampled residuals: the flux of this node only */
        double out[4];
        viscous_flux(c, a->d, ii[0], ii[1], ii[2], out);
        return out[a->comp];
    }
    long N = (long)P->n[0] * P->n[1] * P->n[2];
    long o = ((long)ii[2] * P->n[1] + ii[1]) * P->n[0] + ii[0];
    return c->Vn[(long)(a->d * 4 + a->comp) * N + o];
}

/* viscous_flux of every interior node and direction into c->Vn (the values the divergence
 * differences read; computing them once per residual instead of once per use changes no bit) */
static void viscous_nodes(orc_ctx *c)
{
    const orc_params *P = &c->p;
    long N = (long)P->n[0] * P->n[1] * P->n[2];
    if (!c->Vn) c->Vn = (double *)calloc((size_t)12 * N, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (long line = 0; line < (long)P->n[1] * P->n[2]; line++) {
        int j = (int)(line % P->n[1]), k = (int)(line / P->n[1]);
        for (int i = 0; i < P->n[0]; i++) {
            long o = ((long)k * P->n[1] + j) * P->n[0] + i;
            for (int d = 0; d < 3; d++) {
                if (!c->active[d]) continue;
                double out[4];
                viscous_flux(c, d, i, j, k, out);
                for (int q = 0; q < 4; q++) c->Vn[(long)(d * 4 + q) * N + o] = out[q];
            }
        }
    }
    c->vn_valid = 1;
}

/* central convective flux component along direction d at node index s of the line */
typedef struct { const orc_ctx *c; int d, comp, i, j, k; } cf_ud;
static double cflux_fetch(const void *ud, int s)
{
    const cf_ud *a = (const cf_ud *)ud;
    const orc_ctx *c = a->c;
    int ii[3] = {a->i, a->j, a->k};
    ii[a->d] = (c->p.bc[a->d][0] == ORC_PERIODIC) ? wrapi(s, c->p.n[a->d]) : s;
    long id = IDX(c, ii[0], ii[1], ii[2]);
    double u5[5], S[3], F[5];
    load_state(c->U, id, c->ntot, u5);
    for (int cc = 0; cc < 3; cc++) S[cc] = c->S[(a->d * 3 + cc) * c->ntot + id];
    orc_flux(c->p.gamma, u5, S, F);
    return F[a->comp];
}

/* ------------------------------------------------------------------------------------------
 * Residual at one interior node: R = conv_x + conv_y + conv_z + viscous  (Eqs. 1-3, 10).
 * ------------------------------------------------------------------------------------------ */
static void residual_at(const orc_ctx *c, int i, int j, int k, double *R, double *margin, int *cut,
                        double *jm)
{
    const orc_params *P = &c->p;
    long id = IDX(c, i, j, k);
    int ii[3] = {i, j, k};
    for (int v = 0; v < NV; v++) R[v] = 0.0;
    for (int d = 0; d < 3; d++) {
        if (!c->active[d]) continue;
        double fac = c->shat[d] * c->Jr[id];
        if (c->gate && !cut && P->scheme != ORC_CENTRAL4) {
            /* gated form: interfaces i+1/2 and i-1/2 of this direction */
            double Fp[NV], Fm[NV], jdummy = INFINITY;
            int il[3] = {i, j, k};
            il[d] = ii[d] - 1;
            gated_flux(c, d, ii, Fp, margin, jm ? jm : &jdummy);
            gated_flux(c, d, il, Fm, margin, jm ? jm : &jdummy);
            for (int v = 0; v < NV; v++) R[v] -= fac * (Fp[v] - Fm[v]);
        } else if (P->scheme == ORC_CENTRAL4) {
            for (int v = 0; v < NV; v++) {
                cf_ud ud = {c, d, v, i, j, k};
                double D = deriv4(cflux_fetch, &ud, ii[d], P->n[d], P->bc[d][0] == ORC_PERIODIC);
                R[v] -= fac * D;
            }
        } else {
            double Fp[NV], Fm[NV];
            interface_flux(c, d, id, Fp, margin, cut);
            interface_flux(c, d, id - c->st[d], Fm, margin, cut);
            for (int v = 0; v < NV; v++) R[v] -= fac * (Fp[v] - Fm[v]);
        }
    }
    if (P->Re > 0.0) {
        for (int d = 0; d < 3; d++) {
            if (!c->active[d]) continue;
            double fac = c->shat[d] * c->Jr[id];
            for (int comp = 0; comp < 4; comp++) {
                vf_ud ud = {c, d, comp, i, j, k};
                double D = deriv4(vflux_fetch, &ud, ii[d], P->n[d], P->bc[d][0] == ORC_PERIODIC);
                R[1 + comp] += fac * D;
            }
        }
    }
    /* body force per unit volume and its work (the laminar channel's driving force) */
    if (P->force[0] != 0.0 || P->force[1] != 0.0 || P->force[2] != 0.0) {
        double u5[5];
        prim_t w;
        load_state(c->U, id, c->ntot, u5);
        primitives(P, u5, &w);
        for (int q = 0; q < 3; q++) {
            R[1 + q] += P->force[q];
            R[4] += P->force[q] * w.u[q];
        }
    }
}

/* ------------------------------------------------------------------------------------------
 * Public API
 * ------------------------------------------------------------------------------------------ */
void *orc_create(const orc_params *P)
{
    init_coeffs();
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    c->p = *P;
    for (int d = 0; d < 3; d++) {
        c->active[d] = P->n[d] > 1;
        c->g[d] = c->active[d] ? GH : 0;
        c->np[d] = P->n[d] + 2 * c->g[d];
    }
    c->st[0] = 1;
    c->st[1] = c->np[0];
    c->st[2] = (long)c->np[0] * c->np[1];
    c->ntot = (long)c->np[0] * c->np[1] * c->np[2];
    c->U = (double *)calloc((size_t)NV * c->ntot, sizeof(double));
    c->dU = (double *)calloc((size_t)NV * c->ntot, sizeof(double));
    c->Rw = (double *)calloc((size_t)NV * c->ntot, sizeof(double));
    c->S = (double *)calloc((size_t)9 * c->ntot, sizeof(double));
    c->Jr = (double *)calloc((size_t)c->ntot, sizeof(double));
    /* coordinates are only needed here: drop the caller's pointer afterwards */
    compute_metrics(c);
    c->p.coords = NULL;
    return c;
}

void orc_destroy(void *h)
{
    orc_ctx *c = (orc_ctx *)h;
    if (!c) return;
    free(c->U); free(c->dU); free(c->Rw); free(c->S); free(c->Jr); free(c->gate); free(c->Vn);
    free(c);
}

void orc_set_state(void *h, const double *U)
{
    orc_ctx *c = (orc_ctx *)h;
    const orc_params *P = &c->p;
    long plane = (long)P->n[0] * P->n[1] * P->n[2];
    for (int v = 0; v < NV; v++)
        for (int k = 0; k < P->n[2]; k++)
            for (int j = 0; j < P->n[1]; j++)
                for (int i = 0; i < P->n[0]; i++)
                    c->U[v * c->ntot + IDX(c, i, j, k)] =
                        U[v * plane + ((long)k * P->n[1] + j) * P->n[0] + i];
}

void orc_get_state(void *h, double *U)
{
    orc_ctx *c = (orc_ctx *)h;
    const orc_params *P = &c->p;
    long plane = (long)P->n[0] * P->n[1] * P->n[2];
    for (int v = 0; v < NV; v++)
        for (int k = 0; k < P->n[2]; k++)
            for (int j = 0; j < P->n[1]; j++)
                for (int i = 0; i < P->n[0]; i++)
                    U[v * plane + ((long)k * P->n[1] + j) * P->n[0] + i] =
                        c->U[v * c->ntot + IDX(c, i, j, k)];
}

/* Residual R(U) of the current state on every interior node, [5][nz][ny][nx].  When margin
 * is not NULL it receives, per node, the smallest TENO |chi - C_T|/C_T over the interfaces
 * that node's residual used; jmargin (gated form, may be NULL) the smallest |ratio/jump - 1|
 * of the strong-jump tests of those interfaces. */
void orc_residual_ex(void *h, double *R, double *margin, double *jmargin)
{
    orc_ctx *c = (orc_ctx *)h;
    const orc_params *P = &c->p;
    ghost_fill(c);
    if (P->Re > 0.0) viscous_nodes(c);
    long plane = (long)P->n[0] * P->n[1] * P->n[2];
#pragma omp parallel for schedule(dynamic, 1)
    for (long line = 0; line < (long)P->n[1] * P->n[2]; line++) {
        int j = (int)(line % P->n[1]), k = (int)(line / P->n[1]);
        for (int i = 0; i < P->n[0]; i++) {
            double r[NV], mg = INFINITY;
            double jm = INFINITY;
            residual_at(c, i, j, k, r, &mg, NULL, &jm);
            long o = ((long)k * P->n[1] + j) * P->n[0] + i;
            for (int v = 0; v < NV; v++) R[v * plane + o] = r[v];
            if (margin) margin[o] = mg;
            if (jmargin) jmargin[o] = jm;
        }
    }
}

void orc_residual(void *h, double *R, double *margin)
{
    orc_residual_ex(h, R, margin, NULL);
}

/* Install the cell gate of the gated convective form (gate: [nz][ny][nx] bytes, copied; NULL
 * returns to the plain scheme) and its strong-jump ratio.  Later residuals and steps use it. */
void orc_set_gate(void *h, const unsigned char *gate, double jump)
{
    orc_ctx *c = (orc_ctx *)h;
    free(c->gate);
    c->gate = NULL;
    c->jump = jump;
    if (!gate) return;
    long n = (long)c->p.n[0] * c->p.n[1] * c->p.n[2];
    c->gate = (unsigned char *)malloc((size_t)n);
    memcpy(c->gate, gate, (size_t)n);
}

/* Residual at listed interior nodes only: ijk[3*p + d], R[5*p + v]. */
void orc_residual_points(void *h, int npts, const int *ijk, double *R, double *margin)
{
    orc_ctx *c = (orc_ctx *)h;
    ghost_fill(c);
    c->vn_valid = 0;   /* a few points of a possibly large grid: no full-grid table */
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < npts; q++) {
        double r[NV], mg = INFINITY;
        residual_at(c, ijk[3 * q], ijk[3 * q + 1], ijk[3 * q + 2], r, &mg, NULL, NULL);
        for (int v = 0; v < NV; v++) R[5 * q + v] = r[v];
        if (margin) margin[q] = mg;
    }
}

/* Shock-sensor training labels (no counterpart in the paper; the learned sensor is an addition
 * to the method): label 1 where the TENO5 residual of the point used an interface (either side,
 * any characteristic field, any direction) at which a candidate stencil was cut (delta_r = 0,
 * Eq. 24) and the cut moved the reconstruction by more than 5 % of the stencil's range and
 * above the noise floor (see cut_matters), else 0.  labels: [nz][ny][nx] bytes. */
void orc_labels(void *h, unsigned char *labels)
{
    orc_ctx *c = (orc_ctx *)h;
    const orc_params *P = &c->p;
    ghost_fill(c);
    if (P->Re > 0.0) viscous_nodes(c);
#pragma omp parallel for schedule(dynamic, 1)
    for (long line = 0; line < (long)P->n[1] * P->n[2]; line++) {
        int j = (int)(line % P->n[1]), k = (int)(line / P->n[1]);
        for (int i = 0; i < P->n[0]; i++) {
            double r[NV], mg = INFINITY;
            int cut = 0;
            residual_at(c, i, j, k, r, &mg, &cut, NULL);
            labels[((long)k * P->n[1] + j) * P->n[0] + i] = (unsigned char)cut;
        }
    }
}

/* ------------------------------------------------------------------------------------------
 * Low-storage 2N Runge-Kutta (Eqs. 36-38): dU = A_i dU + dt R(U), U = U + B_i dU, dU^(0) = 0
 * each step.  The paper does not print A_i, B_i.  rk = 0: Williamson's 3-stage 3rd-order
 * scheme, A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15).  rk = 1: the 5-stage 4th-order 2N
 * scheme of Carpenter & Kennedy (1994, the paper's cited reference for its 4th-order
 * low-storage RK), their published rational coefficients.
 * rk = 2: the 3rd-order strong-stability-preserving scheme the paper takes from Gottlieb & Shu
 * (1998), whose coefficients it does not print either.  Reading: their optimal 3-stage SSP
 * scheme in its convex form -- each stage a convex combination of U^n and one forward-Euler
 * step of the previous stage,
 *     U1 = U^n + dt R(U^n),  U2 = 3/4 U^n + 1/4 (U1 + dt R(U1)),
 *     U^{n+1} = 1/3 U^n + 2/3 (U2 + dt R(U2)),
 * with the second register holding U^n (the same two arrays per equation as the 2N form).
 * ------------------------------------------------------------------------------------------ */
static const int RK_STAGES[3] = {3, 5, 3};
static const double SSP_ALPHA[3] = {0.0, 3.0 / 4.0, 1.0 / 3.0};   /* weight of U^n per stage */
static const double RK_A[2][5] = {{0.0, -5.0 / 9.0, -153.0 / 128.0, 0.0, 0.0},
                                  {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0, -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0}};
static const double RK_B[2][5] = {{1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0, 0.0, 0.0},
                                  {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0, 1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0, 2277821191437.0 / 14882151754819.0}};

/* one stage of the 2N register update on n values (shared by the solver and the pins) */
static void rk_stage_update(int rk, int stage, double dt, long n, double *U, double *dU, const double *R)
{
    if (rk == 2) {
        const double a = SSP_ALPHA[stage];
        for (long q = 0; q < n; q++) {
            if (stage == 0) dU[q] = U[q];
            U[q] = a * dU[q] + (1.0 - a) * (U[q] + dt * R[q]);
        }
        return;
    }
    for (long q = 0; q < n; q++) {
        dU[q] = RK_A[rk][stage] * dU[q] + dt * R[q];
        U[q] = U[q] + RK_B[rk][stage] * dU[q];
    }
}

/* Scalar test equation y' = lambda y, lambda = lr + i li, advanced nsteps with the same stage
 * update as the solver; y stored as the real 2-vector (Re y, Im y). */
void orc_rk_linear(int rk, double lr, double li, double dt, int nsteps, double *yr, double *yi)
{
    double U[2] = {*yr, *yi}, dU[2], R[2];
    for (int n = 0; n < nsteps; n++) {
        dU[0] = 0.0; dU[1] = 0.0;
        for (int s = 0; s < RK_STAGES[rk]; s++) {
            R[0] = lr * U[0] - li * U[1];
            R[1] = li * U[0] + lr * U[1];
            rk_stage_update(rk, s, dt, 2, U, dU, R);
        }
    }
    *yr = U[0];
    *yi = U[1];
}

void orc_rk3_linear(double lr, double li, double dt, int nsteps, double *yr, double *yi)
{
    orc_rk_linear(0, lr, li, dt, nsteps, yr, yi);
}

/* Advance nsteps RK steps (P->rk).  Returns 0, or -1 when a non-finite value appears. */
int orc_step(void *h, int nsteps)
{
    orc_ctx *c = (orc_ctx *)h;
    const orc_params *P = &c->p;
    long plane = (long)P->n[0] * P->n[1] * P->n[2];
    double *Ui = (double *)malloc(sizeof(double) * NV * plane);
    double *dUi = (double *)malloc(sizeof(double) * NV * plane);
    double *Ri = (double *)malloc(sizeof(double) * NV * plane);
    int rc = 0;
    for (int n = 0; n < nsteps && rc == 0; n++) {
        for (long q = 0; q < NV * plane; q++) dUi[q] = 0.0;
        const int rk = (P->rk == 1 || P->rk == 2) ? P->rk : 0;
        for (int s = 0; s < RK_STAGES[rk]; s++) {
            orc_residual(c, Ri, NULL);
            orc_get_state(c, Ui);
            rk_stage_update(rk, s, P->dt, NV * plane, Ui, dUi, Ri);
            orc_set_state(c, Ui);
            impose_boundary_nodes(c);
        }
        orc_get_state(c, Ui);
        for (long q = 0; q < NV * plane; q++)
            if (!isfinite(Ui[q])) { rc = -1; break; }
    }
    free(Ui); free(dUi); free(Ri);
    return rc;
}

/* metric export for tests: S~ [3][3][nz][ny][nx], 1/Jinv [nz][ny][nx], shat[3] */
void orc_get_metrics(void *h, double *S, double *Jr, double *shat)
{
    orc_ctx *c = (orc_ctx *)h;
    const orc_params *P = &c->p;
    long plane = (long)P->n[0] * P->n[1] * P->n[2];
    for (int k = 0; k < P->n[2]; k++)
        for (int j = 0; j < P->n[1]; j++)
            for (int i = 0; i < P->n[0]; i++) {
                long o = ((long)k * P->n[1] + j) * P->n[0] + i;
                long id = IDX(c, i, j, k);
                for (int q = 0; q < 9; q++) S[q * plane + o] = c->S[q * c->ntot + id];
                Jr[o] = c->Jr[id];
            }
    for (int d = 0; d < 3; d++) shat[d] = c->shat[d];
}

/* ghost-filled state export for the boundary-condition checks: [5][np2][np1][np0] */
void orc_get_ghosted(void *h, double *Ug, int *np)
{
    orc_ctx *c = (orc_ctx *)h;
    ghost_fill(c);
    memcpy(Ug, c->U, sizeof(double) * NV * c->ntot);
    for (int d = 0; d < 3; d++) np[d] = c->np[d];
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------------
 * Exact Riemann solver for the 1D Euler equations (Sod pin, Sec. 5.1).  Textbook construction:
 * Newton iteration on the star pressure p* for f_L(p) + f_R(p) + (u_R - u_L) = 0 with the
 * shock (Rankine-Hugoniot) and rarefaction (isentropic) branches, then sampling of the
 * self-similar solution at x/t.
 * ------------------------------------------------------------------------------------------ */
static void pfun(double g, double p, double rk, double pk, double ak, double *f, double *df)
{
    if (p > pk) {
        double A = 2.0 / ((g + 1.0) * rk), B = (g - 1.0) / (g + 1.0) * pk;
        double q = sqrt(A / (p + B));
        *f = (p - pk) * q;
        *df = q * (1.0 - 0.5 * (p - pk) / (B + p));
    } else {
        double pr = p / pk;
        *f = 2.0 * ak / (g - 1.0) * (pow(pr, (g - 1.0) / (2.0 * g)) - 1.0);
        *df = 1.0 / (rk * ak) * pow(pr, -(g + 1.0) / (2.0 * g));
    }
}

void orc_riemann_star(double g, const double *WL, const double *WR, double *pstar, double *ustar)
{
    double rl = WL[0], ul = WL[1], pl = WL[2], rr = WR[0], ur = WR[1], pr = WR[2];
    double al = sqrt(g * pl / rl), ar = sqrt(g * pr / rr);
    double p = 0.5 * (pl + pr);
    if (p < 1e-12) p = 1e-12;
    for (int it = 0; it < 200; it++) {
        double fl, dfl, fr, dfr;
        pfun(g, p, rl, pl, al, &fl, &dfl);
        pfun(g, p, rr, pr, ar, &fr, &dfr);
        double pn = p - (fl + fr + ur - ul) / (dfl + dfr);
        if (pn < 1e-14) pn = 1e-14;
        double ch = 2.0 * fabs(pn - p) / (pn + p);
        p = pn;
        if (ch < 1e-15) break;
    }
    double fl, dfl, fr, dfr;
    pfun(g, p, rl, pl, al, &fl, &dfl);
    pfun(g, p, rr, pr, ar, &fr, &dfr);
    *pstar = p;
    *ustar = 0.5 * (ul + ur) + 0.5 * (fr - fl);
}

/* sample the exact solution at positions x[q] (diaphragm x0, time t) -> rho, u, p */
void orc_riemann_sample(double g, const double *WL, const double *WR, double x0, double t,
                        int nq, const double *x, double *rho, double *u, double *p)
{
    double ps, us;
    orc_riemann_star(g, WL, WR, &ps, &us);
    double rl = WL[0], ul = WL[1], pl = WL[2], rr = WR[0], ur = WR[1], pr = WR[2];
    double al = sqrt(g * pl / rl), ar = sqrt(g * pr / rr);
    for (int q = 0; q < nq; q++) {
        double S = (x[q] - x0) / t;
        double r_, u_, p_;
        if (S <= us) {           /* left of contact */
            if (ps > pl) {       /* left shock */
                double sl = ul - al * sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g));
                if (S <= sl) { r_ = rl; u_ = ul; p_ = pl; }
                else {
                    r_ = rl * ((ps / pl + (g - 1.0) / (g + 1.0)) / ((g - 1.0) / (g + 1.0) * ps / pl + 1.0));
                    u_ = us; p_ = ps;
                }
            } else {             /* left rarefaction */
                double shl = ul - al;
                double asl = al * pow(ps / pl, (g - 1.0) / (2.0 * g));
                double stl = us - asl;
                if (S <= shl) { r_ = rl; u_ = ul; p_ = pl; }
                else if (S >= stl) { r_ = rl * pow(ps / pl, 1.0 / g); u_ = us; p_ = ps; }
                else {
                    double cf = 2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * al) * (ul - S);
                    r_ = rl * pow(cf, 2.0 / (g - 1.0));
                    u_ = 2.0 / (g + 1.0) * (al + (g - 1.0) / 2.0 * ul + S);
                    p_ = pl * pow(cf, 2.0 * g / (g - 1.0));
                }
            }
        } else {                 /* right of contact */
            if (ps > pr) {       /* right shock */
                double sr = ur + ar * sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g));
                if (S >= sr) { r_ = rr; u_ = ur; p_ = pr; }
                else {
                    r_ = rr * ((ps / pr + (g - 1.0) / (g + 1.0)) / ((g - 1.0) / (g + 1.0) * ps / pr + 1.0));
                    u_ = us; p_ = ps;
                }
            } else {             /* right rarefaction */
                double shr = ur + ar;
                double asr = ar * pow(ps / pr, (g - 1.0) / (2.0 * g));
                double str = us + asr;
                if (S >= shr) { r_ = rr; u_ = ur; p_ = pr; }
                else if (S <= str) { r_ = rr * pow(ps / pr, 1.0 / g); u_ = us; p_ = ps; }
                else {
                    double cf = 2.0 / (g + 1.0) - (g - 1.0) / ((g + 1.0) * ar) * (ur - S);
                    r_ = rr * pow(cf, 2.0 / (g - 1.0));
                    u_ = 2.0 / (g + 1.0) * (-ar + (g - 1.0) / 2.0 * ur + S);
                    p_ = pr * pow(cf, 2.0 * g / (g - 1.0));
                }
            }
        }
        rho[q] = r_; u[q] = u_; p[q] = p_;
    }
}
