/*
 * mbs_oracle.c -- plain, slow, FP64 CPU oracle for the full-wave 1D
 * Maxwell-Bloch time step of Riesch & Jirauschek, "mbsolve: An open-source
 * solver tool for the Maxwell-Bloch equations" (CPC 2021).
 *
 * TEST INFRASTRUCTURE ONLY.  The parity tests, the smoke check and the CPU
 * baseline leg of the benchmark call it; the product (CUDA) path never links,
 * imports or runs it, and it shares no code with that path.
 *
 * Representation: the most literal one available.  Every medium cell carries
 * its full complex N x N density matrix; relaxation and H0 enter through the
 * complex N^2 x N^2 Liouvillian superoperator acting on row-major vec(rho).
 *
 * What it computes, per time step n (Sec. 3.2, Algorithm 1):
 *   1. H update on interior faces, Eq. (hupdate), plus total-field /
 *      scattered-field source corrections;
 *   2. every medium cell: rho^{n+1/2} = S_h U(E^n) S_h rho^{n-1/2}, the
 *      operator splitting of Sec. 2.2 read as a Strang splitting with
 *      S_h = expm(L0 dt/2) (H0 plus the dissipator D of Eq. (lindbladdiss))
 *      and U(E) rho = e^{+i mu E dt/hbar} rho e^{-i mu E dt/hbar}, the exact
 *      solution of the field term of Eq. (master1D), taken through the
 *      eigenbasis of mu;
 *   3. (d_t P)^{n+1/2} = n3D tr{mu L(rho^{n+1/2})} (Sec. 2, polarisation
 *      term); the field part of L drops out since tr(mu [mu, rho]) = 0;
 *   4. E update, Eq. (eupdate), source corrections, boundary condition;
 *   5. record E^{n+1} and rho^{n+1/2} at the probe cells.
 *
 * Readings taken where the paper is silent (each listed in the design notes):
 *   - cell-centred grid dz = L/Nx, cell m at (m + 1/2) dz, E and rho at the
 *     centre, H at the faces f = 0..Nx; face f uses the material of cell f;
 *   - dt = C dz / c_max, Nt = ceil(t_end / dt) (dt is not shrunk);
 *   - reflectivity 0 = first-order Mur, 1 = perfect electric conductor,
 *     0 < R < 1: with the amplitude reflection r = -sqrt(R) and M the Mur
 *     value, E_b^{n+1} = (1 + r) M^{n+1} - r E_b^{n-1} (E_b^{-1} = E_b^0):
 *     at Courant number 1 in vacuum the arriving wave is E_nb^n less the
 *     part already reflected, r E_b^{n-1} / (1 + r), and the cell holds
 *     (1 + r) times it, so r times the arriving wave goes back exactly;
 *   - soft sources are one-way total-field/scattered-field injections;
 *   - rho at n = -1/2 is the initial density matrix; E^0 = the initial field
 *     (zero unless given; Sec. 2.1 initial conditions), H^{-1/2} = 0.
 *
 * Matrix exponential: Pade [13/13] with scaling and squaring (Higham 2005,
 * "The scaling and squaring method for the matrix exponential revisited").
 * Eigen-decomposition of mu: cyclic complex Jacobi rotations (Golub & Van
 * Loan, Sec. 8.5).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* CODATA 2018 */
#define ORC_PLANCK 6.62607015e-34
#define ORC_PI 3.14159265358979323846
#define ORC_HBAR (ORC_PLANCK / (2.0 * ORC_PI))
#define ORC_EPS0 8.8541878128e-12
#define ORC_MU0 1.25663706212e-6

/* ---------------------------------------------------------------- inputs */
typedef struct {
    int n;                 /* number of levels N */
    double n3d;            /* density of quantum systems [m^-3] */
    const double *h0;      /* N*N complex (re, im interleaved), row-major [J] */
    const double *mu;      /* N*N complex [C m] */
    int n_ops;             /* explicit Lindblad operators */
    const double *rates;   /* [n_ops] */
    const double *ops;     /* [n_ops][N*N] complex */
    const double *scat;    /* N*N real or NULL: scat[i*N+j] = gamma_ij (j -> i) */
    const double *deph;    /* N(N-1)/2 or NULL: pure dephasing 12,13,23,14,... */
    const double *rho0;    /* N*N complex */
} orc_qm;

typedef struct { double eps_r, mu_r, sigma, overlap; int qm; } orc_mat;
typedef struct { int mat; double x0, x1; } orc_region;
typedef struct { int kind; int cell; double e0, tau, t0, omega, phase; int shape; } orc_source;
typedef struct { int cell; int q; int i, j; } orc_probe;

typedef struct {
    int n_qm; const orc_qm *qm;
    int n_mat; const orc_mat *mat;
    int n_reg; const orc_region *reg;
    double length; int nx;
    double refl_l, refl_r;
    const double *jitter;  /* nx*2 (density factor, H0 factor) or NULL */
    double courant; double t_end; long n_steps;
    int n_src; const orc_source *src;
    int n_probe; const orc_probe *probe;
    const double *e_init;  /* nx initial field values [V/m] or NULL (zero) */
} orc_problem;

enum { SRC_TFSF_RIGHT = 0, SRC_TFSF_LEFT = 1, SRC_HARD = 2 };
enum { Q_E = 0, Q_H = 1, Q_RHO_RE = 2, Q_RHO_IM = 3 };

/* ------------------------------------------------------- small algebra */
static void mat_mul(int n, const cplx *a, const cplx *b, cplx *c)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            cplx s = 0;
            for (int k = 0; k < n; k++) s += a[i * n + k] * b[k * n + j];
            c[i * n + j] = s;
        }
}

static void mat_vec(int n, const cplx *a, const cplx *x, cplx *y)
{
    for (int i = 0; i < n; i++) {
        cplx s = 0;
        for (int k = 0; k < n; k++) s += a[i * n + k] * x[k];
        y[i] = s;
    }
}

static void adjoint(int n, const cplx *a, cplx *b)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) b[j * n + i] = conj(a[i * n + j]);
}

static void load_c(int n, const double *src, cplx *dst)
{
    for (int k = 0; k < n * n; k++) dst[k] = src[2 * k] + I * src[2 * k + 1];
}

/* Solve A X = B (n x n, m right-hand sides) by Gaussian elimination with
 * partial pivoting; A and B are overwritten, X returned in B. */
static int lu_solve(int n, cplx *a, cplx *b)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        for (int i = k + 1; i < n; i++)
            if (cabs(a[i * n + k]) > cabs(a[p * n + k])) p = i;
        if (cabs(a[p * n + k]) == 0.0) return -1;
        if (p != k)
            for (int j = 0; j < n; j++) {
                cplx t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t;
                t = b[k * n + j]; b[k * n + j] = b[p * n + j]; b[p * n + j] = t;
            }
        for (int i = k + 1; i < n; i++) {
            cplx f = a[i * n + k] / a[k * n + k];
            for (int j = k; j < n; j++) a[i * n + j] -= f * a[k * n + j];
            for (int j = 0; j < n; j++) b[i * n + j] -= f * b[k * n + j];
        }
    }
    for (int k = n - 1; k >= 0; k--)
        for (int j = 0; j < n; j++) {
            cplx s = b[k * n + j];
            for (int i = k + 1; i < n; i++) s -= a[k * n + i] * b[i * n + j];
            b[k * n + j] = s / a[k * n + k];
        }
    return 0;
}

/* expm(A), Pade [13/13] with scaling and squaring (Higham 2005).  The Pade
 * numerator coefficients are b_j = (2m-j)! m! / ((2m)! j! (m-j)!), m = 13,
 * built by their ratio recurrence; the denominator is the numerator at -A.
 * A/2^s is scaled until its 1-norm is below theta_13 = 5.371920351148152,
 * the bound Higham derives for unit-roundoff backward error. */
int orc_expm(int n, const double *a_in, double *x_out)
{
    const int m = 13;
    const double theta13 = 5.371920351148152;
    size_t nn = (size_t)n * n;
    cplx *a = malloc(nn * sizeof(cplx)), *pw = malloc(nn * sizeof(cplx));
    cplx *p = malloc(nn * sizeof(cplx)), *q = malloc(nn * sizeof(cplx));
    cplx *t = malloc(nn * sizeof(cplx));
    load_c(n, a_in, a);
    double norm1 = 0.0;
    for (int j = 0; j < n; j++) {
        double s = 0.0;
        for (int i = 0; i < n; i++) s += cabs(a[i * n + j]);
        if (s > norm1) norm1 = s;
    }
    int s = 0;
    if (norm1 > theta13) s = (int)ceil(log2(norm1 / theta13));
    double scale = ldexp(1.0, -s);
    for (size_t k = 0; k < nn; k++) a[k] *= scale;

    double b[14];
    b[0] = 1.0;
    for (int j = 1; j <= m; j++) b[j] = b[j - 1] * (double)(m - j + 1) / ((double)(2 * m - j + 1) * j);
    /* p = sum b_j A^j, q = sum (-1)^j b_j A^j */
    for (size_t k = 0; k < nn; k++) { p[k] = 0; q[k] = 0; pw[k] = 0; }
    for (int i = 0; i < n; i++) pw[i * n + i] = 1.0;
    for (int j = 0; j <= m; j++) {
        double sg = (j % 2) ? -1.0 : 1.0;
        for (size_t k = 0; k < nn; k++) { p[k] += b[j] * pw[k]; q[k] += sg * b[j] * pw[k]; }
        if (j < m) { mat_mul(n, pw, a, t); memcpy(pw, t, nn * sizeof(cplx)); }
    }
    int rc = lu_solve(n, q, p);       /* p <- q^{-1} p */
    for (int k = 0; k < s; k++) { mat_mul(n, p, p, t); memcpy(p, t, nn * sizeof(cplx)); }
    for (size_t k = 0; k < nn; k++) { x_out[2 * k] = creal(p[k]); x_out[2 * k + 1] = cimag(p[k]); }
    free(a); free(pw); free(p); free(q); free(t);
    return rc;
}

/* Hermitian eigen-decomposition A = V diag(w) V^+ by cyclic complex Jacobi
 * rotations.  Each rotation first removes the phase of a_pq with
 * D = diag(1, e^{-i phi}) on the (p, q) plane, then applies the real
 * symmetric Jacobi rotation that annihilates the (now real) off-diagonal
 * pair; A <- W^+ A W, V <- V W with W = D G. */
int orc_eigh(int n, const double *a_in, double *w, double *v_out)
{
    cplx *a = malloc((size_t)n * n * sizeof(cplx)), *v = malloc((size_t)n * n * sizeof(cplx));
    cplx *W = malloc((size_t)n * n * sizeof(cplx)), *Wh = malloc((size_t)n * n * sizeof(cplx));
    cplx *t = malloc((size_t)n * n * sizeof(cplx));
    load_c(n, a_in, a);
    for (int i = 0; i < n * n; i++) v[i] = 0;
    for (int i = 0; i < n; i++) v[i * n + i] = 1.0;
    double fro = 0.0;
    for (int i = 0; i < n * n; i++) fro += creal(a[i] * conj(a[i]));
    fro = sqrt(fro);
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                if (i != j) off += creal(a[i * n + j] * conj(a[i * n + j]));
        if (sqrt(off) <= 1e-300 + 1e-17 * fro) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                double r = cabs(a[p * n + q]);
                if (r == 0.0) continue;
                cplx ph = a[p * n + q] / r;             /* e^{i phi} */
                double tau = (creal(a[q * n + q]) - creal(a[p * n + p])) / (2.0 * r);
                double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + tt * tt), s = tt * c;
                for (int i = 0; i < n * n; i++) W[i] = 0;
                for (int i = 0; i < n; i++) W[i * n + i] = 1.0;
                /* W = D G, D = diag(1, conj(ph)) on (p,q), G = [[c, s], [-s, c]] */
                W[p * n + p] = c;
                W[p * n + q] = s;
                W[q * n + p] = -s * conj(ph);
                W[q * n + q] = c * conj(ph);
                adjoint(n, W, Wh);
                mat_mul(n, Wh, a, t);
                mat_mul(n, t, W, a);
                mat_mul(n, v, W, t);
                memcpy(v, t, (size_t)n * n * sizeof(cplx));
                a[p * n + q] = 0; a[q * n + p] = 0;
            }
    }
    for (int i = 0; i < n; i++) w[i] = creal(a[i * n + i]);
    for (int i = 0; i < n * n; i++) { v_out[2 * i] = creal(v[i]); v_out[2 * i + 1] = cimag(v[i]); }
    free(a); free(v); free(W); free(Wh); free(t);
    return 0;
}

/* Liouvillian L0 of Eq. (master1D) without the field term, as a complex
 * N^2 x N^2 matrix acting on row-major vec(rho) (vec(A rho B) =
 * (A kron B^T) vec(rho)):
 *   -i/hbar (H0 kron 1 - 1 kron H0^T)
 *   + sum_k g_k [L_k kron conj(L_k) - 1/2 (L_k^+ L_k) kron 1 - 1/2 1 kron (L_k^+ L_k)^T]
 * plus, when the rate form is given, the population equation Eq.
 * (relax_pop) (d rho_ii = sum_j gamma_ij rho_jj - tau_i^{-1} rho_ii with
 * tau_j^{-1} = sum_{i != j} gamma_ij) and the coherence equation
 * d rho_ij = -[(tau_i^{-1} + tau_j^{-1})/2 + gamma_ij,p] rho_ij written out
 * element by element.  `h0_scale` multiplies H0 (per-cell jitter). */
int orc_liouvillian(const orc_qm *qm, double h0_scale, double *l_out)
{
    int n = qm->n, n2 = n * n;
    cplx *L = calloc((size_t)n2 * n2, sizeof(cplx));
    cplx *h = malloc(n2 * sizeof(cplx)), *op = malloc(n2 * sizeof(cplx));
    cplx *oph = malloc(n2 * sizeof(cplx)), *ll = malloc(n2 * sizeof(cplx));
    load_c(n, qm->h0, h);
#define LIDX(i, j, k, l) L[(size_t)((i) * n + (j)) * n2 + (k) * n + (l)]
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++)
                for (int l = 0; l < n; l++) {
                    cplx v = 0;
                    if (j == l) v += h[i * n + k];          /* H0 kron 1 */
                    if (i == k) v -= h[l * n + j];          /* 1 kron H0^T */
                    LIDX(i, j, k, l) += -I / ORC_HBAR * h0_scale * v;
                }
    for (int o = 0; o < qm->n_ops; o++) {
        double g = qm->rates[o];
        load_c(n, qm->ops + (size_t)2 * n2 * o, op);
        adjoint(n, op, oph);
        mat_mul(n, oph, op, ll);
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                for (int k = 0; k < n; k++)
                    for (int l = 0; l < n; l++) {
                        cplx v = op[i * n + k] * conj(op[j * n + l]);
                        if (j == l) v -= 0.5 * ll[i * n + k];
                        if (i == k) v -= 0.5 * ll[l * n + j];
                        LIDX(i, j, k, l) += g * v;
                    }
    }
    if (qm->scat) {
        double *inv_tau = calloc(n, sizeof(double));
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++)
                if (i != j) inv_tau[j] += qm->scat[i * n + j];
        for (int i = 0; i < n; i++) {
            for (int j = 0; j < n; j++)
                if (j != i) LIDX(i, i, j, j) += qm->scat[i * n + j];
            LIDX(i, i, i, i) -= inv_tau[i];
        }
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                if (i != j) LIDX(i, j, i, j) -= 0.5 * (inv_tau[i] + inv_tau[j]);
        free(inv_tau);
    }
    if (qm->deph) {
        int k = 0;
        for (int j = 1; j < n; j++)
            for (int i = 0; i < j; i++, k++) {
                LIDX(i, j, i, j) -= qm->deph[k];
                LIDX(j, i, j, i) -= qm->deph[k];
            }
    }
#undef LIDX
    for (int k = 0; k < n2 * n2; k++) { l_out[2 * k] = creal(L[k]); l_out[2 * k + 1] = cimag(L[k]); }
    free(L); free(h); free(op); free(oph); free(ll);
    return 0;
}

/* ------------------------------------------------- one cell's propagators */
typedef struct {
    int n;
    double n3d;
    cplx *Sh;      /* N^2 x N^2: expm(L0 dt/2) */
    cplx *L0;      /* N^2 x N^2 */
    cplx *mu;      /* N x N */
    double *lam;   /* eigenvalues of mu */
    cplx *V;       /* eigenvectors of mu (columns) */
} cellprop;

static int build_cellprop(const orc_qm *qm, double h0_scale, double dens_scale, double dt, cellprop *cp)
{
    int n = qm->n, n2 = n * n;
    cp->n = n;
    cp->n3d = qm->n3d * dens_scale;
    cp->Sh = malloc((size_t)n2 * n2 * sizeof(cplx));
    cp->L0 = malloc((size_t)n2 * n2 * sizeof(cplx));
    double *tmp = malloc((size_t)2 * n2 * n2 * sizeof(double));
    double *tmp2 = malloc((size_t)2 * n2 * n2 * sizeof(double));
    orc_liouvillian(qm, h0_scale, tmp);
    for (int k = 0; k < n2 * n2; k++) cp->L0[k] = tmp[2 * k] + I * tmp[2 * k + 1];
    for (int k = 0; k < 2 * n2 * n2; k++) tmp2[k] = tmp[k] * (0.5 * dt);
    int rc = orc_expm(n2, tmp2, tmp);
    for (int k = 0; k < n2 * n2; k++) cp->Sh[k] = tmp[2 * k] + I * tmp[2 * k + 1];
    free(tmp); free(tmp2);
    return rc;
}

static void free_cellprop(cellprop *cp)
{
    free(cp->Sh); free(cp->L0);
}

/* rho <- S_h U(E) S_h rho ; returns d_t P = n3D Re tr(mu L0 rho) of the result */
static double cell_step(const cellprop *cp, const cplx *mu, const double *lam, const cplx *V,
                        double e, double dt, cplx *rho, cplx *work)
{
    int n = cp->n, n2 = n * n;
    cplx *t1 = work, *t2 = work + n2, *U = work + 2 * n2, *Uh = work + 3 * n2, *d = work + 4 * n2;
    cplx ph[16];
    for (int k = 0; k < n; k++) ph[k] = cexp(I * lam[k] * e * dt / ORC_HBAR);
    mat_vec(n2, cp->Sh, rho, t1);                         /* S_h */
    for (int i = 0; i < n; i++)                           /* U = V diag(e^{i lam E dt/hbar}) V^+ */
        for (int j = 0; j < n; j++) {
            cplx s = 0;
            for (int k = 0; k < n; k++) s += V[i * n + k] * ph[k] * conj(V[j * n + k]);
            U[i * n + j] = s;
        }
    adjoint(n, U, Uh);
    mat_mul(n, U, t1, t2);                                /* U rho U^+ */
    mat_mul(n, t2, Uh, t1);
    mat_vec(n2, cp->Sh, t1, rho);                         /* S_h */
    mat_vec(n2, cp->L0, rho, d);                          /* L0 rho */
    cplx tr = 0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) tr += mu[j * n + i] * d[i * n + j];
    return cp->n3d * creal(tr);
}

/* Single driven cell: rho^{-1/2} = rho0, then for n = 0..nt-1 one split step
 * with the prescribed field e[n]; writes rho^{n+1/2} (N*N complex) for each n
 * to traj and d_t P to pdot (either may be NULL). */
int orc_cell_evolve(const orc_qm *qm, double dt, long nt, const double *e, double *traj, double *pdot)
{
    int n = qm->n, n2 = n * n;
    cellprop cp;
    if (build_cellprop(qm, 1.0, 1.0, dt, &cp)) return -1;
    cplx *mu = malloc(n2 * sizeof(cplx)), *V = malloc(n2 * sizeof(cplx));
    double *lam = malloc(n * sizeof(double)), *vtmp = malloc(2 * n2 * sizeof(double));
    load_c(n, qm->mu, mu);
    orc_eigh(n, qm->mu, lam, vtmp);
    load_c(n, vtmp, V);
    cplx *rho = malloc(n2 * sizeof(cplx)), *work = malloc(5 * n2 * sizeof(cplx));
    load_c(n, qm->rho0, rho);
    for (long s = 0; s < nt; s++) {
        double pd = cell_step(&cp, mu, lam, V, e[s], dt, rho, work);
        if (traj)
            for (int k = 0; k < n2; k++) {
                traj[(size_t)s * 2 * n2 + 2 * k] = creal(rho[k]);
                traj[(size_t)s * 2 * n2 + 2 * k + 1] = cimag(rho[k]);
            }
        if (pdot) pdot[s] = pd;
    }
    free_cellprop(&cp);
    free(mu); free(V); free(lam); free(vtmp); free(rho); free(work);
    return 0;
}

/* ---------------------------------------------------------- full sweep */
/* Sec. 3.1.2, classes sech_pulse (shape 0) and gaussian_pulse (shape 1):
 * e0 envelope((t - t0)/tau) sin(omega t + phase), the Gaussian envelope
 * read as exp(-x^2) (the paper names the class only) */
static double waveform(const orc_source *s, double t)
{
    const double x = (t - s->t0) / s->tau;
    const double env = s->shape == 1 ? exp(-x * x) : 1.0 / cosh(x);
    return s->e0 * env * sin(s->omega * t + s->phase);
}

/* smallest eigenvalue of a Hermitian N x N matrix (N <= 8) via orc_eigh */
static double min_eig(int n, const cplx *rho)
{
    double a[128], w[8], v[128];
    for (int k = 0; k < n * n; k++) { a[2 * k] = creal(rho[k]); a[2 * k + 1] = cimag(rho[k]); }
    orc_eigh(n, a, w, v);
    double m = w[0];
    for (int i = 1; i < n; i++) if (w[i] < m) m = w[i];
    return m;
}

/* Run the whole sweep.  rec: [n_probe][nt] doubles.  out_info[0] = dt,
 * out_info[1] = nt.  If check != 0, stats[0] = max |tr rho - 1|,
 * stats[1] = max |rho - rho^+|, stats[2] = min eigenvalue over every medium
 * cell and step (expensive).  Returns 0 or a negative error code. */
/* Material of each cell (the region containing the cell centre, first
 * match), dt = C dz / c_max over the cells' materials and Nt.  cm may be
 * NULL.  Returns -1 if a cell centre lies in no region. */
static int grid_setup(const orc_problem *pb, int *cm, double *dt_out, long *nt_out)
{
    int nx = pb->nx;
    double dz = pb->length / nx, cmax = 0.0;
    for (int m = 0; m < nx; m++) {
        double x = (m + 0.5) * dz;
        int k = -1;
        for (int r = 0; r < pb->n_reg; r++)
            if (x >= pb->reg[r].x0 && x < pb->reg[r].x1) { k = pb->reg[r].mat; break; }
        if (k < 0) return -1;
        if (cm) cm[m] = k;
        const orc_mat *mt = &pb->mat[k];
        double c = 1.0 / sqrt(ORC_EPS0 * mt->eps_r * ORC_MU0 * mt->mu_r);
        if (c > cmax) cmax = c;
    }
    *dt_out = pb->courant * dz / cmax;
    *nt_out = pb->n_steps > 0 ? pb->n_steps : (long)ceil(pb->t_end / *dt_out);
    return 0;
}

int orc_grid(const orc_problem *pb, double *out_info)
{
    double dt; long nt;
    if (grid_setup(pb, NULL, &dt, &nt)) return -1;
    out_info[0] = dt;
    out_info[1] = (double)nt;
    return 0;
}

int orc_run(const orc_problem *pb, int n_threads, int check, double *rec, double *out_info, double *stats)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    int nx = pb->nx;
    double dz = pb->length / nx;
    int *cm = malloc(nx * sizeof(int));
    double dt; long nt;
    if (grid_setup(pb, cm, &dt, &nt)) { free(cm); return -1; }
    out_info[0] = dt;
    out_info[1] = (double)nt;

    /* update coefficients, Eqs. (eupdate), (hupdate) */
    double *ca = malloc(nx * sizeof(double)), *cb = malloc(nx * sizeof(double));
    double *cg = malloc(nx * sizeof(double)), *ch = malloc((nx + 1) * sizeof(double));
    for (int m = 0; m < nx; m++) {
        const orc_mat *mt = &pb->mat[cm[m]];
        double eps = ORC_EPS0 * mt->eps_r, k = dt * mt->sigma / (2.0 * eps);
        ca[m] = (1.0 - k) / (1.0 + k);
        cb[m] = (dt / eps) / (1.0 + k);
        cg[m] = mt->overlap;
        ch[m] = dt / (dz * ORC_MU0 * mt->mu_r);
    }
    ch[nx] = 0.0;
    double dzinv = 1.0 / dz;

    /* per-cell quantum state */
    int nmax = 1;
    for (int q = 0; q < pb->n_qm; q++) if (pb->qm[q].n > nmax) nmax = pb->qm[q].n;
    cellprop *cp = calloc(nx, sizeof(cellprop));
    cplx **rho = calloc(nx, sizeof(cplx *));
    cplx **qmu = calloc(pb->n_qm, sizeof(cplx *)), **qV = calloc(pb->n_qm, sizeof(cplx *));
    double **qlam = calloc(pb->n_qm, sizeof(double *));
    for (int q = 0; q < pb->n_qm; q++) {
        int n = pb->qm[q].n;
        double *vt = malloc(2 * n * n * sizeof(double));
        qmu[q] = malloc(n * n * sizeof(cplx)); qV[q] = malloc(n * n * sizeof(cplx));
        qlam[q] = malloc(n * sizeof(double));
        load_c(n, pb->qm[q].mu, qmu[q]);
        orc_eigh(n, pb->qm[q].mu, qlam[q], vt);
        load_c(n, vt, qV[q]);
        free(vt);
    }
    /* cells without jitter share one propagator per quantum description */
    cellprop *shared = calloc(pb->n_qm, sizeof(cellprop));
    if (!pb->jitter)
        for (int q = 0; q < pb->n_qm; q++) build_cellprop(&pb->qm[q], 1.0, 1.0, dt, &shared[q]);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+:bad)
    for (int m = 0; m < nx; m++) {
        int q = pb->mat[cm[m]].qm;
        if (q < 0) continue;
        int n = pb->qm[q].n;
        if (pb->jitter) bad += build_cellprop(&pb->qm[q], pb->jitter[2 * m + 1], pb->jitter[2 * m], dt, &cp[m]) != 0;
        else cp[m] = shared[q];
        rho[m] = malloc(n * n * sizeof(cplx));
        load_c(n, pb->qm[q].rho0, rho[m]);
    }

    double *E = calloc(nx, sizeof(double)), *En = calloc(nx, sizeof(double));
    if (pb->e_init)
        for (int m = 0; m < nx; m++) E[m] = pb->e_init[m];
    double prev_l = E[0], prev_r = E[nx - 1];   /* E_b^{n-1} of the two ends */
    double *H = calloc(nx + 1, sizeof(double)), *pd = calloc(nx, sizeof(double));
    double st_tr = 0.0, st_herm = 0.0, st_min = 1e300;
    int m0 = 0, mN = nx - 1;
    double kl = 0.0, kr = 0.0;
    {
        const orc_mat *a = &pb->mat[cm[m0]], *b = &pb->mat[cm[mN]];
        double cl = 1.0 / sqrt(ORC_EPS0 * a->eps_r * ORC_MU0 * a->mu_r);
        double cr = 1.0 / sqrt(ORC_EPS0 * b->eps_r * ORC_MU0 * b->mu_r);
        kl = (cl * dt - dz) / (cl * dt + dz);
        kr = (cr * dt - dz) / (cr * dt + dz);
    }

    for (long s = 0; s < nt; s++) {
        double tn = s * dt;
        /* 1. H on interior faces */
#pragma omp parallel for schedule(static)
        for (int f = 1; f < nx; f++) H[f] += ch[f] * (E[f] - E[f - 1]);
        for (int k = 0; k < pb->n_src; k++) {
            const orc_source *sr = &pb->src[k];
            if (sr->kind == SRC_TFSF_RIGHT) H[sr->cell] -= ch[sr->cell] * waveform(sr, tn);
            else if (sr->kind == SRC_TFSF_LEFT) H[sr->cell + 1] += ch[sr->cell + 1] * waveform(sr, tn);
        }
        /* 2./3. density matrices and polarisation current */
        double l_tr = 0.0, l_herm = 0.0, l_min = 1e300;
#pragma omp parallel reduction(max:l_tr, l_herm) reduction(min:l_min)
        {
            cplx *work = malloc(5 * nmax * nmax * sizeof(cplx));
#pragma omp for schedule(static)
            for (int m = 0; m < nx; m++) {
                int q = pb->mat[cm[m]].qm;
                if (q < 0) { pd[m] = 0.0; continue; }
                pd[m] = cell_step(&cp[m], qmu[q], qlam[q], qV[q], E[m], dt, rho[m], work);
                if (check) {
                    int n = cp[m].n;
                    cplx tr = 0;
                    for (int i = 0; i < n; i++) tr += rho[m][i * n + i];
                    if (cabs(tr - 1.0) > l_tr) l_tr = cabs(tr - 1.0);
                    for (int i = 0; i < n; i++)
                        for (int j = 0; j < n; j++) {
                            double h = cabs(rho[m][i * n + j] - conj(rho[m][j * n + i]));
                            if (h > l_herm) l_herm = h;
                        }
                    double me = min_eig(n, rho[m]);
                    if (me < l_min) l_min = me;
                }
            }
            free(work);
        }
        if (check) {
            if (l_tr > st_tr) st_tr = l_tr;
            if (l_herm > st_herm) st_herm = l_herm;
            if (l_min < st_min) st_min = l_min;
        }
        /* 4. E update (H[0], H[nx] are boundary slots and stay zero) */
#pragma omp parallel for schedule(static)
        for (int m = 0; m < nx; m++)
            En[m] = ca[m] * E[m] - cb[m] * cg[m] * pd[m] + cb[m] * dzinv * (H[m + 1] - H[m]);
        for (int k = 0; k < pb->n_src; k++) {
            const orc_source *sr = &pb->src[k];
            int c = sr->cell;
            const orc_mat *mt = &pb->mat[cm[c]];
            double eta = sqrt(ORC_MU0 * mt->mu_r / (ORC_EPS0 * mt->eps_r));
            double cc = 1.0 / sqrt(ORC_EPS0 * mt->eps_r * ORC_MU0 * mt->mu_r);
            double th = tn + 0.5 * dt + 0.5 * dz / cc;
            if (sr->kind == SRC_TFSF_RIGHT || sr->kind == SRC_TFSF_LEFT)
                En[c] += cb[c] * dzinv * waveform(sr, th) / eta;
            else if (sr->kind == SRC_HARD)
                En[c] = waveform(sr, tn + dt);
        }
        /* boundaries: R = 0 first-order Mur, R = 1 perfect conductor,
           0 < R < 1 partially reflecting (see the header) */
        {
            const double cur_l = E[0], cur_r = E[nx - 1];
            if (pb->refl_l >= 1.0) En[0] = 0.0;
            else if (nx > 1) {
                En[0] = E[1] + kl * (En[1] - E[0]);
                if (pb->refl_l > 0.0) {
                    const double r = -sqrt(pb->refl_l);
                    En[0] = (1.0 + r) * En[0] - r * prev_l;
                }
            }
            if (pb->refl_r >= 1.0) En[nx - 1] = 0.0;
            else if (nx > 1) {
                En[nx - 1] = E[nx - 2] + kr * (En[nx - 2] - E[nx - 1]);
                if (pb->refl_r > 0.0) {
                    const double r = -sqrt(pb->refl_r);
                    En[nx - 1] = (1.0 + r) * En[nx - 1] - r * prev_r;
                }
            }
            prev_l = cur_l;
            prev_r = cur_r;
        }
        double *tsw = E; E = En; En = tsw;
        /* 5. records */
        for (int k = 0; k < pb->n_probe; k++) {
            const orc_probe *pr = &pb->probe[k];
            double v = 0.0;
            int c = pr->cell;
            if (pr->q == Q_E) v = E[c];
            else if (pr->q == Q_H) v = H[c];
            else {
                int q = pb->mat[cm[c]].qm;
                if (q >= 0) {
                    int n = pb->qm[q].n;
                    cplx r = rho[c][pr->i * n + pr->j];
                    v = (pr->q == Q_RHO_RE) ? creal(r) : cimag(r);
                }
            }
            rec[(size_t)k * nt + s] = v;
        }
    }
    if (stats) { stats[0] = st_tr; stats[1] = st_herm; stats[2] = st_min; }

    for (int m = 0; m < nx; m++) {
        if (rho[m]) free(rho[m]);
        if (pb->jitter && pb->mat[cm[m]].qm >= 0) free_cellprop(&cp[m]);
    }
    if (!pb->jitter) for (int q = 0; q < pb->n_qm; q++) free_cellprop(&shared[q]);
    for (int q = 0; q < pb->n_qm; q++) { free(qmu[q]); free(qV[q]); free(qlam[q]); }
    free(shared); free(qmu); free(qV); free(qlam); free(cp); free(rho);
    free(E); free(En); free(H); free(pd); free(ca); free(cb); free(cg); free(ch); free(cm);
    return bad ? -2 : 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
