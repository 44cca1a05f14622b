/*
 * Plain FP64 CPU oracle for the Wilson-clover SAP-FGMRES method of
 * arXiv:1502.04025 (Sec. 3.1, "Algorithm and implementation overview").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or constant with the CUDA library, and the CUDA library never calls
 * it.  It is written for a reader checking it against the definitions by eye:
 * no blocking, no fusion, no spin projection tricks, full 12x12 clover
 * matrices, single thread.
 *
 * The paper names the operator (Wilson-clover), the outer solver (flexible
 * GMRES), the preconditioner (multiplicative Schwarz / Schwarz alternating
 * procedure) and the domain solver (minimal residual with even-odd
 * preconditioning) but prints no formula for any of them; each function below
 * states the textbook definition it writes out and the reading taken where
 * the paper is silent.
 *
 * Conventions (readings of the paper, Sec. 3.1):
 *   site        n = x + Lx*(y + Ly*(z + Lz*t)), periodic in all directions
 *   links       U[n][mu][a][b] (complex), U_mu(n) joins n -> n+mu
 *   spinors     psi[n][s][c], 12 complex per site
 *   gammas      Euclidean Hermitian chiral basis:
 *               gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = x,y,z),
 *               gamma_t = [[0, 1], [1, 0]], gamma_5 = gamma_x gamma_y gamma_z gamma_t
 *   operator    D = A - kappa*H
 *               H psi(n) = sum_mu (1 - gamma_mu) U_mu(n) psi(n+mu)
 *                                + (1 + gamma_mu) U_mu(n-mu)^+ psi(n-mu)
 *               A(n) = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(n)
 *               sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu]
 *               F_{mu nu} = (Q - Q^+)/8 with the trace removed, Q the sum of
 *               the four plaquette leaves at n in the (mu,nu) plane
 *   domains     blocks of dom[0..3] sites; colour = (sum of block coords) mod 2;
 *               colour 0 (the block holding the origin) is swept first
 *   MR          on the Schur complement  Dhat = A_ee - D_eo A_oo^{-1} D_oe
 *               of the Dirichlet domain operator, zero start, no relaxation
 *   FGMRES(m)   right preconditioned, modified Gram-Schmidt, complex Givens,
 *               tolerance relative to |b|, restart from the true residual
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */

static long vol(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords(const int L[4], long n, int c[4])
{
    for (int mu = 0; mu < 4; mu++) {
        c[mu] = (int)(n % L[mu]);
        n /= L[mu];
    }
}

static long index_of(const int L[4], const int c[4])
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

/* neighbour of n one step in direction mu (step = +1 or -1), periodic */
static long neighbour(const int L[4], long n, int mu, int step)
{
    int c[4];
    coords(L, n, c);
    c[mu] = (c[mu] + step + L[mu]) % L[mu];
    return index_of(L, c);
}

/* ------------------------------------------------------------------ */
/* gamma matrices                                                      */
/* ------------------------------------------------------------------ */

static cplx gam[5][4][4];     /* gamma_x, gamma_y, gamma_z, gamma_t, gamma_5 */
static cplx sig[4][4][4][4];  /* sigma_{mu nu}[s][t] */
static int gam_ready = 0;

static void matmul4(cplx a[4][4], cplx b[4][4], cplx out[4][4])
{
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            cplx s = 0;
            for (int k = 0; k < 4; k++) s += a[i][k] * b[k][j];
            out[i][j] = s;
        }
}

static void init_gammas(void)
{
    if (gam_ready) return;
    /* Pauli matrices */
    cplx pauli[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(gam, 0, sizeof(gam));
    for (int k = 0; k < 3; k++)
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) {
                gam[k][i][2 + j] = -I * pauli[k][i][j]; /* upper-right block: -i sigma_k */
                gam[k][2 + i][j] = I * pauli[k][i][j];  /* lower-left block:   i sigma_k */
            }
    for (int i = 0; i < 2; i++) {
        gam[3][i][2 + i] = 1;
        gam[3][2 + i][i] = 1;
    }
    cplx t1[4][4], t2[4][4];
    matmul4(gam[0], gam[1], t1);
    matmul4(t1, gam[2], t2);
    matmul4(t2, gam[3], gam[4]);
    for (int mu = 0; mu < 4; mu++)
        for (int nu = 0; nu < 4; nu++) {
            cplx ab[4][4], ba[4][4];
            matmul4(gam[mu], gam[nu], ab);
            matmul4(gam[nu], gam[mu], ba);
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++) sig[mu][nu][i][j] = 0.5 * I * (ab[i][j] - ba[i][j]);
        }
    gam_ready = 1;
}

/* ------------------------------------------------------------------ */
/* 3x3 colour matrices                                                 */
/* ------------------------------------------------------------------ */

typedef struct { cplx m[3][3]; } su3;

static su3 link_at(const cplx *U, long n, int mu)
{
    su3 r;
    const cplx *p = U + ((size_t)n * 4 + mu) * 9;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) r.m[a][b] = p[a * 3 + b];
    return r;
}

static su3 mul3(su3 a, su3 b)
{
    su3 r;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx s = 0;
            for (int k = 0; k < 3; k++) s += a.m[i][k] * b.m[k][j];
            r.m[i][j] = s;
        }
    return r;
}

static su3 dag3(su3 a)
{
    su3 r;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) r.m[i][j] = conj(a.m[j][i]);
    return r;
}

/* ------------------------------------------------------------------ */
/* clover term                                                         */
/* ------------------------------------------------------------------ */

/*
 * F_{mu nu}(n): the four plaquette leaves at n, all oriented mu -> nu,
 *   Q = U_mu(n) U_nu(n+mu) U_mu(n+nu)^+ U_nu(n)^+
 *     + U_nu(n) U_mu(n+nu-mu)^+ U_nu(n-mu)^+ U_mu(n-mu)
 *     + U_mu(n-mu)^+ U_nu(n-mu-nu)^+ U_mu(n-mu-nu) U_nu(n-nu)
 *     + U_nu(n-nu)^+ U_mu(n-nu) U_nu(n-nu+mu) U_mu(n)^+
 *   F = (Q - Q^+)/8, then F -= tr(F)/3.
 */
static su3 field_strength(const int L[4], const cplx *U, long n, int mu, int nu)
{
    long n_pm = neighbour(L, n, mu, +1), n_mm = neighbour(L, n, mu, -1);
    long n_pn = neighbour(L, n, nu, +1), n_mn = neighbour(L, n, nu, -1);
    long n_mm_pn = neighbour(L, n_mm, nu, +1);
    long n_mm_mn = neighbour(L, n_mm, nu, -1);
    long n_pm_mn = neighbour(L, n_pm, nu, -1);

    su3 l1 = mul3(mul3(link_at(U, n, mu), link_at(U, n_pm, nu)),
                  mul3(dag3(link_at(U, n_pn, mu)), dag3(link_at(U, n, nu))));
    su3 l2 = mul3(mul3(link_at(U, n, nu), dag3(link_at(U, n_mm_pn, mu))),
                  mul3(dag3(link_at(U, n_mm, nu)), link_at(U, n_mm, mu)));
    su3 l3 = mul3(mul3(dag3(link_at(U, n_mm, mu)), dag3(link_at(U, n_mm_mn, nu))),
                  mul3(link_at(U, n_mm_mn, mu), link_at(U, n_mn, nu)));
    su3 l4 = mul3(mul3(dag3(link_at(U, n_mn, nu)), link_at(U, n_mn, mu)),
                  mul3(link_at(U, n_pm_mn, nu), dag3(link_at(U, n, mu))));
    su3 F;
    cplx tr = 0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            cplx q = l1.m[a][b] + l2.m[a][b] + l3.m[a][b] + l4.m[a][b];
            cplx qd = conj(l1.m[b][a] + l2.m[b][a] + l3.m[b][a] + l4.m[b][a]);
            F.m[a][b] = (q - qd) / 8.0;
        }
    for (int a = 0; a < 3; a++) tr += F.m[a][a];
    for (int a = 0; a < 3; a++) F.m[a][a] -= tr / 3.0;
    return F;
}

/* A(n) as a full 12x12 matrix, row/column index s*3 + a */
static void clover_site(const int L[4], const cplx *U, double csw, double kappa, long n, cplx *A)
{
    init_gammas();
    for (int i = 0; i < 144; i++) A[i] = 0;
    for (int i = 0; i < 12; i++) A[i * 12 + i] = 1;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++) {
            su3 F = field_strength(L, U, n, mu, nu);
            for (int s = 0; s < 4; s++)
                for (int t = 0; t < 4; t++)
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++)
                            A[(s * 3 + a) * 12 + t * 3 + b] += I * kappa * csw * sig[mu][nu][s][t] * F.m[a][b];
        }
}

/* Inverse of a 12x12 complex matrix by Gauss-Jordan elimination with partial
 * pivoting.  Returns 0, or -1 for a singular matrix. */
static int invert12(const cplx *A, cplx *Ainv)
{
    cplx M[12][24];
    for (int i = 0; i < 12; i++)
        for (int j = 0; j < 12; j++) {
            M[i][j] = A[i * 12 + j];
            M[i][12 + j] = (i == j) ? 1 : 0;
        }
    for (int col = 0; col < 12; col++) {
        int piv = col;
        for (int r = col + 1; r < 12; r++)
            if (cabs(M[r][col]) > cabs(M[piv][col])) piv = r;
        if (cabs(M[piv][col]) == 0.0) return -1;
        if (piv != col)
            for (int j = 0; j < 24; j++) {
                cplx tmp = M[col][j];
                M[col][j] = M[piv][j];
                M[piv][j] = tmp;
            }
        cplx d = M[col][col];
        for (int j = 0; j < 24; j++) M[col][j] /= d;
        for (int r = 0; r < 12; r++) {
            if (r == col) continue;
            cplx f = M[r][col];
            if (f == 0) continue;
            for (int j = 0; j < 24; j++) M[r][j] -= f * M[col][j];
        }
    }
    for (int i = 0; i < 12; i++)
        for (int j = 0; j < 12; j++) Ainv[i * 12 + j] = M[i][12 + j];
    return 0;
}

/* ------------------------------------------------------------------ */
/* Wilson hopping term                                                 */
/* ------------------------------------------------------------------ */

/* out += (1 + sgn*gamma_mu) applied to in (both 12-component spinors) */
static void add_projected(int mu, int sgn, const cplx *in, cplx *out)
{
    for (int s = 0; s < 4; s++)
        for (int a = 0; a < 3; a++) {
            cplx v = in[s * 3 + a];
            for (int t = 0; t < 4; t++) v += sgn * gam[mu][s][t] * in[t * 3 + a];
            out[s * 3 + a] += v;
        }
}

/* out[s][a] = sum_b u[a][b] in[s][b]  (dagger: sum_b conj(u[b][a]) in[s][b]) */
static void colour_mul(su3 u, int dagger, const cplx *in, cplx *out)
{
    for (int s = 0; s < 4; s++)
        for (int a = 0; a < 3; a++) {
            cplx v = 0;
            for (int b = 0; b < 3; b++) v += (dagger ? conj(u.m[b][a]) : u.m[a][b]) * in[s * 3 + b];
            out[s * 3 + a] = v;
        }
}

/*
 * H psi at site n, with optional restriction to the sites accepted by `keep`
 * (used for the Dirichlet domain operator): a hop from neighbour m is dropped
 * when keep != NULL and keep[m] == 0.
 */
static void hop_site(const int L[4], const cplx *U, const cplx *psi, long n, const unsigned char *keep, cplx out[12])
{
    init_gammas();
    cplx tmp[12];
    for (int i = 0; i < 12; i++) out[i] = 0;
    for (int mu = 0; mu < 4; mu++) {
        long nf = neighbour(L, n, mu, +1);
        if (!keep || keep[nf]) {
            colour_mul(link_at(U, n, mu), 0, psi + nf * 12, tmp);
            add_projected(mu, -1, tmp, out);
        }
        long nb = neighbour(L, n, mu, -1);
        if (!keep || keep[nb]) {
            colour_mul(link_at(U, nb, mu), 1, psi + nb * 12, tmp);
            add_projected(mu, +1, tmp, out);
        }
    }
}

static void mat12_mul(const cplx *A, const cplx *in, cplx *out)
{
    for (int i = 0; i < 12; i++) {
        cplx v = 0;
        for (int j = 0; j < 12; j++) v += A[i * 12 + j] * in[j];
        out[i] = v;
    }
}

/* (D psi)(n) = A(n) psi(n) - kappa (H psi)(n) */
static void dirac_site(const int L[4], const cplx *U, const cplx *A_n, double kappa, const cplx *psi, long n, cplx out[12])
{
    cplx h[12], a[12];
    hop_site(L, U, psi, n, NULL, h);
    mat12_mul(A_n, psi + n * 12, a);
    for (int i = 0; i < 12; i++) out[i] = a[i] - kappa * h[i];
}

/* ------------------------------------------------------------------ */
/* complex vector helpers                                              */
/* ------------------------------------------------------------------ */

static cplx cdot(const cplx *a, const cplx *b, long len)
{
    cplx s = 0;
    for (long i = 0; i < len; i++) s += conj(a[i]) * b[i];
    return s;
}

static double norm2(const cplx *a, long len)
{
    double s = 0;
    for (long i = 0; i < len; i++) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

/* ------------------------------------------------------------------ */
/* exported: gammas, clover, operator                                  */
/* ------------------------------------------------------------------ */

/* gamma matrix mu (0..3 = x,y,z,t; 4 = gamma_5) as 4x4 complex, row-major */
int ora_gamma(int mu, double *out)
{
    init_gammas();
    if (mu < 0 || mu > 4) return -1;
    cplx *o = (cplx *)out;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) o[i * 4 + j] = gam[mu][i][j];
    return 0;
}

/* F_{mu nu}(n) (traceless, anti-Hermitian) at one site, 3x3 complex */
int ora_field_strength(const int *L, const double *U, long n, int mu, int nu, double *out)
{
    su3 F = field_strength(L, (const cplx *)U, n, mu, nu);
    cplx *o = (cplx *)out;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) o[a * 3 + b] = F.m[a][b];
    return 0;
}

/* A(n) for every site: out has V*144 complex */
int ora_clover(const int *L, const double *U, double csw, double kappa, double *A)
{
    long V = vol(L);
    for (long n = 0; n < V; n++) clover_site(L, (const cplx *)U, csw, kappa, n, (cplx *)A + n * 144);
    return 0;
}

/* per-site 12x12 inverses */
int ora_invert_clover(const int *L, const double *A, double *Ainv)
{
    long V = vol(L);
    for (long n = 0; n < V; n++)
        if (invert12((const cplx *)A + n * 144, (cplx *)Ainv + n * 144)) return -1;
    return 0;
}

/* y = D x over the whole lattice, with precomputed A */
int ora_apply_D(const int *L, const double *U, const double *A, double kappa, const double *x, double *y)
{
    long V = vol(L);
    for (long n = 0; n < V; n++)
        dirac_site(L, (const cplx *)U, (const cplx *)A + n * 144, kappa, (const cplx *)x, n, (cplx *)y + n * 12);
    return 0;
}

/* y = H x over the whole lattice (hopping term only) */
int ora_apply_H(const int *L, const double *U, const double *x, double *y)
{
    long V = vol(L);
    for (long n = 0; n < V; n++) hop_site(L, (const cplx *)U, (const cplx *)x, n, NULL, (cplx *)y + n * 12);
    return 0;
}

/* (D x)(n) at a list of sites, building A(n) on the fly (no V-sized clover
 * array), for sampled checks on lattices too large for a full oracle apply. */
int ora_apply_D_sites(const int *L, const double *U, double csw, double kappa, const double *x,
                      long nsites, const long *sites, double *y)
{
    cplx A[144];
    long V = vol(L);
    for (long i = 0; i < nsites; i++) {
        if (sites[i] < 0 || sites[i] >= V) return -1;
        clover_site(L, (const cplx *)U, csw, kappa, sites[i], A);
        dirac_site(L, (const cplx *)U, A, kappa, (const cplx *)x, sites[i], (cplx *)y + i * 12);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* domains                                                             */
/* ------------------------------------------------------------------ */

typedef struct {
    int L[4], dom[4], nb[4];
    long V, Vd;
    int Nd;
} dd_t;

static int dd_init(dd_t *g, const int L[4], const int dom[4])
{
    g->V = vol(L);
    g->Vd = 1;
    g->Nd = 1;
    for (int mu = 0; mu < 4; mu++) {
        g->L[mu] = L[mu];
        g->dom[mu] = dom[mu];
        if (dom[mu] < 2 || dom[mu] % 2 || L[mu] % dom[mu]) return -1;
        g->nb[mu] = L[mu] / dom[mu];
        if (g->nb[mu] < 2 || g->nb[mu] % 2) return -1;
        g->Vd *= dom[mu];
        g->Nd *= g->nb[mu];
    }
    return 0;
}

static void block_coords(const dd_t *g, int d, int b[4])
{
    for (int mu = 0; mu < 4; mu++) {
        b[mu] = d % g->nb[mu];
        d /= g->nb[mu];
    }
}

static int block_colour(const dd_t *g, int d)
{
    int b[4];
    block_coords(g, d, b);
    return (b[0] + b[1] + b[2] + b[3]) & 1;
}

/* the global site indices of the domain with block index d, and their parities */
static void domain_sites(const dd_t *g, int d, long *sites, unsigned char *parity)
{
    int b[4], c[4];
    block_coords(g, d, b);
    long k = 0;
    for (int t = 0; t < g->dom[3]; t++)
        for (int z = 0; z < g->dom[2]; z++)
            for (int y = 0; y < g->dom[1]; y++)
                for (int x = 0; x < g->dom[0]; x++) {
                    c[0] = b[0] * g->dom[0] + x;
                    c[1] = b[1] * g->dom[1] + y;
                    c[2] = b[2] * g->dom[2] + z;
                    c[3] = b[3] * g->dom[3] + t;
                    sites[k] = index_of(g->L, c);
                    parity[k] = (unsigned char)((c[0] + c[1] + c[2] + c[3]) & 1);
                    k++;
                }
}

/*
 * Approximate solve of the Dirichlet domain system D_Lambda delta = rho_Lambda
 * by nmr minimal-residual steps on the even-odd Schur complement (Sec. 3.1,
 * footnote on the domain inversion):
 *   bhat_e = rho_e - D_eo A_oo^{-1} rho_o
 *   x_e = 0, r = bhat_e; repeat nmr:
 *       p = Dhat r,  Dhat = A_ee - D_eo A_oo^{-1} D_oe
 *       alpha = <p,r>/<p,p>;  x_e += alpha r;  r -= alpha p
 *   x_o = A_oo^{-1} (rho_o - D_oe x_e)
 * with D_eo = -kappa H_eo, D_oe = -kappa H_oe, hops leaving the domain dropped.
 * Full-lattice work arrays are used; only the domain's sites are touched.
 * delta receives the solution on the domain's sites.
 */
static void mr_domain(const dd_t *g, const cplx *U, const cplx *A, const cplx *Ainv, double kappa,
                      const long *sites, const unsigned char *par, const unsigned char *inside,
                      const cplx *rho, int nmr, cplx *x, cplx *r, cplx *p, cplx *t, cplx *delta)
{
    long Vd = g->Vd;
    cplx h[12];
    /* t_o = A_oo^{-1} rho_o */
    for (long k = 0; k < Vd; k++) {
        long n = sites[k];
        if (par[k] == 1) mat12_mul(Ainv + n * 144, rho + n * 12, t + n * 12);
        else for (int i = 0; i < 12; i++) t[n * 12 + i] = 0;
    }
    /* bhat_e = rho_e - D_eo t_o = rho_e + kappa H_eo t_o */
    for (long k = 0; k < Vd; k++) {
        long n = sites[k];
        if (par[k] != 0) continue;
        hop_site(g->L, U, t, n, inside, h);
        for (int i = 0; i < 12; i++) {
            r[n * 12 + i] = rho[n * 12 + i] + kappa * h[i];
            x[n * 12 + i] = 0;
        }
    }
    /* zero odd entries of r and x so that hops read only even data */
    for (long k = 0; k < Vd; k++) {
        long n = sites[k];
        if (par[k] == 1)
            for (int i = 0; i < 12; i++) r[n * 12 + i] = x[n * 12 + i] = 0;
    }
    for (int it = 0; it < nmr; it++) {
        /* t_o = A_oo^{-1} D_oe r = A_oo^{-1} (-kappa H_oe r) */
        for (long k = 0; k < Vd; k++) {
            long n = sites[k];
            if (par[k] != 1) continue;
            cplx u[12];
            hop_site(g->L, U, r, n, inside, h);
            for (int i = 0; i < 12; i++) u[i] = -kappa * h[i];
            mat12_mul(Ainv + n * 144, u, t + n * 12);
        }
        /* p_e = A_ee r_e - D_eo t_o = A_ee r_e + kappa H_eo t_o */
        cplx pr = 0;
        double pp = 0;
        for (long k = 0; k < Vd; k++) {
            long n = sites[k];
            if (par[k] != 0) continue;
            cplx a[12];
            hop_site(g->L, U, t, n, inside, h);
            mat12_mul(A + n * 144, r + n * 12, a);
            for (int i = 0; i < 12; i++) p[n * 12 + i] = a[i] + kappa * h[i];
            pr += cdot(p + n * 12, r + n * 12, 12);
            pp += norm2(p + n * 12, 12);
        }
        if (pp == 0.0) break;
        cplx alpha = pr / pp;
        for (long k = 0; k < Vd; k++) {
            long n = sites[k];
            if (par[k] != 0) continue;
            for (int i = 0; i < 12; i++) {
                x[n * 12 + i] += alpha * r[n * 12 + i];
                r[n * 12 + i] -= alpha * p[n * 12 + i];
            }
        }
    }
    /* x_o = A_oo^{-1} (rho_o - D_oe x_e) = A_oo^{-1} (rho_o + kappa H_oe x_e) */
    for (long k = 0; k < Vd; k++) {
        long n = sites[k];
        if (par[k] == 0) {
            for (int i = 0; i < 12; i++) delta[n * 12 + i] = x[n * 12 + i];
        } else {
            cplx u[12];
            hop_site(g->L, U, x, n, inside, h);
            for (int i = 0; i < 12; i++) u[i] = rho[n * 12 + i] + kappa * h[i];
            mat12_mul(Ainv + n * 144, u, delta + n * 12);
        }
    }
}

/*
 * Multiplicative Schwarz (Schwarz alternating procedure), Sec. 3.1:
 *   psi = 0, rho = eta
 *   for each half-sweep (colour 0, colour 1, colour 0, ...; n_half of them):
 *     for every domain Lambda of that colour:
 *       delta = MR approximation of D_Lambda^{-1} rho_Lambda
 *       psi  += delta (on Lambda)
 *       rho  -= D delta   (delta extended by zero outside Lambda), evaluated
 *                         on Lambda and on every neighbour of Lambda
 * n_half = 2 * (number of Schwarz cycles).  rho, if not NULL, receives the
 * maintained residual eta - D psi.
 */
int ora_sap(const int *L, const int *dom, const double *U_, const double *A_, const double *Ainv_,
            double kappa, const double *eta_, double *psi_, double *rho_out, int nmr, int n_half)
{
    dd_t g;
    if (dd_init(&g, L, dom)) return -1;
    const cplx *U = (const cplx *)U_, *A = (const cplx *)A_, *Ainv = (const cplx *)Ainv_;
    long V = g.V, Vd = g.Vd;
    size_t fsz = (size_t)V * 12 * sizeof(cplx);
    cplx *psi = (cplx *)psi_;
    cplx *rho = (cplx *)malloc(fsz), *x = (cplx *)calloc(V * 12, sizeof(cplx)),
         *r = (cplx *)calloc(V * 12, sizeof(cplx)), *p = (cplx *)calloc(V * 12, sizeof(cplx)),
         *t = (cplx *)calloc(V * 12, sizeof(cplx)), *delta = (cplx *)calloc(V * 12, sizeof(cplx));
    long *sites = (long *)malloc(Vd * sizeof(long));
    long *closure = (long *)malloc((size_t)9 * Vd * sizeof(long));
    unsigned char *par = (unsigned char *)malloc(Vd);
    unsigned char *inside = (unsigned char *)calloc(V, 1);
    unsigned char *mark = (unsigned char *)calloc(V, 1);
    if (!rho || !x || !r || !p || !t || !delta || !sites || !closure || !par || !inside || !mark) return -2;
    memcpy(rho, eta_, fsz);
    memset(psi, 0, fsz);

    for (int hs = 0; hs < n_half; hs++) {
        int colour = hs & 1;
        for (int d = 0; d < g.Nd; d++) {
            if (block_colour(&g, d) != colour) continue;
            domain_sites(&g, d, sites, par);
            for (long k = 0; k < Vd; k++) inside[sites[k]] = 1;
            mr_domain(&g, U, A, Ainv, kappa, sites, par, inside, rho, nmr, x, r, p, t, delta);
            /* psi += delta on Lambda */
            for (long k = 0; k < Vd; k++)
                for (int i = 0; i < 12; i++) psi[sites[k] * 12 + i] += delta[sites[k] * 12 + i];
            /* the closure: Lambda and every site one hop away from it */
            long nc = 0;
            for (long k = 0; k < Vd; k++) {
                long n = sites[k];
                if (!mark[n]) { mark[n] = 1; closure[nc++] = n; }
                for (int mu = 0; mu < 4; mu++)
                    for (int st = -1; st <= 1; st += 2) {
                        long m = neighbour(L, n, mu, st);
                        if (!mark[m]) { mark[m] = 1; closure[nc++] = m; }
                    }
            }
            /* rho -= D delta~, with delta~ = delta on Lambda and 0 elsewhere */
            for (long c = 0; c < nc; c++) {
                long n = closure[c];
                cplx dn[12], h[12], a[12];
                hop_site(L, U, delta, n, inside, h);
                if (inside[n]) mat12_mul(A + n * 144, delta + n * 12, a);
                else for (int i = 0; i < 12; i++) a[i] = 0;
                for (int i = 0; i < 12; i++) {
                    dn[i] = a[i] - kappa * h[i];
                    rho[n * 12 + i] -= dn[i];
                }
            }
            for (long c = 0; c < nc; c++) mark[closure[c]] = 0;
            for (long k = 0; k < Vd; k++) {
                inside[sites[k]] = 0;
                for (int i = 0; i < 12; i++) delta[sites[k] * 12 + i] = 0;
            }
        }
    }
    if (rho_out) memcpy(rho_out, rho, fsz);
    free(rho); free(x); free(r); free(p); free(t); free(delta);
    free(sites); free(closure); free(par); free(inside); free(mark);
    return 0;
}

/* ------------------------------------------------------------------ */
/* FGMRES(m)                                                           */
/* ------------------------------------------------------------------ */

typedef struct {
    const int *L, *dom;
    const cplx *U, *A, *Ainv;
    double kappa;
    int use_sap, nmr, ncy;
} op_t;

static void op_D(const op_t *o, const cplx *x, cplx *y)
{
    ora_apply_D(o->L, (const double *)o->U, (const double *)o->A, o->kappa, (const double *)x, (double *)y);
}

static int op_M(const op_t *o, const cplx *v, cplx *z, long len)
{
    if (!o->use_sap) {
        memcpy(z, v, len * sizeof(cplx));
        return 0;
    }
    return ora_sap(o->L, o->dom, (const double *)o->U, (const double *)o->A, (const double *)o->Ainv, o->kappa,
                   (const double *)v, (double *)z, NULL, o->nmr, 2 * o->ncy);
}

/*
 * Flexible GMRES(m) with right preconditioning (the outer solver of Sec. 3.1,
 * taken without the deflated restarts):
 *   x_0 = 0 (or the input x if x_in_is_guess), r = b - D x, beta = |r|, v_1 = r/beta
 *   for j = 1..m:
 *       z_j = M v_j;  w = D z_j
 *       for i = 1..j:  h_ij = <v_i, w>;  w -= h_ij v_i      (modified Gram-Schmidt)
 *       h_{j+1,j} = |w|;  v_{j+1} = w / h_{j+1,j}
 *       apply the previous Givens rotations to column j, form a new one that
 *       annihilates h_{j+1,j}; |g_{j+1}| is the residual-norm estimate
 *       stop the cycle when |g_{j+1}| <= tol |b| or h_{j+1,j} = 0
 *   y = R^{-1} g;  x += Z y;  true residual r = b - D x
 *   stop when |r| <= tol |b|, else restart (at most max_restarts restarts).
 * res_hist receives the estimated relative residual after every iteration,
 * followed at each restart boundary by the true relative residual.
 * Returns 0 when converged, 1 when not converged, negative on error.
 */
int ora_fgmres(const int *L, const int *dom, const double *U, const double *A, const double *Ainv, double kappa,
               const double *b_, double *x_, int x_in_is_guess, double tol, int m, int max_restarts, int use_sap,
               int nmr, int ncy, int *iters_out, int *restarts_out, double *true_rel_out, double *res_hist,
               int max_hist, int *n_hist)
{
    op_t o = {L, dom, (const cplx *)U, (const cplx *)A, (const cplx *)Ainv, kappa, use_sap, nmr, ncy};
    long len = vol(L) * 12;
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    cplx *r = (cplx *)malloc(len * sizeof(cplx)), *w = (cplx *)malloc(len * sizeof(cplx));
    cplx *Vb = (cplx *)malloc((size_t)(m + 1) * len * sizeof(cplx));
    cplx *Zb = (cplx *)malloc((size_t)m * len * sizeof(cplx));
    cplx *H = (cplx *)calloc((size_t)(m + 1) * m, sizeof(cplx));
    cplx *g = (cplx *)calloc(m + 1, sizeof(cplx)), *y = (cplx *)calloc(m, sizeof(cplx));
    double *cs = (double *)calloc(m, sizeof(double));
    cplx *sn = (cplx *)calloc(m, sizeof(cplx));
    if (!r || !w || !Vb || !Zb || !H || !g || !y || !cs || !sn) return -2;
    if (!x_in_is_guess) memset(x, 0, len * sizeof(cplx));
    int iters = 0, restarts = 0, nh = 0, status = 1;
    double bnorm = sqrt(norm2(b, len));
    double rel = 0;
    if (bnorm == 0.0) {
        memset(x, 0, len * sizeof(cplx));
        status = 0;
        goto done;
    }
    for (;;) {
        /* true residual */
        op_D(&o, x, r);
        for (long i = 0; i < len; i++) r[i] = b[i] - r[i];
        double beta = sqrt(norm2(r, len));
        rel = beta / bnorm;
        if (restarts > 0 && res_hist && nh < max_hist) res_hist[nh++] = rel;
        if (rel <= tol) { status = 0; break; }
        if (restarts > max_restarts) break;
        for (long i = 0; i < len; i++) Vb[i] = r[i] / beta;
        memset(H, 0, (size_t)(m + 1) * m * sizeof(cplx));
        memset(g, 0, (m + 1) * sizeof(cplx));
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m; j++) {
            cplx *vj = Vb + (size_t)j * len, *zj = Zb + (size_t)j * len;
            if (op_M(&o, vj, zj, len)) { status = -3; goto done; }
            op_D(&o, zj, w);
            for (int i = 0; i <= j; i++) {
                cplx *vi = Vb + (size_t)i * len;
                cplx hij = cdot(vi, w, len);
                H[i * m + j] = hij;
                for (long q = 0; q < len; q++) w[q] -= hij * vi[q];
            }
            double hn = sqrt(norm2(w, len));
            H[(j + 1) * m + j] = hn;
            if (hn != 0.0)
                for (long q = 0; q < len; q++) Vb[(size_t)(j + 1) * len + q] = w[q] / hn;
            /* previous rotations on column j */
            for (int i = 0; i < j; i++) {
                cplx a = H[i * m + j], c2 = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * c2;
                H[(i + 1) * m + j] = -conj(sn[i]) * a + cs[i] * c2;
            }
            /* new rotation: [c s; -conj(s) c] [a; b] = [rr; 0] */
            cplx a = H[j * m + j], bb = H[(j + 1) * m + j];
            double nu = sqrt(creal(a) * creal(a) + cimag(a) * cimag(a) + creal(bb) * creal(bb) + cimag(bb) * cimag(bb));
            if (cabs(a) == 0.0) {
                cs[j] = 0.0;
                sn[j] = 1.0;
                H[j * m + j] = bb;
            } else {
                cs[j] = cabs(a) / nu;
                sn[j] = (a / cabs(a)) * conj(bb) / nu;
                H[j * m + j] = (a / cabs(a)) * nu;
            }
            H[(j + 1) * m + j] = 0;
            g[j + 1] = -conj(sn[j]) * g[j];
            g[j] = cs[j] * g[j];
            iters++;
            k = j + 1;
            double est = cabs(g[j + 1]) / bnorm;
            if (res_hist && nh < max_hist) res_hist[nh++] = est;
            if (est <= tol || hn == 0.0) break;
        }
        /* y = R^{-1} g (back substitution), x += Z y */
        for (int i = k - 1; i >= 0; i--) {
            cplx s = g[i];
            for (int l = i + 1; l < k; l++) s -= H[i * m + l] * y[l];
            y[i] = s / H[i * m + i];
        }
        for (int i = 0; i < k; i++) {
            cplx *zi = Zb + (size_t)i * len;
            for (long q = 0; q < len; q++) x[q] += y[i] * zi[q];
        }
        restarts++;
    }
done:
    if (iters_out) *iters_out = iters;
    if (restarts_out) *restarts_out = restarts > 0 ? restarts - 1 : 0;
    if (true_rel_out) *true_rel_out = rel;
    if (n_hist) *n_hist = nh;
    free(r); free(w); free(Vb); free(Zb); free(H); free(g); free(y); free(cs); free(sn);
    return status;
}

/* number of domains of each colour, for the host-side checks of the layout */
int ora_domain_colour(const int *L, const int *dom, int d)
{
    dd_t g;
    if (dd_init(&g, L, dom)) return -1;
    if (d < 0 || d >= g.Nd) return -1;
    return block_colour(&g, d);
}
