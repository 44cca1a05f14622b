/*
 * su3gen.c -- the SU(3) step of the seeded gauge-field recipe (input
 * generation only; no part of the solver).
 *
 * For each link, given eight normal numbers h_a, form the Hermitian traceless
 * H = sum_a h_a lambda_a / 2 (lambda_a the Gell-Mann matrices), the
 * anti-Hermitian A = i eps H, and U = exp(A) by a Taylor series with scaling
 * and squaring: with s squarings chosen so that the Frobenius norm of
 * A / 2^s is at most 1/2, the series is summed to 18 terms (truncation below
 * 1e-21 relative) by Horner's rule, then squared s times.  U is then
 * re-unitarised (Gram-Schmidt on its rows) and its phase fixed so that
 * det U = 1.
 *
 * Built with -ffp-contract=off so that the results do not depend on whether
 * the compiler fuses multiply-adds (x86 and Arm give the same bits); links
 * are independent, so the OpenMP split does not change any result.
 */
#include <complex.h>
#include <math.h>

typedef double complex cplx;

static void gell_mann_h(const double *h, cplx H[3][3])
{
    const double r3 = 1.0 / sqrt(3.0);
    /* lambda_1..8 in the standard order; H = sum h_a lambda_a / 2 */
    H[0][0] = 0.5 * (h[2] + r3 * h[7]);
    H[1][1] = 0.5 * (-h[2] + r3 * h[7]);
    H[2][2] = 0.5 * (-2.0 * r3 * h[7]);
    H[0][1] = 0.5 * (h[0] - I * h[1]);
    H[1][0] = conj(H[0][1]);
    H[0][2] = 0.5 * (h[3] - I * h[4]);
    H[2][0] = conj(H[0][2]);
    H[1][2] = 0.5 * (h[5] - I * h[6]);
    H[2][1] = conj(H[1][2]);
}

static void mul3(cplx a[3][3], cplx b[3][3], cplx c[3][3])
{
    cplx t[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx s = 0;
            for (int k = 0; k < 3; k++) s += a[i][k] * b[k][j];
            t[i][j] = s;
        }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) c[i][j] = t[i][j];
}

static void expm3(cplx A[3][3], cplx E[3][3])
{
    double nrm = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) nrm += creal(A[i][j] * conj(A[i][j]));
    nrm = sqrt(nrm);
    int s = 0;
    while (nrm > 0.5 && s < 60) {
        nrm *= 0.5;
        s++;
    }
    const double f = ldexp(1.0, -s);
    cplx B[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) B[i][j] = A[i][j] * f;
    /* Horner: E = I + B/1 (I + B/2 (I + ... (I + B/18))) */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) E[i][j] = (i == j) ? 1.0 : 0.0;
    for (int k = 18; k >= 1; k--) {
        cplx T[3][3];
        mul3(B, E, T);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) E[i][j] = T[i][j] / (double)k + ((i == j) ? 1.0 : 0.0);
    }
    for (int q = 0; q < s; q++) mul3(E, E, E);
}

static void reunitarise(cplx U[3][3])
{
    for (int r = 0; r < 3; r++) {
        for (int p = 0; p < r; p++) {
            cplx d = 0;
            for (int c = 0; c < 3; c++) d += conj(U[p][c]) * U[r][c];
            for (int c = 0; c < 3; c++) U[r][c] -= d * U[p][c];
        }
        double n = 0;
        for (int c = 0; c < 3; c++) n += creal(U[r][c] * conj(U[r][c]));
        n = sqrt(n);
        for (int c = 0; c < 3; c++) U[r][c] /= n;
    }
    cplx det = U[0][0] * (U[1][1] * U[2][2] - U[1][2] * U[2][1]) - U[0][1] * (U[1][0] * U[2][2] - U[1][2] * U[2][0]) +
               U[0][2] * (U[1][0] * U[2][1] - U[1][1] * U[2][0]);
    cplx ph = cexp(-I * carg(det) / 3.0);
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) U[r][c] *= ph;
}

/* out[n][3][3] complex (interleaved re, im) = the SU(3) matrix of h[n][8] */
int su3gen_from_normals(long n, const double *h, double eps, double *out)
{
    long k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < n; k++) {
        cplx H[3][3], A[3][3], U[3][3];
        gell_mann_h(h + 8 * k, H);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) A[i][j] = I * eps * H[i][j];
        expm3(A, U);
        reunitarise(U);
        double *o = out + 18 * k;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                o[2 * (3 * i + j)] = creal(U[i][j]);
                o[2 * (3 * i + j) + 1] = cimag(U[i][j]);
            }
    }
    return 0;
}
