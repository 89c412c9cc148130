/*
 * FP64 ORACLE -- test infrastructure only.  Nothing in the product library links or
 * calls this file; only the tests, the smoke check and the bench's CPU-baseline leg
 * load it (through oracle/__init__.py).
 *
 * Cyclic complex Jacobi eigenvalue iteration for a Hermitian matrix, used by the oracle
 * to obtain the singular values / right singular vectors of the steering matrix W
 * (SVD-PHAT Section 3, Eq. 10) from the Gram matrix of its smaller side.
 *
 * Method (Golub & Van Loan, "Matrix Computations", Section 8.5, extended to the
 * Hermitian case): for each off-diagonal pair (p,q) with b = A_pq = |b| e^{i phi},
 * the unitary U = diag(1, e^{-i phi}) * [[c, s], [-s, c]] acting on coordinates p,q
 * turns the 2x2 block real-symmetric and then annihilates it with the classical
 * symmetric Schur rotation (tau = (a_qq - a_pp) / (2|b|), t = sgn(tau)/(|tau| +
 * sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c).  A <- U^H A U, V <- V U.
 * Sweeps run row by row over all p < q until off(A) <= tol * ||A||_F.
 *
 * Storage: row-major n x n, real and imaginary parts in separate arrays.  The
 * eigenvectors come back transposed: row p of (Vr, Vi) is the eigenvector of A[p][p].
 * Compiled with -O2 -ffp-contract=off (no fused multiply-add contraction).
 */
#include <math.h>

int oracle_jacobi_herm(int n, double *Ar, double *Ai, double *Vr, double *Vi,
                       double tol, int max_sweeps)
{
    int i, j, k, p, q, sweep;
    double fro2 = 0.0;

    for (i = 0; i < n; ++i)
        for (j = 0; j < n; ++j) {
            Vr[i * n + j] = (i == j) ? 1.0 : 0.0;
            Vi[i * n + j] = 0.0;
            fro2 += Ar[i * n + j] * Ar[i * n + j] + Ai[i * n + j] * Ai[i * n + j];
        }
    for (i = 0; i < n; ++i) Ai[i * n + i] = 0.0;   /* Hermitian: real diagonal */

    for (sweep = 0; sweep <= max_sweeps; ++sweep) {
        double off2 = 0.0;
        for (i = 0; i < n; ++i)
            for (j = 0; j < n; ++j)
                if (i != j) off2 += Ar[i * n + j] * Ar[i * n + j] + Ai[i * n + j] * Ai[i * n + j];
        if (off2 <= tol * tol * fro2) return sweep;
        if (sweep == max_sweeps) break;

        for (p = 0; p < n - 1; ++p) {
            for (q = p + 1; q < n; ++q) {
                double br = Ar[p * n + q], bi = Ai[p * n + q];
                double babs = hypot(br, bi);
                double app, aqq, tau, t, c, s, er, ei;
                if (babs == 0.0) continue;
                /* e^{i phi} = b / |b| */
                er = br / babs;
                ei = bi / babs;
                app = Ar[p * n + p];
                aqq = Ar[q * n + q];
                tau = (aqq - app) / (2.0 * babs);
                t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                c = 1.0 / sqrt(1.0 + t * t);
                s = t * c;

                /* columns: A[:,p] <- c A[:,p] - s e^{-i phi} A[:,q]
                 *          A[:,q] <- s A[:,p] + c e^{-i phi} A[:,q]            */
                for (k = 0; k < n; ++k) {
                    double xr = Ar[k * n + p], xi = Ai[k * n + p];
                    double yr = Ar[k * n + q], yi = Ai[k * n + q];
                    /* e^{-i phi} y = (er - i ei)(yr + i yi) */
                    double zr = er * yr + ei * yi, zi = er * yi - ei * yr;
                    Ar[k * n + p] = c * xr - s * zr;
                    Ai[k * n + p] = c * xi - s * zi;
                    Ar[k * n + q] = s * xr + c * zr;
                    Ai[k * n + q] = s * xi + c * zi;
                }
                /* rows: A[p,:] <- c A[p,:] - s e^{i phi} A[q,:]
                 *       A[q,:] <- s A[p,:] + c e^{i phi} A[q,:]                 */
                for (k = 0; k < n; ++k) {
                    double xr = Ar[p * n + k], xi = Ai[p * n + k];
                    double yr = Ar[q * n + k], yi = Ai[q * n + k];
                    /* e^{i phi} y = (er + i ei)(yr + i yi) */
                    double zr = er * yr - ei * yi, zi = er * yi + ei * yr;
                    Ar[p * n + k] = c * xr - s * zr;
                    Ai[p * n + k] = c * xi - s * zi;
                    Ar[q * n + k] = s * xr + c * zr;
                    Ai[q * n + k] = s * xi + c * zi;
                }
                Ar[p * n + q] = Ai[p * n + q] = 0.0;
                Ar[q * n + p] = Ai[q * n + p] = 0.0;
                Ai[p * n + p] = Ai[q * n + q] = 0.0;

                /* eigenvectors: V <- V U (same column rule as A); V is held transposed
                 * (row p of Vt is column p of V) so that this update runs along rows */
                for (k = 0; k < n; ++k) {
                    double xr = Vr[p * n + k], xi = Vi[p * n + k];
                    double yr = Vr[q * n + k], yi = Vi[q * n + k];
                    double zr = er * yr + ei * yi, zi = er * yi - ei * yr;
                    Vr[p * n + k] = c * xr - s * zr;
                    Vi[p * n + k] = c * xi - s * zi;
                    Vr[q * n + k] = s * xr + c * zr;
                    Vi[q * n + k] = s * xi + c * zi;
                }
            }
        }
    }
    return -1;
}
