/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the multimode Floquet hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file's shared library.  It shares no code, header,
 * table or helper with the CUDA path; the two only consume the same seeded inputs.
 *
 * Paper: G. A. Sinuco-Leon, "OPENMMF: a library for multimode driven quantum
 * systems" (arXiv 2005.03426).  Every function below names the passage it follows.
 *
 * Conventions (all complex arrays are interleaved (re, im) doubles = C99 double _Complex):
 *   D        number of levels, K number of modes, N[k] Fourier truncation of mode k
 *   M        = prod_k (2 N[k] + 1) Fourier blocks,  n = D * M
 *   flat index of state |i, nvec>:  i + D * sum_k (n_k + N[k]) * S_k,
 *            S_0 = 1, S_k = prod_{k'<k} (2 N[k'] + 1)   (mode 1 innermost, Appendix A)
 *   H0       D x D row-major, Hermitian
 *   V        all couplings concatenated: for mode k = 0..K-1, harmonic h = 1..nharm[k]:
 *            a D x D row-major block V^{k+1,h}
 *   HF, Z    n x n row-major
 *
 * Compile with -ffp-contract=off so that a*b+c is never fused: the Floquet diagonal
 * E_ii - sum_k n_k w_k is then rounded exactly as written (one rounding per operation,
 * accumulated over k ascending).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

/* ------------------------------------------------------------------ dimensions */
int64_t oracle_blocks(int K, const int *N)
{
    int64_t m = 1;
    for (int k = 0; k < K; ++k) m *= (int64_t)(2 * N[k] + 1);
    return m;
}

int64_t oracle_dim(int D, int K, const int *N) { return (int64_t)D * oracle_blocks(K, N); }

/* Fourier vector n_k of Fourier block b (b = sum_k (n_k + N_k) S_k). */
static void block_to_nvec(int64_t b, int K, const int *N, int *nv)
{
    for (int k = 0; k < K; ++k) {
        int64_t w = 2 * N[k] + 1;
        nv[k] = (int)(b % w) - N[k];
        b /= w;
    }
}

/* n.omega accumulated over k ascending, one rounding per product and per sum. */
static double ndotw(int K, const int *nv, const double *omega)
{
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        double p = (double)nv[k] * omega[k];
        s = s + p;
    }
    return s;
}

/* ------------------------------------------------------------------ S1: H_F
 * Eq. 6 with the index of the second coupling term read as U^{n-m} (the only form
 * consistent with substituting Eq. 5 into Eq. 2), laid out as in Appendix A:
 *   diagonal block n:                  E - (n.omega) I
 *   block (n, n + h e_l):              V^{l,h}            (upper side)
 *   block (n + h e_l, n):              V^{l,h} dagger     (lower side)
 * Fourier blocks with index outside [-N_l, N_l] are dropped (truncation, Sec. 2).
 */
int oracle_build_hf(int D, int K, const int *N, const double *omega, const int *nharm,
                    const cplx *H0, const cplx *V, cplx *HF)
{
    if (D < 1 || K < 0) return -1;
    int64_t M = oracle_blocks(K, N);
    int64_t n = (int64_t)D * M;
    memset(HF, 0, sizeof(cplx) * (size_t)(n * n));

    int64_t S[16];
    int64_t s = 1;
    for (int k = 0; k < K; ++k) { S[k] = s; s *= (2 * N[k] + 1); }

    int nv[16];
    for (int64_t b = 0; b < M; ++b) {
        block_to_nvec(b, K, N, nv);
        double sh = ndotw(K, nv, omega);
        /* diagonal block: E - (n.omega) on the diagonal */
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                cplx e = H0[i * D + j];
                if (i == j) e = (creal(e) - sh) + 0.0 * I;
                HF[(b * D + i) * n + (b * D + j)] = e;
            }
        /* coupling blocks */
        const cplx *Vk = V;
        for (int l = 0; l < K; ++l) {
            for (int h = 1; h <= nharm[l]; ++h) {
                const cplx *Vlh = Vk + (size_t)(h - 1) * D * D;
                if (nv[l] + h <= N[l]) {
                    int64_t bc = b + (int64_t)h * S[l];
                    for (int i = 0; i < D; ++i)
                        for (int j = 0; j < D; ++j) {
                            HF[(b * D + i) * n + (bc * D + j)] = Vlh[i * D + j];
                            HF[(bc * D + j) * n + (b * D + i)] = conj(Vlh[i * D + j]);
                        }
                }
            }
            Vk += (size_t)nharm[l] * D * D;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ S2: eigensolver
 * Full Hermitian eigendecomposition by the cyclic-by-row complex Jacobi method
 * (Forsythe & Henrici 1960).  The paper delegates this step to LAPACK (Sec. 3.2);
 * any exact diagonalisation computes the same eigenpairs.
 *
 * For the pivot (p, q) with a_pq = |a_pq| e^{i phi}, J = diag(1, e^{-i phi}) G with
 * G = [[c, s], [-s, c]] the real symmetric Schur rotation of
 * [[a_pp, |a_pq|], [|a_pq|, a_qq]] (Rutishauser's formulas, Golub & Van Loan Sec. 8.5):
 *   theta = (a_qq - a_pp) / (2 |a_pq|),  t = sign(theta) / (|theta| + sqrt(1 + theta^2)),
 *   c = 1 / sqrt(1 + t^2),  s = t c.
 * A <- J^H A J and Z <- Z J.  Sweeps stop when off(A) <= tol * ||A||_F.
 * Eigenvalues are returned ascending (ties by column index), Z[:, k] the k-th vector.
 * Returns 0, or 1 if max_sweeps was reached.
 */
int oracle_jacobi_eigh(int64_t n, cplx *A, double *w, cplx *Z, int max_sweeps, double tol,
                       int *sweeps_out)
{
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) Z[i * n + j] = (i == j) ? 1.0 : 0.0;

    double fro = 0.0;
    for (int64_t i = 0; i < n * n; ++i) fro += creal(A[i]) * creal(A[i]) + cimag(A[i]) * cimag(A[i]);
    fro = sqrt(fro);

    int status = 1, sweep;
    for (sweep = 0; sweep < max_sweeps; ++sweep) {
        double off = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j)
                if (i != j) off += creal(A[i * n + j]) * creal(A[i * n + j]) +
                                   cimag(A[i * n + j]) * cimag(A[i * n + j]);
        off = sqrt(off);
        if (off <= tol * fro) { status = 0; break; }

        for (int64_t p = 0; p < n - 1; ++p) {
            for (int64_t q = p + 1; q < n; ++q) {
                cplx apq = A[p * n + q];
                double r = cabs(apq);
                if (r == 0.0) continue;
                double app = creal(A[p * n + p]), aqq = creal(A[q * n + q]);
                cplx eph = apq / r;            /* e^{i phi} */
                double theta = (aqq - app) / (2.0 * r);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                /* J = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] */
                cplx jpp = c, jpq = s, jqp = -s * conj(eph), jqq = c * conj(eph);
                /* columns: A <- A J */
                for (int64_t k = 0; k < n; ++k) {
                    cplx akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = akp * jpp + akq * jqp;
                    A[k * n + q] = akp * jpq + akq * jqq;
                }
                /* rows: A <- J^H A */
                for (int64_t k = 0; k < n; ++k) {
                    cplx apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = conj(jpp) * apk + conj(jqp) * aqk;
                    A[q * n + k] = conj(jpq) * apk + conj(jqq) * aqk;
                }
                /* eigenvectors: Z <- Z J */
                for (int64_t k = 0; k < n; ++k) {
                    cplx zkp = Z[k * n + p], zkq = Z[k * n + q];
                    Z[k * n + p] = zkp * jpp + zkq * jqp;
                    Z[k * n + q] = zkp * jpq + zkq * jqq;
                }
                /* the pivot is annihilated in exact arithmetic; store it so */
                A[p * n + q] = 0.0;
                A[q * n + p] = 0.0;
                A[p * n + p] = creal(A[p * n + p]);
                A[q * n + q] = creal(A[q * n + q]);
            }
        }
    }
    if (sweeps_out) *sweeps_out = sweep;

    /* sort ascending, ties by index (insertion sort on an index permutation) */
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    cplx *Zs = (cplx *)malloc(sizeof(cplx) * (size_t)(n * n));
    for (int64_t i = 0; i < n; ++i) { perm[i] = i; d[i] = creal(A[i * n + i]); }
    for (int64_t i = 1; i < n; ++i) {
        int64_t pi = perm[i];
        int64_t j = i - 1;
        while (j >= 0 && (d[perm[j]] > d[pi])) { perm[j + 1] = perm[j]; --j; }
        perm[j + 1] = pi;
    }
    for (int64_t k = 0; k < n; ++k) {
        w[k] = d[perm[k]];
        for (int64_t i = 0; i < n; ++i) Zs[i * n + k] = Z[i * n + perm[k]];
    }
    memcpy(Z, Zs, sizeof(cplx) * (size_t)(n * n));
    free(perm); free(d); free(Zs);
    return status;
}

/* ------------------------------------------------------------------ S7: U(t, t0)
 * Eq. 3-5 (with Eq. 4 read as U_F(t') Ubar(t',t) U_F(t)^dagger), summed over all
 * Floquet copies of the truncated space:
 *   U(t, t0)_{j i} = sum_lambda sum_nvec e^{-i (nvec.omega) t} <j,nvec|lambda>
 *                    e^{-i E_lambda (t - t0)} <lambda|i,0>
 * Z is n x n row-major with columns = eigenvectors; U is nt x D x D with
 * U[k][j][i] = <j| U(t_k, t0) |i>.
 */
int oracle_time_evolution(int D, int K, const int *N, const double *omega, const double *E,
                          const cplx *Z, double t0, int nt, const double *t, cplx *U)
{
    int64_t M = oracle_blocks(K, N);
    int64_t n = (int64_t)D * M;
    int nv[16];
    int zero[16];
    for (int k = 0; k < K; ++k) zero[k] = N[k];
    int64_t b0 = 0, s = 1;
    for (int k = 0; k < K; ++k) { b0 += (int64_t)zero[k] * s; s *= (2 * N[k] + 1); }

    for (int it = 0; it < nt; ++it) {
        for (int j = 0; j < D; ++j)
            for (int i = 0; i < D; ++i) {
                cplx acc = 0.0;
                for (int64_t lam = 0; lam < n; ++lam) {
                    cplx ph = cexp(-I * E[lam] * (t[it] - t0));
                    cplx zi0 = conj(Z[(b0 * D + i) * n + lam]);
                    cplx inner = 0.0;
                    for (int64_t b = 0; b < M; ++b) {
                        block_to_nvec(b, K, N, nv);
                        double nw = ndotw(K, nv, omega);
                        inner += cexp(-I * nw * t[it]) * Z[(b * D + j) * n + lam];
                    }
                    acc += inner * ph * zi0;
                }
                U[((int64_t)it * D + j) * D + i] = acc;
            }
    }
    return 0;
}

/* ------------------------------------------------------------------ S8: Pbar
 * Time- and phase-averaged transition probability (the paper's transition-average
 * routine, Sec. 4.3; the formula is derived, the paper is silent on it): the average
 * of |U_{ji}(t, t0)|^2 over t and t - t0 keeps only pairs with equal (E, nvec), so
 *   Pbar_{i->j} = sum_nvec sum_C | sum_{lambda in C} <j,nvec|lambda> <lambda|i,0> |^2
 * where clusters C group ascending eigenvalues whose consecutive gaps are
 * < delta = cluster_rel * max|E| (single linkage).  E must be ascending.
 * P[i * D + j] = Pbar_{i->j}.
 */
int oracle_transition_avg(int D, int K, const int *N, const double *E, const cplx *Z,
                          double cluster_rel, double *P)
{
    int64_t M = oracle_blocks(K, N);
    int64_t n = (int64_t)D * M;
    int64_t b0 = 0, s = 1;
    for (int k = 0; k < K; ++k) { b0 += (int64_t)N[k] * s; s *= (2 * N[k] + 1); }
    double emax = 0.0;
    for (int64_t l = 0; l < n; ++l) if (fabs(E[l]) > emax) emax = fabs(E[l]);
    double delta = cluster_rel * emax;

    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double acc = 0.0;
            int64_t c0 = 0;
            while (c0 < n) {
                int64_t c1 = c0 + 1;
                while (c1 < n && (E[c1] - E[c1 - 1]) < delta) ++c1;
                for (int64_t b = 0; b < M; ++b) {
                    cplx amp = 0.0;
                    for (int64_t l = c0; l < c1; ++l)
                        amp += Z[(b * D + j) * n + l] * conj(Z[(b0 * D + i) * n + l]);
                    acc += creal(amp) * creal(amp) + cimag(amp) * cimag(amp);
                }
                c0 = c1;
            }
            P[i * D + j] = acc;
        }
    return 0;
}

/* ------------------------------------------------------------------ micromotion
 * Micromotion operator of Eq. 5 restricted to one Floquet zone:
 *   U_F(t)_{j, a} = sum_nvec e^{-i (nvec.omega) t} <j,nvec|lambda_a>
 * for the D zone representatives lambda_a given in ``reps`` (column indices of Z).
 * UF[k][j][a].
 */
int oracle_micromotion(int D, int K, const int *N, const double *omega, const cplx *Z,
                       const int64_t *reps, int nt, const double *t, cplx *UF)
{
    int64_t M = oracle_blocks(K, N);
    int64_t n = (int64_t)D * M;
    int nv[16];
    for (int it = 0; it < nt; ++it)
        for (int j = 0; j < D; ++j)
            for (int a = 0; a < D; ++a) {
                cplx acc = 0.0;
                for (int64_t b = 0; b < M; ++b) {
                    block_to_nvec(b, K, N, nv);
                    double nw = ndotw(K, nv, omega);
                    acc += cexp(-I * nw * t[it]) * Z[(b * D + j) * n + reps[a]];
                }
                UF[((int64_t)it * D + j) * D + a] = acc;
            }
    return 0;
}

/* ------------------------------------------------------------------ brute force
 * Time-domain integration of i dpsi/dt = H(t) psi with H(t) from Eq. 1
 *   H(t) = H0 + sum_{l,h} ( V^{l,h} e^{+i h w_l t} + V^{l,h}^dagger e^{-i h w_l t} )
 * by the classical fixed-step fourth-order Runge-Kutta method, for all D initial basis
 * states at once.  Returns U(t1, t0) (D x D row-major, U[j][i] = <j|U|i>).
 */
static void ham_at(int D, int K, const double *omega, const int *nharm, const cplx *H0,
                   const cplx *V, double t, cplx *H)
{
    for (int i = 0; i < D * D; ++i) H[i] = H0[i];
    const cplx *Vk = V;
    for (int l = 0; l < K; ++l) {
        for (int h = 1; h <= nharm[l]; ++h) {
            const cplx *Vlh = Vk + (size_t)(h - 1) * D * D;
            cplx e = cexp(I * (double)h * omega[l] * t);
            for (int i = 0; i < D; ++i)
                for (int j = 0; j < D; ++j)
                    H[i * D + j] += Vlh[i * D + j] * e + conj(Vlh[j * D + i]) * conj(e);
        }
        Vk += (size_t)nharm[l] * D * D;
    }
}

/* dU/dt = -i H(t) U */
static void rhs(int D, const cplx *H, const cplx *U, cplx *out)
{
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            cplx a = 0.0;
            for (int k = 0; k < D; ++k) a += H[i * D + k] * U[k * D + j];
            out[i * D + j] = -I * a;
        }
}

int oracle_rk4(int D, int K, const double *omega, const int *nharm, const cplx *H0,
               const cplx *V, double t0, double t1, int64_t steps, cplx *U)
{
    size_t sz = sizeof(cplx) * (size_t)(D * D);
    cplx *H = (cplx *)malloc(sz), *k1 = (cplx *)malloc(sz), *k2 = (cplx *)malloc(sz);
    cplx *k3 = (cplx *)malloc(sz), *k4 = (cplx *)malloc(sz), *Y = (cplx *)malloc(sz);
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) U[i * D + j] = (i == j) ? 1.0 : 0.0;
    double h = (t1 - t0) / (double)steps;
    for (int64_t s = 0; s < steps; ++s) {
        double t = t0 + h * (double)s;
        ham_at(D, K, omega, nharm, H0, V, t, H);
        rhs(D, H, U, k1);
        for (int i = 0; i < D * D; ++i) Y[i] = U[i] + 0.5 * h * k1[i];
        ham_at(D, K, omega, nharm, H0, V, t + 0.5 * h, H);
        rhs(D, H, Y, k2);
        for (int i = 0; i < D * D; ++i) Y[i] = U[i] + 0.5 * h * k2[i];
        rhs(D, H, Y, k3);
        for (int i = 0; i < D * D; ++i) Y[i] = U[i] + h * k3[i];
        ham_at(D, K, omega, nharm, H0, V, t + h, H);
        rhs(D, H, Y, k4);
        for (int i = 0; i < D * D; ++i) U[i] += (h / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    free(H); free(k1); free(k2); free(k3); free(k4); free(Y);
    return 0;
}
