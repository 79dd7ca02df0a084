/*
 * cr_oracle.c -- CPU reference for cyclic reduction (CR) on Hermitian
 * positive definite block-tridiagonal systems: classic CR (reduce to the even
 * system, back-substitute the odd unknowns) and, at the end of the file, the
 * paper's Algorithm 1 (reduce to both halves and recurse on both).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle: it is used by
 * the tests, by the package's smoke check and by the CPU-baseline leg of
 * bench.py, and by nothing else.  It shares no code with the CUDA path.
 *
 * It is deliberately plain: std C99 complex doubles, naive loops, no BLAS, no
 * blocking or fusion.  The only parallelism is an OpenMP loop over the
 * independent blocks of one reduction level (the paper notes that the block
 * formulas are independent across j, Sec. 2 "Formulas for the Odd and Even
 * System").
 *
 * What it computes (the paper's notation, 1-based block indices):
 *   system (Sec. 1, eq. Axb): diagonal blocks A_j, sub-diagonal blocks B_j at
 *   block position (j+1, j), B_j^H at (j, j+1); unknowns x_j, rhs y_j.
 *   Boundary auxiliaries (Sec. 2): B_0 = B_N = 0, A_0 = A_{N+1} = I.
 *   One level (eq. even with eq. Formulas, products by the Cholesky rule of
 *   Sec. 4 "Numerical stability": G^H M^{-1} G = (L\G)^H (L\G)):
 *     for odd i:   A_i = L_i L_i^H,  P_i = L_i^{-1} B_{i-1},
 *                  Q_i = L_i^{-1} B_i^H,  r_i = L_i^{-1} y_i
 *     for j = 1..floor(N/2):
 *       V_j = A_{2j} - Q_{2j-1}^H Q_{2j-1} - P_{2j+1}^H P_{2j+1}
 *       F_j = -Q_{2j+1}^H P_{2j+1}                       (j < floor(N/2))
 *       v_j = y_{2j} - Q_{2j-1}^H r_{2j-1} - P_{2j+1}^H r_{2j+1}
 *   The even system (V, F, v) is again of the form eq. Axb and is reduced
 *   recursively until one block is left; that block is solved by Cholesky
 *   (Sec. 2 "Determination of Positive Definiteness").
 *   Classic CR solves only the even system; the odd unknowns follow from the
 *   odd block rows of eq. Axb (the first block row of the reordered matrix
 *   [D1 C^H; C D2] of Sec. 2):  x_i = L_i^{-H} (r_i - P_i x_{i-1} - Q_i x_{i+1}),
 *   with x_0 = x_{N+1} = 0.
 *
 * Readings where the paper is silent or garbled:
 *   - any N >= 1 (the paper assumes N even / a power of two): odd count
 *     ceil(N/2), even count floor(N/2); the boundary auxiliaries cover an odd
 *     last block.
 *   - only the lower triangle of each A_j is read; imaginary parts of its
 *     diagonal are ignored.
 *   - breakdown: a pivot d fails iff !(d > 0) (this also catches NaN).  The
 *     reported failure is the first level with a failure and, within it, the
 *     smallest 1-based local block index.
 *   - the reduced V_j is formed from its lower triangle and mirrored, so it
 *     is exactly Hermitian (Sec. 4 asks for "bit-wise hermitian" blocks; the
 *     printed product Z := G~^H G~^H reads as G~^H G~).
 *   - subtraction order in V_j and v_j: the left term, then the right term;
 *     inner sums in ascending index order.  Compiled with -ffp-contract=off.
 *
 * Layouts: A [N][m][m], B [N-1][m][m], y and x [N][m][k], all row-major
 * interleaved complex128.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zc;

typedef struct {
    int32_t status;     /* 0 = ok, 1 = not positive definite */
    int32_t level;      /* 0-based level of the first breakdown */
    int64_t block;      /* 1-based block index within that level */
    int64_t orig_block; /* 1-based index in the original system: block * 2^level */
} oracle_info;

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Cholesky A = L L^H of an m x m Hermitian matrix given by its lower
 * triangle.  L is lower triangular with a real positive diagonal; its strict
 * upper triangle is set to zero.  Returns 0, or r+1 when pivot r fails. */
static int chol_lower(int m, const zc *A, zc *L)
{
    memset(L, 0, sizeof(zc) * (size_t)m * m);
    for (int j = 0; j < m; ++j) {
        double d = creal(A[j * m + j]);
        for (int s = 0; s < j; ++s) {
            zc l = L[j * m + s];
            d -= creal(l) * creal(l) + cimag(l) * cimag(l);
        }
        if (!(d > 0.0)) return j + 1;
        double ljj = sqrt(d);
        L[j * m + j] = ljj;
        for (int i = j + 1; i < m; ++i) {
            zc v = A[i * m + j];
            for (int s = 0; s < j; ++s) v -= L[i * m + s] * conj(L[j * m + s]);
            L[i * m + j] = v / ljj;
        }
    }
    return 0;
}

/* X := L^{-1} X for X of size m x n (forward substitution, column by column). */
static void forward_subst(int m, int n, const zc *L, zc *X)
{
    for (int c = 0; c < n; ++c)
        for (int i = 0; i < m; ++i) {
            zc v = X[i * n + c];
            for (int s = 0; s < i; ++s) v -= L[i * m + s] * X[s * n + c];
            X[i * n + c] = v / creal(L[i * m + i]);
        }
}

/* X := L^{-H} X for X of size m x n (backward substitution). */
static void backward_subst(int m, int n, const zc *L, zc *X)
{
    for (int c = 0; c < n; ++c)
        for (int i = m - 1; i >= 0; --i) {
            zc v = X[i * n + c];
            for (int s = i + 1; s < m; ++s) v -= conj(L[s * m + i]) * X[s * n + c];
            X[i * n + c] = v / creal(L[i * m + i]);
        }
}

/* out (n1 x n2) := G1^H G2 with G1 (m x n1), G2 (m x n2). */
static void ctrans_prod(int m, int n1, int n2, const zc *G1, const zc *G2, zc *out)
{
    for (int a = 0; a < n1; ++a)
        for (int b = 0; b < n2; ++b) {
            zc v = 0;
            for (int s = 0; s < m; ++s) v += conj(G1[s * n1 + a]) * G2[s * n2 + b];
            out[a * n2 + b] = v;
        }
}

/* out (m x m) := G^H G computed on the lower triangle and mirrored, so that
 * the result is exactly Hermitian with a real diagonal. */
static void herk_lower(int m, const zc *G, zc *out)
{
    for (int a = 0; a < m; ++a) {
        double d = 0;
        for (int s = 0; s < m; ++s) {
            zc g = G[s * m + a];
            d += creal(g) * creal(g) + cimag(g) * cimag(g);
        }
        out[a * m + a] = d;
        for (int b = 0; b < a; ++b) {
            zc v = 0;
            for (int s = 0; s < m; ++s) v += conj(G[s * m + a]) * G[s * m + b];
            out[a * m + b] = v;
            out[b * m + a] = conj(v);
        }
    }
}

/* out (m x n) := X1 - X2 elementwise. */
static void sub_into(int64_t len, zc *X1, const zc *X2)
{
    for (int64_t e = 0; e < len; ++e) X1[e] -= X2[e];
}

/*
 * One reduction level of classic CR on a level system with Nl blocks.
 * Inputs A [Nl][m][m], B [Nl-1][m][m] (may be NULL when Nl == 1), y [Nl][m][k]
 * (may be NULL, then k is ignored and r, yn are not written).
 * Outputs, for the no = ceil(Nl/2) odd blocks t = 0..no-1 (1-based i = 2t+1):
 *   L [no][m][m], P [no][m][m], Q [no][m][m], r [no][m][k];
 * and the even system with ne = floor(Nl/2) blocks:
 *   An [ne][m][m], Bn [ne-1][m][m], yn [ne][m][k].
 * Returns 0 or the smallest failing 1-based local block index.
 */
int64_t oracle_cr_level(int64_t Nl, int m, int k, const zc *A, const zc *B, const zc *y,
                        zc *L, zc *P, zc *Q, zc *r, zc *An, zc *Bn, zc *yn)
{
    const int64_t no = (Nl + 1) / 2, ne = Nl / 2;
    const size_t mm = (size_t)m * m, mk = (size_t)m * k;
    int64_t fail = 0;

    /* odd blocks: Cholesky, P, Q, r */
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < no; ++t) {
        const int64_t c = 2 * t; /* 0-based position of odd block i = 2t+1 */
        int f = chol_lower(m, A + c * mm, L + t * mm);
        if (f) {
#pragma omp critical
            { if (fail == 0 || c + 1 < fail) fail = c + 1; }
            continue;
        }
        zc *Pt = P + t * mm, *Qt = Q + t * mm;
        /* P_i = L_i^{-1} B_{i-1}; B_{i-1} is B[c-1] (0-based), zero for i = 1 */
        if (c >= 1) memcpy(Pt, B + (c - 1) * mm, sizeof(zc) * mm);
        else memset(Pt, 0, sizeof(zc) * mm);
        /* Q_i = L_i^{-1} B_i^H; B_i is B[c] (0-based), zero for i = Nl */
        if (c + 1 <= Nl - 1) {
            const zc *Bc = B + c * mm;
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) Qt[a * m + b] = conj(Bc[b * m + a]);
        } else {
            memset(Qt, 0, sizeof(zc) * mm);
        }
        forward_subst(m, m, L + t * mm, Pt);
        forward_subst(m, m, L + t * mm, Qt);
        if (y) {
            memcpy(r + t * mk, y + c * mk, sizeof(zc) * mk);
            forward_subst(m, k, L + t * mm, r + t * mk);
        }
    }
    if (fail) return fail;

    /* even blocks j = 1..ne at 0-based position 2j-1; left odd t = j-1, right odd t = j */
#pragma omp parallel for schedule(static)
    for (int64_t j = 1; j <= ne; ++j) {
        zc *tmp = (zc *)malloc(sizeof(zc) * mm);
        zc *tmpk = (zc *)malloc(sizeof(zc) * (mk > 0 ? mk : 1));
        const int64_t pos = 2 * j - 1, tl = j - 1, tr = j;
        const int has_right = (2 * j + 1 <= Nl);
        zc *V = An + (j - 1) * mm;
        /* V_j: lower triangle of A_{2j}, made Hermitian */
        for (int a = 0; a < m; ++a) {
            for (int b = 0; b < a; ++b) {
                V[a * m + b] = A[pos * mm + a * m + b];
                V[b * m + a] = conj(A[pos * mm + a * m + b]);
            }
            V[a * m + a] = creal(A[pos * mm + a * m + a]);
        }
        herk_lower(m, Q + tl * mm, tmp);          /* Q_{2j-1}^H Q_{2j-1} */
        sub_into((int64_t)mm, V, tmp);
        if (has_right) {
            herk_lower(m, P + tr * mm, tmp);      /* P_{2j+1}^H P_{2j+1} */
            sub_into((int64_t)mm, V, tmp);
        }
        if (j < ne) {                              /* F_j = -Q_{2j+1}^H P_{2j+1} */
            zc *F = Bn + (j - 1) * mm;
            ctrans_prod(m, m, m, Q + tr * mm, P + tr * mm, F);
            for (size_t e = 0; e < mm; ++e) F[e] = -F[e];
        }
        if (y) {
            zc *v = yn + (j - 1) * mk;
            memcpy(v, y + pos * mk, sizeof(zc) * mk);
            ctrans_prod(m, m, k, Q + tl * mm, r + tl * mk, tmpk);   /* Q_{2j-1}^H r_{2j-1} */
            sub_into((int64_t)mk, v, tmpk);
            if (has_right) {
                ctrans_prod(m, m, k, P + tr * mm, r + tr * mk, tmpk); /* P_{2j+1}^H r_{2j+1} */
                sub_into((int64_t)mk, v, tmpk);
            }
        }
        free(tmp);
        free(tmpk);
    }
    return 0;
}

/*
 * Back-substitution of one level: given the stored L, P, Q, r of the no odd
 * blocks and the even unknowns xe [ne][m][k], write x [Nl][m][k]:
 *   x_{2j} = xe_j,  x_i = L_i^{-H} (r_i - P_i x_{i-1} - Q_i x_{i+1}) for odd i.
 */
void oracle_cr_backsub(int64_t Nl, int m, int k, const zc *L, const zc *P, const zc *Q,
                       const zc *r, const zc *xe, zc *x)
{
    const int64_t no = (Nl + 1) / 2, ne = Nl / 2;
    const size_t mm = (size_t)m * m, mk = (size_t)m * k;
    for (int64_t j = 1; j <= ne; ++j) memcpy(x + (2 * j - 1) * mk, xe + (j - 1) * mk, sizeof(zc) * mk);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < no; ++t) {
        const int64_t c = 2 * t;
        zc *xi = x + c * mk;
        memcpy(xi, r + t * mk, sizeof(zc) * mk);
        for (int a = 0; a < m; ++a)
            for (int b = 0; b < k; ++b) {
                zc v = xi[a * k + b];
                if (c >= 1) /* left even neighbour x_{i-1} */
                    for (int s = 0; s < m; ++s) v -= P[t * mm + a * m + s] * x[(c - 1) * mk + s * k + b];
                if (c + 1 <= Nl - 1) /* right even neighbour x_{i+1} */
                    for (int s = 0; s < m; ++s) v -= Q[t * mm + a * m + s] * x[(c + 1) * mk + s * k + b];
                xi[a * k + b] = v;
            }
        backward_subst(m, k, L + t * mm, xi);
    }
}

/* Full classic CR solve.  Returns 0 (x written) or 1 (not positive definite;
 * x filled with NaN).  info may be NULL. */
int oracle_cr_solve(int64_t N, int m, int k, const zc *A, const zc *B, const zc *y, zc *x,
                    oracle_info *info)
{
    const size_t mm = (size_t)m * m, mk = (size_t)m * k;
    int nlev = 1;
    for (int64_t n = N; n > 1; n /= 2) ++nlev;
    int64_t *Nl = (int64_t *)malloc(sizeof(int64_t) * nlev);
    /* per level: the level system (LA, LB, LY), the stored odd-block results
     * (SL, SP, SQ, SR) and the level's unknowns SX */
    zc **LA = calloc(nlev, sizeof(zc *)), **LB = calloc(nlev, sizeof(zc *)), **LY = calloc(nlev, sizeof(zc *));
    zc **SL = calloc(nlev, sizeof(zc *)), **SP = calloc(nlev, sizeof(zc *)), **SQ = calloc(nlev, sizeof(zc *)),
       **SR = calloc(nlev, sizeof(zc *)), **SX = calloc(nlev, sizeof(zc *));
    Nl[0] = N;
    for (int l = 1; l < nlev; ++l) Nl[l] = Nl[l - 1] / 2;
    int status = 0, flevel = 0, used = nlev;
    int64_t fblock = 0;
    for (int l = 0; l < nlev; ++l) {
        const int64_t no = (Nl[l] + 1) / 2, ne = Nl[l] / 2;
        const zc *Al = l ? LA[l] : A, *Bl = l ? LB[l] : B, *yl = l ? LY[l] : y;
        SL[l] = malloc(sizeof(zc) * mm * no); SP[l] = malloc(sizeof(zc) * mm * no);
        SQ[l] = malloc(sizeof(zc) * mm * no); SR[l] = malloc(sizeof(zc) * mk * no);
        zc *An = NULL, *Bn = NULL, *yn = NULL;
        if (l + 1 < nlev) {
            An = LA[l + 1] = malloc(sizeof(zc) * mm * ne);
            Bn = LB[l + 1] = malloc(sizeof(zc) * mm * (ne > 1 ? ne - 1 : 1));
            yn = LY[l + 1] = malloc(sizeof(zc) * mk * ne);
        }
        int64_t f = oracle_cr_level(Nl[l], m, k, Al, Bl, yl, SL[l], SP[l], SQ[l], SR[l], An, Bn, yn);
        if (f) { status = 1; flevel = l; fblock = f; used = l + 1; break; }
    }
    if (status == 0) {
        /* upward sweep, coarsest level first */
        for (int l = nlev - 1; l >= 0; --l) {
            SX[l] = (l == 0) ? x : malloc(sizeof(zc) * mk * Nl[l]);
            oracle_cr_backsub(Nl[l], m, k, SL[l], SP[l], SQ[l], SR[l], l + 1 < nlev ? SX[l + 1] : NULL, SX[l]);
        }
    } else {
        for (int64_t e = 0; e < N * (int64_t)mk; ++e) x[e] = CMPLX(NAN, NAN);
    }
    if (info) {
        info->status = status;
        info->level = status ? flevel : 0;
        info->block = status ? fblock : 0;
        info->orig_block = status ? (fblock << flevel) : 0;
    }
    (void)used;
    for (int l = 0; l < nlev; ++l) {
        free(SL[l]); free(SP[l]); free(SQ[l]); free(SR[l]);
        free(LA[l]); free(LB[l]); free(LY[l]);
        if (l > 0) free(SX[l]);
    }
    free(Nl); free(LA); free(LB); free(LY); free(SL); free(SP); free(SQ); free(SR); free(SX);
    return status;
}

/* out_j = A_j x_j + B_{j-1} x_{j-1} + B_j^H x_{j+1} (eq. Axb), with A_j the
 * Hermitian matrix given by its lower triangle and real diagonal. */
void oracle_matvec(int64_t N, int m, int k, const zc *A, const zc *B, const zc *x, zc *out)
{
    const size_t mm = (size_t)m * m, mk = (size_t)m * k;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < N; ++j)
        for (int a = 0; a < m; ++a)
            for (int b = 0; b < k; ++b) {
                zc v = 0;
                for (int s = 0; s < m; ++s) {
                    zc aas = (a > s) ? A[j * mm + a * m + s]
                           : (a < s) ? conj(A[j * mm + s * m + a]) : creal(A[j * mm + a * m + a]);
                    v += aas * x[j * mk + s * k + b];
                }
                if (j >= 1)
                    for (int s = 0; s < m; ++s) v += B[(j - 1) * mm + a * m + s] * x[(j - 1) * mk + s * k + b];
                if (j + 1 < N)
                    for (int s = 0; s < m; ++s) v += conj(B[j * mm + s * m + a]) * x[(j + 1) * mk + s * k + b];
                out[j * mk + a * k + b] = v;
            }
}

/*
 * Adjoint of x = A^{-1} y for the loss gradient gx = dL/dx (PyTorch's
 * convention for complex tensors: dL/dRe + i dL/dIm).  Writes
 *   gy  = A^{-1} gx                           (A is Hermitian)
 *   gA_j = -1/2 (gy_j x_j^H + x_j gy_j^H)     (Hermitian part of -gy_j x_j^H)
 *   gB_j = -(gy_{j+1} x_j^H + x_{j+1} gy_j^H) (B_j enters at (j+1,j) and, as
 *                                              B_j^H, at (j,j+1))
 * gA / gB may be NULL.  Returns the status of the re-solve.
 */
int oracle_cr_backward(int64_t N, int m, int k, const zc *A, const zc *B, const zc *x,
                       const zc *gx, zc *gy, zc *gA, zc *gB)
{
    const size_t mm = (size_t)m * m, mk = (size_t)m * k;
    int st = oracle_cr_solve(N, m, k, A, B, gx, gy, NULL);
    if (gA) {
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < N; ++j)
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) {
                    zc v = 0;
                    for (int c = 0; c < k; ++c)
                        v += gy[j * mk + a * k + c] * conj(x[j * mk + b * k + c])
                           + x[j * mk + a * k + c] * conj(gy[j * mk + b * k + c]);
                    gA[j * mm + a * m + b] = -0.5 * v;
                }
    }
    if (gB) {
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < N - 1; ++j)
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) {
                    zc v = 0;
                    for (int c = 0; c < k; ++c)
                        v += gy[(j + 1) * mk + a * k + c] * conj(x[j * mk + b * k + c])
                           + x[(j + 1) * mk + a * k + c] * conj(gy[j * mk + b * k + c]);
                    gB[j * mm + a * m + b] = -v;
                }
    }
    return st;
}

/* ------------------------------------------------------------------------
 * The paper's own method (Sec. 2 "Formulation of the Method" and Sec. 3,
 * Algorithm 1): both halves are reduced.  For a system of n = 2^L blocks,
 * with the boundary auxiliaries B_0 = B_n = 0 and A_0 = A_{n+1} = I, the odd
 * system (U, E, u) and the even system (V, F, v) of eq. Formulas are, for
 * j = 1..n/2,
 *   U_j = A_{2j-1} - B_{2j-2} A_{2j-2}^{-1} B_{2j-2}^H - B_{2j-1}^H A_{2j}^{-1} B_{2j-1}
 *   E_j = -B_{2j} A_{2j}^{-1} B_{2j-1}                              (j < n/2)
 *   u_j = y_{2j-1} - B_{2j-2} A_{2j-2}^{-1} y_{2j-2} - B_{2j-1}^H A_{2j}^{-1} y_{2j}
 *   V_j = A_{2j} - B_{2j-1} A_{2j-1}^{-1} B_{2j-1}^H - B_{2j}^H A_{2j+1}^{-1} B_{2j}
 *   F_j = -B_{2j+1} A_{2j+1}^{-1} B_{2j}                            (j < n/2)
 *   v_j = y_{2j} - B_{2j-1} A_{2j-1}^{-1} y_{2j-1} - B_{2j}^H A_{2j+1}^{-1} y_{2j+1}
 * Every product G1^H M^{-1} G2 is formed by Sec. 4's rule: M = L L^H,
 * (L\G1)^H (L\G2), and G^H M^{-1} G as the Hermitian (L\G)^H (L\G) built on
 * its lower triangle.  Both systems are solved recursively down to single
 * m x m blocks, which are solved by Cholesky; x is reassembled as
 * x_{2j-1} = (x_o)_j, x_{2j} = (x_e)_j.
 *
 * Readings: n must be a power of two (Algorithm 1 assumes it).  Each A_i of a
 * system is factored once, before the formulas use it.  Breakdown: a failing
 * pivot of the factorisation of some A_i ends that subsystem; the reported
 * failure is the smallest recursion depth with a failure and, within it, the
 * smallest 1-based index of the failing block in the original system (the
 * unknown x_i that the failing block belongs to).
 * ------------------------------------------------------------------------ */

/* G1^H M^{-1} G2 = (L\G1)^H (L\G2) for m x n1 and m x n2 operands. */
static void chol_cross(int m, int n1, int n2, const zc *L, const zc *G1, const zc *G2, zc *out)
{
    zc *T1 = (zc *)malloc(sizeof(zc) * (size_t)m * n1);
    zc *T2 = (zc *)malloc(sizeof(zc) * (size_t)m * n2);
    memcpy(T1, G1, sizeof(zc) * (size_t)m * n1);
    memcpy(T2, G2, sizeof(zc) * (size_t)m * n2);
    forward_subst(m, n1, L, T1);
    forward_subst(m, n2, L, T2);
    ctrans_prod(m, n1, n2, T1, T2, out);
    free(T1);
    free(T2);
}

/* G^H M^{-1} G = (L\G)^H (L\G), exactly Hermitian, for an m x m operand G. */
static void chol_herk(int m, const zc *L, const zc *G, zc *out)
{
    zc *T = (zc *)malloc(sizeof(zc) * (size_t)m * m);
    memcpy(T, G, sizeof(zc) * (size_t)m * m);
    forward_subst(m, m, L, T);
    herk_lower(m, T, out);
    free(T);
}

static void ctranspose(int m, const zc *X, zc *out)
{
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) out[a * m + b] = conj(X[b * m + a]);
}

/* The Hermitian matrix that the lower triangle of X describes. */
static void herm_lower(int m, const zc *X, zc *out)
{
    for (int a = 0; a < m; ++a) {
        for (int b = 0; b < a; ++b) {
            out[a * m + b] = X[a * m + b];
            out[b * m + a] = conj(X[a * m + b]);
        }
        out[a * m + a] = creal(X[a * m + a]);
    }
}

/*
 * One split of Algorithm 1 on a system of n blocks (n even): Cholesky of
 * every A_i (i = 1..n), then eq. Formulas for both halves.  Outputs U, V
 * [n/2][m][m], E, F [n/2-1][m][m], u, v [n/2][m][k] (u, v only when y is
 * given).  Returns 0 or the smallest failing 1-based block index i.
 */
int64_t oracle_alg1_split(int64_t n, int m, int k, const zc *A, const zc *B, const zc *y,
                          zc *U, zc *E, zc *u, zc *V, zc *F, zc *v)
{
    const size_t mm = (size_t)m * m, mk = (size_t)m * k;
    const int64_t h = n / 2;
    int64_t fail = 0;
    /* chol[i] = Cholesky factor of A_i, i = 0..n+1 (A_0 = A_{n+1} = I) */
    zc *chol = (zc *)calloc((size_t)(n + 2) * mm, sizeof(zc));
    for (int a = 0; a < m; ++a) {
        chol[a * m + a] = 1.0;
        chol[(size_t)(n + 1) * mm + a * m + a] = 1.0;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 1; i <= n; ++i) {
        if (chol_lower(m, A + (i - 1) * mm, chol + i * mm)) {
#pragma omp critical
            { if (fail == 0 || i < fail) fail = i; }
        }
    }
    if (fail) { free(chol); return fail; }
    zc *zero = (zc *)calloc(mm + mk, sizeof(zc)), *zeroy = zero + mm;
    /* B_i for i = 0..n (B_0 = B_n = 0) and y_i for i = 0..n+1 (y_0 = y_{n+1} = 0:
     * they only ever meet the zero couplings of the auxiliaries) */
#define BLK(i) (((i) >= 1 && (i) <= n - 1) ? B + ((i) - 1) * mm : zero)
#define YV(i) (((i) >= 1 && (i) <= n) ? y + ((i) - 1) * mk : zeroy)
#define LF(i) (chol + (i) * mm)

#pragma omp parallel for schedule(static)
    for (int64_t j = 1; j <= h; ++j) {
        zc *t = (zc *)malloc(sizeof(zc) * mm), *g = (zc *)malloc(sizeof(zc) * mm);
        zc *g2 = (zc *)malloc(sizeof(zc) * mm), *tk = (zc *)malloc(sizeof(zc) * (mk ? mk : 1));
        /* odd system, row j (unknown x_{2j-1}) */
        zc *Uj = U + (j - 1) * mm;
        herm_lower(m, A + (2 * j - 2) * mm, Uj);
        ctranspose(m, BLK(2 * j - 2), g);                 /* B_{2j-2} A_{2j-2}^{-1} B_{2j-2}^H */
        chol_herk(m, LF(2 * j - 2), g, t);
        sub_into((int64_t)mm, Uj, t);
        chol_herk(m, LF(2 * j), BLK(2 * j - 1), t);       /* B_{2j-1}^H A_{2j}^{-1} B_{2j-1} */
        sub_into((int64_t)mm, Uj, t);
        if (j < h) {                                      /* E_j = -B_{2j} A_{2j}^{-1} B_{2j-1} */
            zc *Ej = E + (j - 1) * mm;
            ctranspose(m, BLK(2 * j), g);
            chol_cross(m, m, m, LF(2 * j), g, BLK(2 * j - 1), Ej);
            for (size_t e = 0; e < mm; ++e) Ej[e] = -Ej[e];
        }
        if (y) {
            zc *uj = u + (j - 1) * mk;
            memcpy(uj, YV(2 * j - 1), sizeof(zc) * mk);
            ctranspose(m, BLK(2 * j - 2), g);             /* B_{2j-2} A_{2j-2}^{-1} y_{2j-2} */
            chol_cross(m, m, k, LF(2 * j - 2), g, YV(2 * j - 2), tk);
            sub_into((int64_t)mk, uj, tk);
            chol_cross(m, m, k, LF(2 * j), BLK(2 * j - 1), YV(2 * j), tk); /* B_{2j-1}^H A_{2j}^{-1} y_{2j} */
            sub_into((int64_t)mk, uj, tk);
        }
        /* even system, row j (unknown x_{2j}) */
        zc *Vj = V + (j - 1) * mm;
        herm_lower(m, A + (2 * j - 1) * mm, Vj);
        ctranspose(m, BLK(2 * j - 1), g);                 /* B_{2j-1} A_{2j-1}^{-1} B_{2j-1}^H */
        chol_herk(m, LF(2 * j - 1), g, t);
        sub_into((int64_t)mm, Vj, t);
        chol_herk(m, LF(2 * j + 1), BLK(2 * j), t);       /* B_{2j}^H A_{2j+1}^{-1} B_{2j} */
        sub_into((int64_t)mm, Vj, t);
        if (j < h) {                                      /* F_j = -B_{2j+1} A_{2j+1}^{-1} B_{2j} */
            zc *Fj = F + (j - 1) * mm;
            ctranspose(m, BLK(2 * j + 1), g2);
            chol_cross(m, m, m, LF(2 * j + 1), g2, BLK(2 * j), Fj);
            for (size_t e = 0; e < mm; ++e) Fj[e] = -Fj[e];
        }
        if (y) {
            zc *vj = v + (j - 1) * mk;
            memcpy(vj, YV(2 * j), sizeof(zc) * mk);
            ctranspose(m, BLK(2 * j - 1), g);             /* B_{2j-1} A_{2j-1}^{-1} y_{2j-1} */
            chol_cross(m, m, k, LF(2 * j - 1), g, YV(2 * j - 1), tk);
            sub_into((int64_t)mk, vj, tk);
            chol_cross(m, m, k, LF(2 * j + 1), BLK(2 * j), YV(2 * j + 1), tk); /* B_{2j}^H A_{2j+1}^{-1} y_{2j+1} */
            sub_into((int64_t)mk, vj, tk);
        }
        free(t); free(g); free(g2); free(tk);
    }
#undef BLK
#undef YV
#undef LF
    free(zero);
    free(chol);
    return 0;
}

typedef struct { int have; int32_t level; int64_t orig; } alg1_fail;

static void alg1_note(alg1_fail *f, int32_t level, int64_t orig)
{
    if (!f->have || level < f->level || (level == f->level && orig < f->orig)) {
        f->have = 1;
        f->level = level;
        f->orig = orig;
    }
}

/* SOLVER of Algorithm 1 on a subsystem of n blocks whose block i (1-based)
 * is block orig0 + (i-1) * stride + 1 of the original system. */
static void alg1_solver(int64_t n, int m, int k, const zc *A, const zc *B, const zc *y, zc *x, int32_t depth,
                        int64_t orig0, int64_t stride, alg1_fail *fail)
{
    const size_t mm = (size_t)m * m, mk = (size_t)m * k;
    if (n == 1) {
        zc *L = (zc *)malloc(sizeof(zc) * mm);
        if (chol_lower(m, A, L)) {
            alg1_note(fail, depth, orig0 + 1);
        } else {
            memcpy(x, y, sizeof(zc) * mk);
            forward_subst(m, k, L, x);
            backward_subst(m, k, L, x);
        }
        free(L);
        return;
    }
    const int64_t h = n / 2;
    zc *U = (zc *)malloc(sizeof(zc) * mm * h), *V = (zc *)malloc(sizeof(zc) * mm * h);
    zc *E = (zc *)malloc(sizeof(zc) * mm * (h > 1 ? h - 1 : 1)), *F = (zc *)malloc(sizeof(zc) * mm * (h > 1 ? h - 1 : 1));
    zc *u = (zc *)malloc(sizeof(zc) * mk * h), *v = (zc *)malloc(sizeof(zc) * mk * h);
    zc *xo = (zc *)malloc(sizeof(zc) * mk * h), *xe = (zc *)malloc(sizeof(zc) * mk * h);
    int64_t f = oracle_alg1_split(n, m, k, A, B, y, U, E, u, V, F, v);
    if (f) {
        /* report every failing block of this subsystem at this depth */
        zc *L = (zc *)malloc(sizeof(zc) * mm);
        for (int64_t i = 1; i <= n; ++i)
            if (chol_lower(m, A + (i - 1) * mm, L)) alg1_note(fail, depth, orig0 + (i - 1) * stride + 1);
        free(L);
    } else {
        alg1_solver(h, m, k, U, E, u, xo, depth + 1, orig0, 2 * stride, fail);          /* x_o */
        alg1_solver(h, m, k, V, F, v, xe, depth + 1, orig0 + stride, 2 * stride, fail); /* x_e */
        for (int64_t j = 1; j <= h; ++j) {
            memcpy(x + (2 * j - 2) * mk, xo + (j - 1) * mk, sizeof(zc) * mk);
            memcpy(x + (2 * j - 1) * mk, xe + (j - 1) * mk, sizeof(zc) * mk);
        }
    }
    free(U); free(V); free(E); free(F); free(u); free(v); free(xo); free(xe);
}

/* Full solve by Algorithm 1 (N a power of two).  Returns 0 (x written),
 * 1 (not positive definite; x filled with NaN) or -1 (N not a power of two).
 * info->level is the recursion depth of the first breakdown (0 = the input
 * system, log2 N = the single blocks); the recursion numbers blocks only
 * within each subsystem, so info->block repeats orig_block. */
int oracle_alg1_solve(int64_t N, int m, int k, const zc *A, const zc *B, const zc *y, zc *x, oracle_info *info)
{
    if (N < 1 || (N & (N - 1))) return -1;
    alg1_fail fail = {0, 0, 0};
    alg1_solver(N, m, k, A, B, y, x, 0, 0, 1, &fail);
    if (fail.have)
        for (int64_t e = 0; e < N * (int64_t)m * k; ++e) x[e] = CMPLX(NAN, NAN);
    if (info) {
        info->status = fail.have;
        info->level = fail.have ? fail.level : 0;
        info->block = fail.have ? fail.orig : 0;
        info->orig_block = fail.have ? fail.orig : 0;
    }
    return fail.have;
}
