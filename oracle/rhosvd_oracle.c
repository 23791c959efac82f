/*
 * rhosvd_oracle.c -- plain, slow CPU FP64 oracle for the RHOSVD canonical-to-Tucker
 * reduction (Khoromskaia & Khoromskij, "Reduced Higher Order SVD").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's CPU
 * baseline leg may load this library.  It shares no code with the CUDA library.
 *
 * Every routine follows the definition it implements, written out with plain
 * loops; no blocking, no fusion, no reordering beyond what the definition states.
 *
 *   orc_col_norm          Euclidean norm of a column (scaled to avoid under/overflow)
 *   orc_normalize         Sec. 2.1, eq. can_A3: normalised canonical vectors,
 *                          weights absorb the norms; terms with a zero vector dropped
 *   orc_householder_r     Householder QR (R factor only) -- used when R >= n so that the
 *                          SVD of U (eq. SVD_Ul) reduces to an n x n triangular factor
 *   orc_jacobi_left       one-sided (Hestenes) Jacobi SVD: left singular vectors and
 *                          singular values, descending (eq. SVD_Ul)
 *   orc_side_svd          SVD of one side matrix U^(l) (eq. SVD_Ul; Thm. 2.3 remarks
 *                          that R < n is handled "along the same line")
 *   orc_eps_rank          epsilon-rank of the truncated SVD (eq. svdr; Thm. 2.3)
 *   orc_project           D_{l,0} V_0^T = Z_0^T U^(l)   (Def. 2.2 / Prop. 2.2)
 *   orc_core              beta_0 = xi x_1 [D V_0^T] x_2 ... (Prop. 2.2), explicit loops
 *   orc_c2t               the whole RHOSVD, Def. 2.2
 *   orc_cp_hadamard       Hadamard product of two canonical tensors (Sec. 3 eq. rho_ten;
 *                          Lemma 4.2): columns u^a_i .* u^b_j, weights xi^a_i xi^b_j
 *   orc_cp_sum            alpha A + beta B as a canonical tensor (Sec. 4.3): concatenation
 *
 * Matrices are column-major.  Parity of this oracle: pinned by the tests under tests/
 * (LAPACK SVD, closed forms, brute force on the full tensor).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NOMEM (-2)
#define ORC_ERR_NOTCONV (-3)
#define ORC_ERR_RANK (-4)

/* ||x||_2 = m * sqrt(sum (x_i/m)^2) with m = max |x_i|; exact 0 for the zero vector. */
double orc_col_norm(int n, const double* x)
{
    double m = 0.0;
    for (int i = 0; i < n; ++i) {
        double a = fabs(x[i]);
        if (a > m) m = a;
    }
    if (m == 0.0) return 0.0;
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        double t = x[i] / m;
        s += t * t;
    }
    return m * sqrt(s);
}

/*
 * Normalisation (Sec. 2.1: "with normalized canonical vectors").
 * Input: three side matrices U[l] (n[l] x R, leading dimension ld[l]) and weights xi.
 * Output: Un[l] (n[l] x R, ld n[l]) with unit columns, xin[nu] = xi[nu] * prod_l ||u_nu^l||,
 *         norms[l*R + nu] = ||u_nu^l||, keep[nu] = 1 if the term is kept.
 * A term whose vector is zero in some mode is the zero tensor; it cannot be normalised
 * and is dropped: its columns in Un are zero and xin = 0.
 * Returns the number of kept terms.
 */
int orc_normalize(const int* n, int R, const double* const* U, const int* ld, const double* xi,
                  double* const* Un, double* xin, double* norms, int* keep)
{
    int kept = 0;
    for (int nu = 0; nu < R; ++nu) {
        double w = xi[nu];
        int ok = 1;
        for (int l = 0; l < 3; ++l) {
            double d = orc_col_norm(n[l], U[l] + (size_t)nu * ld[l]);
            norms[(size_t)l * R + nu] = d;
            if (d == 0.0) ok = 0;
        }
        for (int l = 0; l < 3; ++l) {
            const double* src = U[l] + (size_t)nu * ld[l];
            double* dst = Un[l] + (size_t)nu * n[l];
            double d = norms[(size_t)l * R + nu];
            for (int i = 0; i < n[l]; ++i) dst[i] = ok ? src[i] / d : 0.0;
            if (ok) w *= d;
        }
        xin[nu] = ok ? w : 0.0;
        keep[nu] = ok;
        kept += ok;
    }
    return kept;
}

/*
 * Householder QR of A (m x n, m >= n, leading dimension lda), overwriting A.
 * Writes the n x n upper-triangular factor to Rout (leading dimension n).
 * Reflector j: v = x - alpha e_1 with alpha = -sign(x_1) ||x||, H = I - 2 v v^T / v^T v.
 */
int orc_householder_r(int m, int n, double* A, int lda, double* Rout)
{
    if (m < n) return ORC_ERR_ARG;
    double* v = (double*)malloc(sizeof(double) * (size_t)m);
    if (!v) return ORC_ERR_NOMEM;
    for (int j = 0; j < n; ++j) {
        int len = m - j;
        double* x = A + (size_t)j * lda + j;
        double xn = orc_col_norm(len, x);
        if (xn == 0.0) continue;
        double alpha = (x[0] >= 0.0) ? -xn : xn;
        for (int i = 0; i < len; ++i) v[i] = x[i];
        v[0] -= alpha;
        double vv = 0.0;
        for (int i = 0; i < len; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        for (int c = j; c < n; ++c) {
            double* col = A + (size_t)c * lda + j;
            double w = 0.0;
            for (int i = 0; i < len; ++i) w += v[i] * col[i];
            double f = 2.0 * w / vv;
            for (int i = 0; i < len; ++i) col[i] -= f * v[i];
        }
        /* the reflected column j is exactly alpha e_1 */
        x[0] = alpha;
        for (int i = 1; i < len; ++i) x[i] = 0.0;
    }
    for (int c = 0; c < n; ++c)
        for (int r = 0; r < n; ++r)
            Rout[(size_t)c * n + r] = (r <= c) ? A[(size_t)c * lda + r] : 0.0;
    free(v);
    return ORC_OK;
}

/*
 * One-sided (Hestenes) Jacobi: right-multiply A (m x n, leading dimension m) by plane
 * rotations until its columns are mutually orthogonal; then A = Z diag(sigma) V^T with
 * sigma_i = ||a_i|| and z_i = a_i / sigma_i.  For the pair (p,q) with
 * alpha = a_p.a_p, beta = a_q.a_q, gamma = a_p.a_q the rotation angle zeroes gamma:
 * zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
 * c = 1/sqrt(1+t^2), s = c t.  A pair counts as orthogonal when |gamma| <= tol sqrt(alpha beta),
 * tol = m u.  A column whose norm is <= m u ||A||_F is numerically zero (its singular value is
 * below what FP64 resolves in A) and is not rotated; without this rule rotations among such
 * noise-level columns never settle.  Its singular value is reported as exactly 0 and its left
 * vector as a zero column: the noise left in it is not orthogonal to the other columns, so it
 * is no singular vector, and an epsilon-rank taken with eps = 0 must not count it.
 * Output: sigma (n values, descending) and Z (m x n, column i <-> sigma_i; zero column
 * for sigma_i = 0).  A is overwritten.  Returns sweeps used, or ORC_ERR_NOTCONV.
 */
int orc_jacobi_left(int m, int n, double* A, double* sigma, double* Z, int max_sweeps)
{
    const double tol = (double)m * DBL_EPSILON;
    double fro2 = 0.0;
    for (size_t e = 0; e < (size_t)m * n; ++e) fro2 += A[e] * A[e];
    const double negligible = tol * tol * fro2;
    int sweep = 0, converged = 0;
    for (sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
        long rotations = 0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double* ap = A + (size_t)p * m;
                double* aq = A + (size_t)q * m;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int i = 0; i < m; ++i) {
                    alpha += ap[i] * ap[i];
                    beta += aq[i] * aq[i];
                    gamma += ap[i] * aq[i];
                }
                if (alpha <= negligible || beta <= negligible || gamma == 0.0) continue;
                if (fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta)) continue;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t;
                if (fabs(zeta) > 1e150) t = 0.5 / zeta;
                else t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = c * t;
                for (int i = 0; i < m; ++i) {
                    double x = ap[i], y = aq[i];
                    ap[i] = c * x - s * y;
                    aq[i] = s * x + c * y;
                }
                ++rotations;
            }
        }
        if (rotations == 0) converged = 1;
    }
    /* singular values = column norms; order descending (selection sort on an index) */
    int* idx = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double* s = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!idx || !s) { free(idx); free(s); return ORC_ERR_NOMEM; }
    for (int j = 0; j < n; ++j) {
        idx[j] = j;
        s[j] = orc_col_norm(m, A + (size_t)j * m);
        if (s[j] * s[j] <= negligible) s[j] = 0.0;          /* numerically zero column */
    }
    for (int a = 0; a < n; ++a) {
        int best = a;
        for (int b = a + 1; b < n; ++b) if (s[idx[b]] > s[idx[best]]) best = b;
        int tmp = idx[a]; idx[a] = idx[best]; idx[best] = tmp;
    }
    for (int a = 0; a < n; ++a) {
        int j = idx[a];
        sigma[a] = s[j];
        for (int i = 0; i < m; ++i)
            Z[(size_t)a * m + i] = (s[j] > 0.0) ? A[(size_t)j * m + i] / s[j] : 0.0;
    }
    free(idx); free(s);
    return converged ? sweep : ORC_ERR_NOTCONV;
}

/*
 * SVD of one normalised side matrix Un (n x R, leading dimension n), eq. SVD_Ul:
 * Un = Z D V^T.  Returns in sigma the q = min(n, R) singular values (descending) and in
 * Z (n x q) the matching left singular vectors.
 * R >= n: Un^T = Q_h R_h (Householder), so Un = R_h^T Q_h^T and the left singular
 *         vectors / values of Un are those of the n x n matrix R_h^T.
 * R <  n: one-sided Jacobi on Un itself (its R columns).
 */
int orc_side_svd(int n, int R, const double* Un, double* sigma, double* Z, int max_sweeps)
{
    int rc;
    if (R >= n) {
        double* At = (double*)malloc(sizeof(double) * (size_t)R * n);
        double* Rh = (double*)malloc(sizeof(double) * (size_t)n * n);
        double* L = (double*)malloc(sizeof(double) * (size_t)n * n);
        if (!At || !Rh || !L) { free(At); free(Rh); free(L); return ORC_ERR_NOMEM; }
        for (int i = 0; i < n; ++i)
            for (int nu = 0; nu < R; ++nu)
                At[(size_t)i * R + nu] = Un[(size_t)nu * n + i];   /* At = Un^T (R x n) */
        rc = orc_householder_r(R, n, At, R, Rh);
        if (rc == ORC_OK) {
            for (int c = 0; c < n; ++c)
                for (int r = 0; r < n; ++r) L[(size_t)c * n + r] = Rh[(size_t)r * n + c];
            rc = orc_jacobi_left(n, n, L, sigma, Z, max_sweeps);
        }
        free(At); free(Rh); free(L);
    } else {
        double* A = (double*)malloc(sizeof(double) * (size_t)n * R);
        if (!A) return ORC_ERR_NOMEM;
        memcpy(A, Un, sizeof(double) * (size_t)n * R);
        rc = orc_jacobi_left(n, R, A, sigma, Z, max_sweeps);
        free(A);
    }
    return rc;
}

/*
 * epsilon-rank (Thm. 2.3 with a relative Frobenius threshold per mode):
 * the smallest r in [0, q] with sum_{k>r} sigma_k^2 <= eps^2 sum_k sigma_k^2.
 * Tails are summed from the smallest singular value upwards.
 */
int orc_eps_rank(int q, const double* sigma, double eps)
{
    double total = 0.0;
    for (int k = q - 1; k >= 0; --k) total += sigma[k] * sigma[k];
    double thr = eps * eps * total;
    double tail = 0.0;            /* sum_{k > r} sigma_k^2, starting at r = q */
    int r = q;
    while (r > 0) {
        double t = tail + sigma[r - 1] * sigma[r - 1];
        if (t <= thr) { tail = t; --r; } else break;
    }
    return r;
}

/* V (r x R, leading dimension r) = Z0^T Un, Z0 = first r columns of Z (n x ., ld n). */
void orc_project(int n, int R, int r, const double* Z, const double* Un, double* V)
{
    for (int nu = 0; nu < R; ++nu)
        for (int i = 0; i < r; ++i) {
            double s = 0.0;
            for (int x = 0; x < n; ++x) s += Z[(size_t)i * n + x] * Un[(size_t)nu * n + x];
            V[(size_t)nu * r + i] = s;
        }
}

/* beta(i,j,m) = sum_nu xi_nu V1(i,nu) V2(j,nu) V3(m,nu), stored beta[i + r1 (j + r2 m)]. */
void orc_core(int R, const int* r, const double* V1, const double* V2, const double* V3,
              const double* xi, double* beta)
{
    size_t cnt = (size_t)r[0] * r[1] * r[2];
    for (size_t e = 0; e < cnt; ++e) beta[e] = 0.0;
    for (int nu = 0; nu < R; ++nu) {
        double w = xi[nu];
        if (w == 0.0) continue;
        for (int m = 0; m < r[2]; ++m) {
            double a3 = w * V3[(size_t)nu * r[2] + m];
            for (int j = 0; j < r[1]; ++j) {
                double a23 = a3 * V2[(size_t)nu * r[1] + j];
                double* dst = beta + (size_t)r[0] * (j + (size_t)r[1] * m);
                const double* v1 = V1 + (size_t)nu * r[0];
                for (int i = 0; i < r[0]; ++i) dst[i] += a23 * v1[i];
            }
        }
    }
}

/*
 * RHOSVD (Def. 2.2), d = 3.
 * Inputs: n[3], R, U[l] (n[l] x R, leading dimension ld[l]), xi[R], eps, ranks[3]
 *         (ranks[l] > 0 fixes r_l = min(ranks[l], q_l); 0 selects the epsilon rule).
 * Outputs (caller-allocated):
 *   r_out[3]            Tucker ranks
 *   Z[l]                n[l] x q_l, all left singular vectors of the normalised U^(l),
 *                        q_l = min(n[l], R); the first r_l columns are Z_0^(l)
 *   sigma[l]            q_l singular values, descending
 *   V[l]                r_max x R capacity; V^(l) = Z_0^T Un^(l) stored r_l x R (ld r_l)
 *   beta                r_max^3 capacity; r1 x r2 x r3, beta[i + r1 (j + r2 m)]
 *   xin                 R normalised weights (0 for dropped terms)
 *   stats[4]            {kept terms, ||xin||, unused, unused}
 * Returns ORC_OK or an error code (ORC_ERR_RANK if some r_l > r_max).
 */
int orc_c2t(const int* n, int R, const double* const* U, const int* ld, const double* xi,
            double eps, const int* ranks, int r_max, int max_sweeps,
            int* r_out, double* const* Z, double* const* sigma, double* const* V,
            double* beta, double* xin, double* stats)
{
    if (R < 0) return ORC_ERR_ARG;
    for (int l = 0; l < 3; ++l) if (n[l] <= 0 || ld[l] < n[l]) return ORC_ERR_ARG;
    double* Un[3] = {0, 0, 0};
    double* norms = (double*)malloc(sizeof(double) * 3 * (size_t)(R > 0 ? R : 1));
    int* keep = (int*)malloc(sizeof(int) * (size_t)(R > 0 ? R : 1));
    int rc = ORC_OK;
    for (int l = 0; l < 3; ++l) Un[l] = (double*)malloc(sizeof(double) * (size_t)n[l] * (R > 0 ? R : 1));
    if (!norms || !keep || !Un[0] || !Un[1] || !Un[2]) { rc = ORC_ERR_NOMEM; goto done; }

    int kept = orc_normalize(n, R, U, ld, xi, Un, xin, norms, keep);
    double xn2 = 0.0;
    for (int nu = 0; nu < R; ++nu) xn2 += xin[nu] * xin[nu];
    stats[0] = (double)kept;
    stats[1] = sqrt(xn2);

    for (int l = 0; l < 3; ++l) {
        int q = n[l] < R ? n[l] : R;
        if (q > 0) {
            int s = orc_side_svd(n[l], R, Un[l], sigma[l], Z[l], max_sweeps);
            if (s < 0) { rc = s; goto done; }
        }
        int r = ranks[l] > 0 ? (ranks[l] < q ? ranks[l] : q) : orc_eps_rank(q, sigma[l], eps);
        r_out[l] = r;
        if (r > r_max) rc = ORC_ERR_RANK;
    }
    if (rc != ORC_OK) goto done;
    for (int l = 0; l < 3; ++l) orc_project(n[l], R, r_out[l], Z[l], Un[l], V[l]);
    orc_core(R, r_out, V[0], V[1], V[2], xin, beta);
done:
    for (int l = 0; l < 3; ++l) free(Un[l]);
    free(norms); free(keep);
    return rc;
}

/*
 * Hadamard product C = A .* B of canonical tensors (Sec. 3, eq. rho_ten; Lemma 4.2):
 * term nu = i + Ra * j has columns c_nu^(l) = a_i^(l) .* b_j^(l) and weight xa_i * xb_j.
 * All matrices n[l] x rank with leading dimension n[l].
 */
void orc_cp_hadamard(const int* n, int Ra, const double* const* Ua, const double* xa,
                     int Rb, const double* const* Ub, const double* xb,
                     double* const* Uc, double* xc)
{
    for (int j = 0; j < Rb; ++j)
        for (int i = 0; i < Ra; ++i) {
            size_t nu = (size_t)i + (size_t)Ra * j;
            xc[nu] = xa[i] * xb[j];
            for (int l = 0; l < 3; ++l)
                for (int x = 0; x < n[l]; ++x)
                    Uc[l][nu * n[l] + x] = Ua[l][(size_t)i * n[l] + x] * Ub[l][(size_t)j * n[l] + x];
        }
}

/* alpha A + beta B as one canonical tensor: columns [A | B], weights [alpha xa | beta xb]. */
void orc_cp_sum(const int* n, double alpha, int Ra, const double* const* Ua, const double* xa,
                double beta, int Rb, const double* const* Ub, const double* xb,
                double* const* Uc, double* xc)
{
    for (int i = 0; i < Ra; ++i) {
        xc[i] = alpha * xa[i];
        for (int l = 0; l < 3; ++l)
            memcpy(Uc[l] + (size_t)i * n[l], Ua[l] + (size_t)i * n[l], sizeof(double) * n[l]);
    }
    for (int j = 0; j < Rb; ++j) {
        xc[Ra + j] = beta * xb[j];
        for (int l = 0; l < 3; ++l)
            memcpy(Uc[l] + (size_t)(Ra + j) * n[l], Ub[l] + (size_t)j * n[l], sizeof(double) * n[l]);
    }
}
