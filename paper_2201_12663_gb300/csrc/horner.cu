// horner.cu -- the polynomial P(A) = a_0 I + a_1 A + ... + a_n A^n of a canonical tensor A
// (products are Hadamard products, I the all-ones tensor), evaluated by the Horner scheme
// P(x) = a_0 + x (a_1 + x (a_2 + ... + x (a_{n-1} + a_n x)...)) with a rank reduction after every
// product (Sec. 5, the tensor-valued polynomial of a reference potential):
//   Y_n = a_n I;  Y_k = C2C( A (.) Y_{k+1} + a_k I ),  k = n-1 .. 0,
// C2C = RHOSVD (rhosvd_c2t) followed by the slice-SVD Tucker-to-canonical transform (rhosvd_t2c).
// Host code sequencing the library's own entry points; the only kernel here writes the rank-one
// constant term.  The ranks of each step size the next launches, so the stream is synchronised
// twice per degree.
#include "internal.cuh"
#include <cmath>
#include <cstring>

namespace rh {
namespace {

// column `col` of each factor = 1, weight xi[col] = a (the term a I)
__global__ void k_const_term(double* U0, double* U1, double* U2, int n0, int n1, int n2, int ld0, int ld1,
                             int ld2, long long col, double* xi, double a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n0) U0[col * ld0 + i] = 1.0;
    if (i < n1) U1[col * ld1 + i] = 1.0;
    if (i < n2) U2[col * ld2 + i] = 1.0;
    if (i == 0) xi[col] = a;
}

int launch_const_term(double* const U[3], const int ld[3], const int n[3], long long col, double* xi, double a,
                      cudaStream_t st)
{
    const int nm = n[0] > n[1] ? (n[0] > n[2] ? n[0] : n[2]) : (n[1] > n[2] ? n[1] : n[2]);
    k_const_term<<<(nm + 255) / 256, 256, 0, st>>>(U[0], U[1], U[2], n[0], n[1], n[2], ld[0], ld[1], ld[2], col, xi,
                                                    a);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RHOSVD_OK : RHOSVD_ERR_CUDA;
}

struct HornerPlan {
    int deg;                   // degree after dropping trailing zero coefficients (-1: zero polynomial)
    long long rin_max;         // largest rank entering a reduction: R_A R_max + 1
    size_t o_P[3], o_Px, o_Z[3], o_beta, o_sig[3], o_info, o_ints, o_c2t, c2t_bytes, o_t2c, t2c_bytes, total;
};

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

int horner_degree(const double* c, int nc)
{
    int d = -1;
    for (int k = 0; k < nc; ++k)
        if (c[k] != 0.0) d = k;
    return d;
}

int horner_plan(const rhosvd_cp* A, int ncoeffs, const double* coeffs, const rhosvd_opts* o, int R_max,
                HornerPlan* pl)
{
    if (!A || !o || ncoeffs < 1 || R_max < 1 || A->R < 0) return RHOSVD_ERR_INVALID_ARG;
    if (o->r_max < 1 || o->r_max > KMAX) return RHOSVD_ERR_INVALID_ARG;
    if (o->out_fp32 != 0) return RHOSVD_ERR_INVALID_ARG;     // each step reads its Tucker tensor back in FP64
    if ((long long)o->r_max * o->r_max > RHOSVD_T2C_SLICE_MAX) return RHOSVD_ERR_INVALID_ARG;
    pl->deg = coeffs ? horner_degree(coeffs, ncoeffs) : ncoeffs - 1;
    pl->rin_max = (long long)A->R * R_max + 1;
    if (pl->rin_max > 0x7fffffffLL) return RHOSVD_ERR_INVALID_ARG;
    rhosvd_cp big = *A;
    big.R = (int)pl->rin_max;
    const size_t c2t = rhosvd_c2t_workspace_size(&big, o);
    if (c2t == 0) return RHOSVD_ERR_INVALID_ARG;
    rhosvd_tucker_in tin;
    memset(&tin, 0, sizeof(tin));
    for (int l = 0; l < 3; ++l) {
        tin.n[l] = A->n[l];
        tin.r[l] = o->r_max;
    }
    const size_t t2c = rhosvd_t2c_workspace_size(&tin);
    if (t2c == 0) return RHOSVD_ERR_INVALID_ARG;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off += al256(bytes); return at; };
    for (int l = 0; l < 3; ++l) pl->o_P[l] = take(sizeof(double) * (size_t)A->n[l] * (size_t)pl->rin_max);
    pl->o_Px = take(sizeof(double) * (size_t)pl->rin_max);
    for (int l = 0; l < 3; ++l) pl->o_Z[l] = take(sizeof(double) * (size_t)A->n[l] * o->r_max);
    pl->o_beta = take(sizeof(double) * (size_t)o->r_max * o->r_max * o->r_max);
    for (int l = 0; l < 3; ++l) pl->o_sig[l] = take(sizeof(double) * KMAX);
    pl->o_info = take(sizeof(rhosvd_info));
    pl->o_ints = take(sizeof(int) * 2);
    pl->o_c2t = take(c2t);
    pl->c2t_bytes = c2t;
    pl->o_t2c = take(t2c);
    pl->t2c_bytes = t2c;
    pl->total = off;
    return RHOSVD_OK;
}

}  // namespace
}  // namespace rh

extern "C" size_t rhosvd_cp_horner_workspace_size(const rhosvd_cp* A, int ncoeffs, const rhosvd_opts* opts,
                                                  int R_max)
{
    rh::HornerPlan pl;
    return rh::horner_plan(A, ncoeffs, nullptr, opts, R_max, &pl) == RHOSVD_OK ? pl.total : 0;
}

extern "C" int rhosvd_cp_horner(const rhosvd_cp* A, const double* coeffs, int ncoeffs, const rhosvd_opts* opts,
                                double eps_t2c, int R_max, double* const U_out[3], const int ldu[3], double* xi_out,
                                int* R_out, rhosvd_horner_step* steps, void* workspace, size_t bytes, void* stream)
{
    using namespace rh;
    if (!coeffs || !U_out || !ldu || !xi_out || !R_out || !(eps_t2c >= 0.0)) return RHOSVD_ERR_INVALID_ARG;
    for (int k = 0; k < ncoeffs; ++k)
        if (!std::isfinite(coeffs[k])) return RHOSVD_ERR_INVALID_ARG;
    HornerPlan pl;
    int rc = horner_plan(A, ncoeffs, coeffs, opts, R_max, &pl);
    if (rc) return rc;
    for (int l = 0; l < 3; ++l) {
        if (A->n[l] < 1 || A->ld[l] < A->n[l] || !U_out[l] || ldu[l] < A->n[l]) return RHOSVD_ERR_INVALID_ARG;
        if (A->R > 0 && !A->U[l]) return RHOSVD_ERR_INVALID_ARG;
    }
    if (A->R > 0 && !A->xi) return RHOSVD_ERR_INVALID_ARG;
    if (!workspace || bytes < pl.total || ((uintptr_t)workspace & 255) != 0) return RHOSVD_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* ws = (unsigned char*)workspace;
    *R_out = 0;
    if (pl.deg < 0) return RHOSVD_OK;                        // the zero polynomial
    // Y_n = a_n I, held in the output buffers (every Y_k lives there)
    rc = launch_const_term(U_out, ldu, A->n, 0, xi_out, coeffs[pl.deg], st);
    if (rc) return rc;
    int RY = 1;
    double* P[3];
    int ldP[3];
    for (int l = 0; l < 3; ++l) {
        P[l] = (double*)(ws + pl.o_P[l]);
        ldP[l] = A->n[l];
    }
    double* Px = (double*)(ws + pl.o_Px);
    rhosvd_info* info_d = (rhosvd_info*)(ws + pl.o_info);
    int* ints_d = (int*)(ws + pl.o_ints);
    rhosvd_tucker tk;
    memset(&tk, 0, sizeof(tk));
    for (int l = 0; l < 3; ++l) {
        tk.Z[l] = (double*)(ws + pl.o_Z[l]);
        tk.sigma[l] = (double*)(ws + pl.o_sig[l]);
    }
    tk.beta = (double*)(ws + pl.o_beta);
    tk.info = info_d;
    int step = 0;
    for (int k = pl.deg - 1; k >= 0; --k, ++step) {
        // A (.) Y_{k+1}  (+ a_k I)
        rhosvd_cp Y;
        memset(&Y, 0, sizeof(Y));
        for (int l = 0; l < 3; ++l) {
            Y.n[l] = A->n[l];
            Y.U[l] = U_out[l];
            Y.ld[l] = ldu[l];
        }
        Y.R = RY;
        Y.xi = xi_out;
        rc = rhosvd_cp_hadamard(A, &Y, P, ldP, Px, stream);
        if (rc) return rc;
        long long Rin = (long long)A->R * RY;
        if (coeffs[k] != 0.0) {
            rc = launch_const_term(P, ldP, A->n, Rin, Px, coeffs[k], st);
            if (rc) return rc;
            ++Rin;
        }
        rhosvd_cp X;
        memset(&X, 0, sizeof(X));
        for (int l = 0; l < 3; ++l) {
            X.n[l] = A->n[l];
            X.U[l] = P[l];
            X.ld[l] = ldP[l];
        }
        X.R = (int)Rin;
        X.xi = Px;
        const size_t need = rhosvd_c2t_workspace_size(&X, opts);
        if (need == 0 || need > pl.c2t_bytes) return RHOSVD_ERR_WORKSPACE;
        rc = rhosvd_c2t(&X, opts, &tk, ws + pl.o_c2t, pl.c2t_bytes, stream);
        if (rc) return rc;
        rhosvd_info info;
        if (cudaMemcpyAsync(&info, info_d, sizeof(info), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
        rhosvd_horner_step rec;
        rec.k = k;
        rec.R_in = (int)Rin;
        for (int l = 0; l < 3; ++l) rec.r[l] = info.r[l];
        rec.R = 0;
        rec.status = info.status;
        if (info.status != RHOSVD_OK) {
            if (steps) steps[step] = rec;
            return info.status;
        }
        rhosvd_tucker_in tin;
        memset(&tin, 0, sizeof(tin));
        for (int l = 0; l < 3; ++l) {
            tin.n[l] = A->n[l];
            tin.r[l] = info.r[l];
            tin.Z[l] = (const double*)tk.Z[l];
            tin.ldz[l] = A->n[l];
        }
        tin.beta = (const double*)tk.beta;
        rc = rhosvd_t2c(&tin, eps_t2c, R_max, U_out, ldu, xi_out, ints_d, nullptr, ints_d + 1, ws + pl.o_t2c,
                        pl.t2c_bytes, stream);
        if (rc) return rc;
        int h[2];
        if (cudaMemcpyAsync(h, ints_d, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
        rec.R = h[0];
        rec.status = h[1];
        if (steps) steps[step] = rec;
        if (h[1] != RHOSVD_OK) return h[1];
        RY = h[0];
    }
    *R_out = RY;
    return RHOSVD_OK;
}
