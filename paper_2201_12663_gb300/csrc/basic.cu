// basic.cu -- streaming kernels: column norms and term normalisation (Sec. 2.1, eq. can_A3),
// canonical Hadamard product and sum (Sec. 3 eq. rho_ten, Lemma 4.2, Sec. 4.3), identity
// basis for the direct mode.
#include "internal.cuh"

namespace rh {

// One warp per column: ||u|| = m * sqrt(sum (u_i 2^-e)^2) with m = 2^e >= max|u_i|, so the
// scaling is exact and squares neither underflow nor overflow.  grid: (ceil(R/8), 3).

__global__ void k_colnorms(NormArgs a)
{
    const int l = blockIdx.y;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= a.R) return;
    const double* u = a.U[l] + (long long)warp * a.ld[l];
    const int n = a.n[l];
    double mx = 0.0;
    for (int i = lane; i < n; i += 32) mx = fmax(mx, fabs(u[i]));
    mx = warp_max(mx);
    double nrm;
    if (mx == 0.0) {
        nrm = 0.0;
    } else if (!isfinite(mx)) {
        nrm = mx;                     // Inf (NaN propagates through fmax only if all NaN)
    } else {
        int ex;
        frexp(mx, &ex);               // mx = f 2^ex, f in [0.5, 1)
        // scale by 2^-ex in two exact power-of-two steps (2^-ex alone can overflow when the
        // column is subnormal)
        const int e1 = -ex / 2, e2 = -ex - e1;
        const double sc1 = ldexp(1.0, e1), sc2 = ldexp(1.0, e2);
        double s = 0.0;
        bool bad = false;
        for (int i = lane; i < n; i += 32) {
            const double x = u[i];
            if (x != x) bad = true;
            const double t = (x * sc1) * sc2;
            s = fma(t, t, s);
        }
        s = warp_sum(s);
        bad = __any_sync(0xffffffffu, bad);
        nrm = bad ? NAN : ldexp(sqrt(s), ex);
    }
    if (lane == 0) a.norms[(long long)l * a.R + warp] = nrm;
}

// Per term: keep iff all three norms are finite and nonzero (keep[nu] = 1 or 0), weight
// xi' = xi prod_l ||u_l|| (0 for a dropped term).  Non-finite data sets NONFINITE.
__global__ void k_terms(const double* norms, const double* xi, int R, double* keepf, double* xin,
                        double* xi_user, rhosvd_info* info)
{
    for (int nu = blockIdx.x * blockDim.x + threadIdx.x; nu < R; nu += gridDim.x * blockDim.x) {
        const double d0 = norms[nu], d1 = norms[R + nu], d2 = norms[2 * R + nu];
        const double x = xi[nu];
        const bool fin = isfinite(d0) && isfinite(d1) && isfinite(d2) && isfinite(x);
        if (!fin) set_status(info, RHOSVD_ERR_NONFINITE);
        const bool keep = fin && d0 > 0.0 && d1 > 0.0 && d2 > 0.0;
        keepf[nu] = keep ? 1.0 : 0.0;
        const double w = keep ? x * d0 * d1 * d2 : 0.0;
        xin[nu] = w;
        if (xi_user) xi_user[nu] = w;
    }
}

// Normalised copy of the side matrices (Sec. 2.1): Un(:, nu) = u_nu / ||u_nu|| for kept
// terms (to about one ulp), zero columns for dropped terms; nn2 = ||Un(:, nu)||^2 as stored.  One warp per column, grid (ceil(R/8), 3).
__global__ void k_normalize(NormArgs a, const double* keepf, double* Un, long long ustride, double* nn2)
{
    const int l = blockIdx.y;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= a.R) return;
    const int n = a.n[l];
    const double* u = a.U[l] + (long long)warp * a.ld[l];
    double* dst = Un + l * ustride + (long long)warp * n;
    const bool keep = keepf[warp] != 0.0;
    const double d = a.norms[(long long)l * a.R + warp];
    // u / d as (u * (2^e1 / f)) * 2^e2 with d = f 2^e, f in [0.5, 1), e1 + e2 = -e: no overflow
    // for any finite d > 0 (|u| <= d), one FP64 division per column instead of per entry, and
    // within 1.5 ulp of the quotient
    double s1 = 0.0, s2 = 0.0;
    if (keep) {
        int e;
        const double f = frexp(d, &e);
        const int e1 = -e / 2, e2 = -e - e1;
        s1 = ldexp(1.0 / f, e1);
        s2 = ldexp(1.0, e2);
    }
    double s = 0.0;
    for (int i = lane; i < n; i += 32) {
        const double v = (u[i] * s1) * s2;
        dst[i] = v;
        s = fma(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) nn2[(long long)l * a.R + warp] = s;
}

// Deterministic single-block sums: kept terms, ||xi'||^2 and ||U_l normalised||_F^2.
__global__ void k_term_totals(const double* nn2, const double* keepf, const double* xin, int R,
                              double* total, rhosvd_info* info)
{
    __shared__ double red[32];
    double t0 = 0.0, t1 = 0.0, t2 = 0.0, x2 = 0.0, cnt = 0.0;
    for (int nu = threadIdx.x; nu < R; nu += blockDim.x) {
        t0 += nn2[nu];
        t1 += nn2[R + nu];
        t2 += nn2[2 * R + nu];
        x2 += xin[nu] * xin[nu];
        cnt += keepf[nu];
    }
    t0 = block_sum(t0, red);
    t1 = block_sum(t1, red);
    t2 = block_sum(t2, red);
    x2 = block_sum(x2, red);
    cnt = block_sum(cnt, red);
    if (threadIdx.x == 0) {
        total[0] = t0;
        total[1] = t1;
        total[2] = t2;
        info->kept = (int)cnt;
        info->xi_norm = sqrt(x2);
    }
}

// Identity basis Q = I_n (n x n, ld n) for the direct mode of each listed mode.
__global__ void k_identity(double* Q, int n, int ld)
{
    const long long total = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        Q[(long long)j * ld + i] = (i == j) ? 1.0 : 0.0;
    }
}


// ---------------------------------------------------------------- rank growth operations

// C(:, i + Ra j) = A(:, i) .* B(:, j); grid (column blocks, 3 modes); one warp per column.
__global__ void k_hadamard(HadArgs a)
{
    const int l = blockIdx.y;
    const long long R = (long long)a.Ra * a.Rb;
    const int lane = threadIdx.x & 31;
    const int n = a.n[l];
    for (long long nu = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; nu < R;
         nu += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int i = (int)(nu % a.Ra), j = (int)(nu / a.Ra);
        const double* ca = a.A[l] + (long long)i * a.lda[l];
        const double* cb = a.B[l] + (long long)j * a.ldb[l];
        double* cc = a.C[l] + nu * a.ldc[l];
        for (int x = lane; x < n; x += 32) cc[x] = ca[x] * cb[x];
        if (l == 0 && lane == 0) a.xc[nu] = a.xa[i] * a.xb[j];
    }
}


__global__ void k_cpsum(SumArgs a)
{
    const int l = blockIdx.y;
    const int R = a.Ra + a.Rb;
    const int lane = threadIdx.x & 31;
    const int n = a.n[l];
    for (long long nu = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; nu < R;
         nu += ((long long)gridDim.x * blockDim.x) >> 5) {
        const bool fromA = nu < a.Ra;
        const double* src = fromA ? a.A[l] + nu * a.lda[l] : a.B[l] + (nu - a.Ra) * a.ldb[l];
        double* dst = a.C[l] + nu * a.ldc[l];
        for (int x = lane; x < n; x += 32) dst[x] = src[x];
        if (l == 0 && lane == 0) a.xc[nu] = fromA ? a.alpha * a.xa[nu] : a.beta * a.xb[nu - a.Ra];
    }
}


// dst_l(nu, j) = src_l(j, nu): V^(l) (rows j < r_l, ld lds) to nu-contiguous rows (ld ldd = R).
__global__ void k_transpose_v(const double* src, long long sstride, int lds, double* dst, long long dstride, int ldd,
                              int R, const int* dr, int mode0)
{
    const int l = mode0 + blockIdx.y;
    const int r = dr[l];
    const double* S = src + l * sstride;
    double* D = dst + l * dstride;
    const long long total = (long long)R * r;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int nu = (int)(e % R), j = (int)(e / R);
        D[(long long)j * ldd + nu] = S[(long long)nu * lds + j];
    }
}

int launch_transpose_v(const double* src, long long sstride, int lds, double* dst, long long dstride, int ldd, int R,
                       const int* dr, int mode0, int nmodes, cudaStream_t st)
{
    dim3 grid(512, nmodes);
    k_transpose_v<<<grid, 256, 0, st>>>(src, sstride, lds, dst, dstride, ldd, R, dr, mode0);
    RH_CHECK_LAUNCH();
    return 0;
}

__global__ void k_init_state(DevState* s, int k0, int k1, int k2, int m0, int m1, int m2)
{
    s->kin[0] = k0; s->kin[1] = k1; s->kin[2] = k2;
    s->m[0] = m0; s->m[1] = m1; s->m[2] = m2;
}

int launch_colnorms(const NormArgs& a, cudaStream_t st)
{
    if (a.R <= 0) return 0;
    dim3 grid((a.R + 7) / 8, 3);
    k_colnorms<<<grid, 256, 0, st>>>(a);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_terms(const NormArgs& na, const double* xi, double* keepf, double* xin, double* xi_user,
                 rhosvd_info* info, double* Un, long long ustride, double* nn2, double* total, cudaStream_t st)
{
    const int R = na.R;
    if (R > 0) {
        k_terms<<<(R + 255) / 256, 256, 0, st>>>(na.norms, xi, R, keepf, xin, xi_user, info);
        RH_CHECK_LAUNCH();
        dim3 grid((R + 7) / 8, 3);
        k_normalize<<<grid, 256, 0, st>>>(na, keepf, Un, ustride, nn2);
        RH_CHECK_LAUNCH();
    }
    k_term_totals<<<1, 1024, 0, st>>>(nn2, keepf, xin, R, total, info);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_identity(double* Q, int n, int ld, cudaStream_t st)
{
    k_identity<<<(n * n + 255) / 256, 256, 0, st>>>(Q, n, ld);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_init_state(DevState* s, int k0, int k1, int k2, int m0, int m1, int m2, cudaStream_t st)
{
    k_init_state<<<1, 1, 0, st>>>(s, k0, k1, k2, m0, m1, m2);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_hadamard(const HadArgs& a, cudaStream_t st)
{
    const long long R = (long long)a.Ra * a.Rb;
    if (R <= 0) return 0;
    long long blocks = (R + 7) / 8;
    if (blocks > 4096) blocks = 4096;
    dim3 grid((unsigned)blocks, 3);
    k_hadamard<<<grid, 256, 0, st>>>(a);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_cpsum(const SumArgs& a, cudaStream_t st)
{
    const long long R = (long long)a.Ra + a.Rb;
    if (R <= 0) return 0;
    long long blocks = (R + 7) / 8;
    if (blocks > 4096) blocks = 4096;
    dim3 grid((unsigned)blocks, 3);
    k_cpsum<<<grid, 256, 0, st>>>(a);
    RH_CHECK_LAUNCH();
    return 0;
}

}  // namespace rh
