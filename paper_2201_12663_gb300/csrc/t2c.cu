// t2c.cu -- the Tucker-to-canonical transform (T2C) of a Tucker tensor (Z1, Z2, Z3, beta), the
// paper's slice-SVD reduction of the core's canonical rank (Sec. 2.4, Remark rem_can_red):
//   beta = sum_m B_m (x) z_m, B_m = beta(:, :, m)                              (eq. T2C_slice)
//   B_m ~ sum_{k <= p_m} sigma_k u_k v_k^T, the singular values above delta    (eq. T2C_SVD)
//   A_R = sum_m sum_k sigma_k (Z1 u_k) (x) (Z2 v_k) (x) Z3(:, m)               (eq. beta_R)
// with delta = eps ||beta||_F / (r3 sqrt(min(r1, r2))), so ||beta - beta_R|| <= eps ||beta||.
// Kernels: the norm and threshold (one block, deterministic); the slice SVDs (one block per
// slice, one-sided Jacobi on the slice held in shared memory); the output offsets (one block);
// the canonical factors (one block per kept singular triple).
#include "internal.cuh"
#include <float.h>

namespace rh {

namespace {

constexpr int T2C_THREADS = 256;
constexpr int T2C_SWEEPS = 40;                 // Jacobi sweeps at most (converges in ~8-12)
constexpr int KMAX_T2C_R = 1024;               // largest r1, r2 of a core

struct T2cDims {
    int n[3], r[3], ldz[3], ldu[3];
    const double* Z[3];
    double* U[3];
    const double* beta;
    double eps;
    int R_max;
};

// ||beta||_F and delta (one block of 1024 threads, fixed order)
__global__ void k_t2c_norm(T2cDims d, double* delta)
{
    __shared__ double red[32];
    const long long total = (long long)d.r[0] * d.r[1] * d.r[2];
    double s = 0.0;
    for (long long e = threadIdx.x; e < total; e += blockDim.x) s = fma(d.beta[e], d.beta[e], s);
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        const int rmin = d.r[0] < d.r[1] ? d.r[0] : d.r[1];
        delta[0] = d.eps * sqrt(s) / ((double)d.r[2] * sqrt((double)rmin));
    }
}

// SVD of the slice B_m (r1 x r2, column-major in shared memory) by preconditioned one-sided
// Jacobi: a Householder QR with column pivoting B P = Q R (in place), then rotations of pairs of
// rows of R (a^T b = 0 with t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (b^T b - a^T a) /
// (2 a^T b)) until every pair is orthogonal to 64 r1 u of ||a|| ||b|| (or T2C_SWEEPS sweeps; the
// count is written to sweeps[m]).  The pivoting grades R's rows, so few sweeps are needed (about
// 28 without it on the bench's core slices).  The rows end as sigma_k times the right singular
// vectors of B P.  Pairs by the round-robin (circle) schedule over q = min(r1, r2) rounded up to
// even positions, a warp per pair, a block barrier per round.  Then sigma_k = ||row k||, ranked
// descending (ties to the smaller index), p_m = #{sigma > delta}; the kept left vectors
// u_k = B v_k / sigma_k (v_k = P row_k / sigma_k, from the slice in global memory) go to uws
// (r1 x r2 per slice, ranked order) and every sigma to sws (r2 per slice).
__global__ void __launch_bounds__(T2C_THREADS) k_t2c_slice(T2cDims d, const double* delta, double* uws, double* sws,
                                                         int* p_out, int* sweeps)
{
    const int m = blockIdx.x;
    const int r1 = d.r[0], r2 = d.r[1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = T2C_THREADS / 32;
    extern __shared__ double t2c_smem[];
    double* Bs = t2c_smem;                               // r1 x r2
    double* sg = Bs + (size_t)r1 * r2;                   // r2
    int* rk = reinterpret_cast<int*>(sg + r2);           // r2
    int* perm = rk + r2;                                 // r2: the column pivoting
    __shared__ int s_rot, s_p;
    const double* Bg = d.beta + (long long)m * r1 * r2;
    double f2 = 0.0;
    for (int e = tid; e < r1 * r2; e += T2C_THREADS) {
        const double x = Bg[e];
        Bs[e] = x;
        f2 = fma(x, x, f2);
    }
    if (tid == 0) s_p = 0;
    __shared__ double red[T2C_THREADS / 32];
    f2 = block_sum(f2, red);
    // convergence: |a^T b| <= tol ||a|| ||b||, tol a few times r1 u (below that the rounding of
    // the dot products decides).  A pair with a column below 1e-6 delta (or 1e-17 ||B_m||) is not
    // rotated: such a column moves no singular value above delta by more than ~1e-12 delta,
    // and noise-level columns would otherwise keep rotating among themselves
    const double tol = 64.0 * r1 * DBL_EPSILON;
    const double dl0 = delta[0];
    const double tiny = fmax(1e-34 * f2, 1e-12 * dl0 * dl0);
    // ---- QR with column pivoting (Householder, in place): B P = Q R; R's rows are graded,
    // which makes the Jacobi sweeps below converge in a few sweeps (preconditioned one-sided
    // Jacobi).  Column norms of the trailing rows are recomputed at every step.
    const int q = r1 < r2 ? r1 : r2;
    __shared__ int s_piv;
    __shared__ double s_tau, s_alpha;
    for (int c = tid; c < r2; c += T2C_THREADS) perm[c] = c;
    __syncthreads();
    for (int j = 0; j < q; ++j) {
        for (int c = j + warp; c < r2; c += NW) {
            const double* cc = Bs + (size_t)c * r1;
            double ss = 0.0;
            for (int i = j + lane; i < r1; i += 32) ss = fma(cc[i], cc[i], ss);
            ss = warp_sum(ss);
            if (lane == 0) sg[c] = ss;
        }
        __syncthreads();
        if (warp == 0) {
            double bv = -1.0;
            int bi = r2;
            for (int c = j + lane; c < r2; c += 32)
                if (sg[c] > bv) { bv = sg[c]; bi = c; }
            for (int o = 16; o > 0; o >>= 1) {
                const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
                const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
                if (v2 > bv || (v2 == bv && i2 < bi)) { bv = v2; bi = i2; }
            }
            if (lane == 0) s_piv = bi;
        }
        __syncthreads();
        const int pv = s_piv;
        if (pv != j) {
            double* cj = Bs + (size_t)j * r1;
            double* cp = Bs + (size_t)pv * r1;
            for (int i = tid; i < r1; i += T2C_THREADS) {
                const double x = cj[i];
                cj[i] = cp[i];
                cp[i] = x;
            }
            if (tid == 0) {
                const int t0 = perm[j];
                perm[j] = perm[pv];
                perm[pv] = t0;
                const double x = sg[j];
                sg[j] = sg[pv];
                sg[pv] = x;
            }
        }
        __syncthreads();
        double* cj = Bs + (size_t)j * r1;
        if (tid == 0) {
            const double x0 = cj[j], n2 = sg[j];
            double tau = 0.0, alpha = x0;
            if (n2 > 0.0) {
                const double xn = sqrt(n2);
                alpha = x0 >= 0.0 ? -xn : xn;
                const double v0 = x0 - alpha;
                tau = 2.0 / (n2 - x0 * x0 + v0 * v0);
                cj[j] = v0;                          // the reflector v = x - alpha e_1, in place
            }
            s_tau = tau;
            s_alpha = alpha;
        }
        __syncthreads();
        const double tau = s_tau;
        if (tau != 0.0) {
            for (int c = j + 1 + warp; c < r2; c += NW) {
                double* cc = Bs + (size_t)c * r1;
                double w = 0.0;
                for (int i = j + lane; i < r1; i += 32) w = fma(cj[i], cc[i], w);
                w = warp_sum(w) * tau;
                for (int i = j + lane; i < r1; i += 32) cc[i] = fma(-w, cj[i], cc[i]);
            }
        }
        __syncthreads();
        if (tid == 0) cj[j] = s_alpha;               // R(j, j)
        for (int i = j + 1 + tid; i < r1; i += T2C_THREADS) cj[i] = 0.0;
        __syncthreads();
    }
    // ---- one-sided Jacobi on the q rows of R (row i: entries (i, c) at Bs[i + r1 c], c < r2):
    // rotate row pairs until orthogonal; the rows end as sigma_k times the right singular
    // vectors of B P
    const int np = (q + 1) & ~1;
    int nsw = 0;
    for (int sweep = 0; sweep < T2C_SWEEPS && np >= 2; ++sweep) {
        nsw = sweep + 1;
        if (tid == 0) s_rot = 0;
        // row norms, recomputed each sweep and updated by the rotations within it
        // (a'^T a' = a^T a - t a^T b, b'^T b' = b^T b + t a^T b): one dot product a pair
        for (int k = warp; k < q; k += NW) {
            double ss = 0.0;
            for (int c = lane; c < r2; c += 32) {
                const double x = Bs[k + (size_t)r1 * c];
                ss = fma(x, x, ss);
            }
            ss = warp_sum(ss);
            if (lane == 0) sg[k] = ss;
        }
        __syncthreads();
        for (int t = 0; t < np - 1; ++t) {
            for (int pp = warp; pp < np / 2; pp += NW) {
                const int q2 = np - 1 - pp;
                const int a = pp == 0 ? 0 : 1 + (pp - 1 + t) % (np - 1);
                const int b = 1 + (q2 - 1 + t) % (np - 1);
                if (a >= q || b >= q) continue;                    // the padding position
                const double al = sg[a], be = sg[b];
                double ga = 0.0;
                for (int c = lane; c < r2; c += 32) ga = fma(Bs[a + (size_t)r1 * c], Bs[b + (size_t)r1 * c], ga);
                ga = warp_sum(ga);
                double cs = 1.0, sn = 0.0;
                int rot = 0;
                if (lane == 0 && ga != 0.0 && al > tiny && be > tiny && fabs(ga) > tol * sqrt(al * be)) {
                    // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) = sign(d h) |h| / (|d| + sqrt(d^2 + h^2))
                    // with h = 2 a^T b, d = b^T b - a^T a: one reciprocal square root and one
                    // reciprocal on the short-latency helpers (few FP64 instructions)
                    const double h = 2.0 * ga, dd = be - al;
                    const double qq = fma(dd, dd, h * h);
                    const double root = qq * fast_rsqrt(qq);
                    const double tt = ((dd >= 0.0) == (h >= 0.0) ? fabs(h) : -fabs(h)) * fast_rcp(fabs(dd) + root);
                    cs = fast_rsqrt(fma(tt, tt, 1.0));
                    sn = cs * tt;
                    rot = 1;
                    sg[a] = fma(-tt, ga, al);
                    sg[b] = fma(tt, ga, be);
                }
                rot = __shfl_sync(0xffffffffu, rot, 0);
                if (rot) {
                    cs = __shfl_sync(0xffffffffu, cs, 0);
                    sn = __shfl_sync(0xffffffffu, sn, 0);
                    for (int c = lane; c < r2; c += 32) {
                        double* xa = Bs + a + (size_t)r1 * c;
                        double* xb = Bs + b + (size_t)r1 * c;
                        const double x = *xa, y = *xb;
                        *xa = fma(cs, x, -sn * y);
                        *xb = fma(sn, x, cs * y);
                    }
                    if (lane == 0) s_rot = 1;
                }
            }
            __syncthreads();
        }
        const int any = s_rot;
        __syncthreads();                                  // every thread has read s_rot
        if (!any) break;
    }
    // singular values (row norms), their descending ranks, the count above delta; a value at or
    // below the slice's FP64 resolution q u ||B_m||_F counts as zero even for delta = 0 (its left
    // vector B v / sigma would be rounding noise, and re-orthonormalising noise leaves U_p
    // non-orthonormal)
    const double dl = fmax(delta[0], (double)q * DBL_EPSILON * sqrt(f2));
    for (int k = warp; k < q; k += NW) {
        double ss = 0.0;
        for (int c = lane; c < r2; c += 32) {
            const double x = Bs[k + (size_t)r1 * c];
            ss = fma(x, x, ss);
        }
        ss = warp_sum(ss);
        if (lane == 0) sg[k] = sqrt(ss);
    }
    for (int k = q + tid; k < r2; k += T2C_THREADS) sg[k] = 0.0;   // B has at most q nonzero values
    __syncthreads();
    for (int k = tid; k < r2; k += T2C_THREADS) {
        const double v = sg[k];
        int c = 0;
        for (int j = 0; j < r2; ++j) c += (sg[j] > v || (sg[j] == v && j < k)) ? 1 : 0;
        rk[k] = c;
        if (v > dl) atomicAdd(&s_p, 1);
    }
    __syncthreads();
    const int p = s_p;
    for (int k = tid; k < r2; k += T2C_THREADS) sws[(long long)m * r2 + rk[k]] = sg[k];
    // left vectors u = B v / sigma with v = P row / sigma: u = sum_c B(:, perm[c]) row(c) / sigma^2,
    // from the slice as it came in (global memory)
    for (int k = warp; k < q; k += NW) {
        if (rk[k] >= p) continue;
        const double inv2 = 1.0 / (sg[k] * sg[k]);
        double* uk = uws + ((long long)m * r2 + rk[k]) * r1;
        for (int i = lane; i < r1; i += 32) {
            double acc = 0.0;
            for (int c = 0; c < r2; ++c) acc = fma(Bg[i + (long long)r1 * perm[c]], Bs[k + (size_t)r1 * c], acc);
            uk[i] = acc * inv2;
        }
    }
    // Re-orthonormalise the kept u in descending order (classical Gram-Schmidt, two passes).
    // u = B v / sigma carries an error in v along a larger singular direction j multiplied by
    // sigma_j / sigma_k, but that error lies in the span of the larger kept vectors, which the
    // projection removes; beta_R = U_p U_p^T B_m then only needs U_p to span the right space.
    __syncthreads();                                  // uws of this slice written by the block
    double* Us = Bs;                                  // p x r1, u_k at Us + k r1 (Bs is free now)
    const double* ug = uws + (long long)m * r2 * r1;
    for (int e = tid; e < p * r1; e += T2C_THREADS) Us[e] = ug[e];
    __syncthreads();
    __shared__ double red2[T2C_THREADS / 32];
    for (int k = 0; k < p; ++k) {
        double* uk = Us + (size_t)k * r1;
        for (int pass = 0; pass < 2 && k > 0; ++pass) {
            for (int j = warp; j < k; j += NW) {
                const double* uj = Us + (size_t)j * r1;
                double dd = 0.0;
                for (int i = lane; i < r1; i += 32) dd = fma(uj[i], uk[i], dd);
                dd = warp_sum(dd);
                if (lane == 0) sg[j] = dd;
            }
            __syncthreads();
            for (int i = tid; i < r1; i += T2C_THREADS) {
                double acc = 0.0;
                for (int j = 0; j < k; ++j) acc = fma(sg[j], Us[(size_t)j * r1 + i], acc);
                uk[i] -= acc;
            }
            __syncthreads();
        }
        double nn = 0.0;
        for (int i = tid; i < r1; i += T2C_THREADS) nn = fma(uk[i], uk[i], nn);
        nn = block_sum(nn, red2);
        const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
        for (int i = tid; i < r1; i += T2C_THREADS) uk[i] *= inv;
        __syncthreads();
    }
    double* uw = uws + (long long)m * r2 * r1;
    for (int e = tid; e < p * r1; e += T2C_THREADS) uw[e] = Us[e];
    if (tid == 0) {
        p_out[m] = p;
        sweeps[m] = nsw;
    }
}

// Exclusive offsets of the kept triples per slice, the total rank R, and the capacity check
// (one block; R > R_max sets RHOSVD_ERR_RANK_OVERFLOW and nothing is written by k_t2c_factors).
__global__ void k_t2c_offsets(const int* p, int r3, int R_max, int* offs, int* R_out, int* status)
{
    if (threadIdx.x != 0) return;
    int o = 0;
    for (int m = 0; m < r3; ++m) {
        offs[m] = o;
        o += p[m];
    }
    R_out[0] = o;
    status[0] = o > R_max ? RHOSVD_ERR_RANK_OVERFLOW : RHOSVD_OK;
}

// Column o = offs[m] + k of the canonical factors for slice m, triple k: xi = sigma_k,
// U1 = Z1 u_k, U2 = Z2 v_k with v_k = B_m^T u_k / sigma_k, U3 = Z3(:, m).
// grid (r2, r3), block T2C_THREADS; blocks with k >= p_m exit.
__global__ void __launch_bounds__(T2C_THREADS) k_t2c_factors(T2cDims d, const double* uws, const double* sws,
                                                           const int* p, const int* offs, const int* status,
                                                           double* xi)
{
    const int k = blockIdx.x, m = blockIdx.y;
    if (status[0] != RHOSVD_OK || k >= p[m]) return;
    const int r1 = d.r[0], r2 = d.r[1];
    const int o = offs[m] + k;
    __shared__ double us[KMAX_T2C_R], vs[KMAX_T2C_R];
    const double* uk = uws + ((long long)m * r2 + k) * r1;
    const double sk = sws[(long long)m * r2 + k];
    for (int i = threadIdx.x; i < r1; i += blockDim.x) us[i] = uk[i];
    __syncthreads();
    const double* Bm = d.beta + (long long)m * r1 * r2;
    const double inv = 1.0 / sk;
    for (int j = threadIdx.x; j < r2; j += blockDim.x) {
        const double* bj = Bm + (long long)j * r1;
        double a0 = 0.0, a1 = 0.0;
        int i = 0;
        for (; i + 1 < r1; i += 2) {
            a0 = fma(bj[i], us[i], a0);
            a1 = fma(bj[i + 1], us[i + 1], a1);
        }
        if (i < r1) a0 = fma(bj[i], us[i], a0);
        vs[j] = (a0 + a1) * inv;
    }
    __syncthreads();
    if (threadIdx.x == 0) xi[o] = sk;
    for (int l = 0; l < 2; ++l) {
        const double* Z = d.Z[l];
        const double* w = l == 0 ? us : vs;
        const int rl = d.r[l], nl = d.n[l];
        double* out = d.U[l] + (long long)o * d.ldu[l];
        for (int x = threadIdx.x; x < nl; x += blockDim.x) {
            double a0 = 0.0, a1 = 0.0;
            int i = 0;
            for (; i + 1 < rl; i += 2) {
                a0 = fma(Z[x + (long long)i * d.ldz[l]], w[i], a0);
                a1 = fma(Z[x + (long long)(i + 1) * d.ldz[l]], w[i + 1], a1);
            }
            if (i < rl) a0 = fma(Z[x + (long long)i * d.ldz[l]], w[i], a0);
            out[x] = a0 + a1;
        }
    }
    {
        const double* z3 = d.Z[2] + (long long)m * d.ldz[2];
        double* out = d.U[2] + (long long)o * d.ldu[2];
        for (int x = threadIdx.x; x < d.n[2]; x += blockDim.x) out[x] = z3[x];
    }
}

__global__ void k_t2c_empty(int* R_out, int* status)
{
    R_out[0] = 0;
    status[0] = RHOSVD_OK;
}

}  // namespace

}  // namespace rh

namespace {

struct T2cPlan {
    size_t o_delta, o_p, o_offs, o_sws, o_uws, o_sweeps, total;
};

int t2c_plan(const rhosvd_tucker_in* t, T2cPlan* pl)
{
    if (!t) return RHOSVD_ERR_INVALID_ARG;
    for (int l = 0; l < 3; ++l)
        if (t->r[l] < 0 || t->n[l] < 0 || t->r[l] > rh::KMAX_T2C_R) return RHOSVD_ERR_INVALID_ARG;
    if ((long long)t->r[0] * t->r[1] > RHOSVD_T2C_SLICE_MAX) return RHOSVD_ERR_INVALID_ARG;
    const size_t r1 = (size_t)t->r[0], r2 = (size_t)t->r[1], r3 = (size_t)t->r[2];
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o += (bytes + 255) / 256 * 256; return at; };
    pl->o_delta = take(sizeof(double));
    pl->o_p = take(sizeof(int) * (r3 > 0 ? r3 : 1));
    pl->o_offs = take(sizeof(int) * (r3 > 0 ? r3 : 1));
    pl->o_sws = take(sizeof(double) * (r2 * r3 > 0 ? r2 * r3 : 1));
    pl->o_uws = take(sizeof(double) * (r1 * r2 * r3 > 0 ? r1 * r2 * r3 : 1));
    pl->o_sweeps = take(sizeof(int) * (r3 > 0 ? r3 : 1));
    pl->total = o;
    return 0;
}

}  // namespace

extern "C" size_t rhosvd_t2c_workspace_size(const rhosvd_tucker_in* t)
{
    T2cPlan pl;
    return t2c_plan(t, &pl) == 0 ? pl.total : 0;
}

extern "C" int rhosvd_t2c(const rhosvd_tucker_in* t, double eps, int R_max, double* const U[3], const int ldu[3],
                          double* xi, int* R_out, int* p_out, int* status, void* workspace, size_t bytes,
                          void* stream)
{
    T2cPlan pl;
    int rc = t2c_plan(t, &pl);
    if (rc) return rc;
    if (!(eps >= 0.0) || R_max < 0 || !U || !ldu || !R_out || !status) return RHOSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int r1 = t->r[0], r2 = t->r[1], r3 = t->r[2];
    if (r1 == 0 || r2 == 0 || r3 == 0) {
        rh::k_t2c_empty<<<1, 1, 0, st>>>(R_out, status);
        rh::count_launch();
        return cudaGetLastError() == cudaSuccess ? RHOSVD_OK : RHOSVD_ERR_CUDA;
    }
    if (!t->beta) return RHOSVD_ERR_INVALID_ARG;
    if (!workspace || bytes < pl.total || ((uintptr_t)workspace & 255) != 0) return RHOSVD_ERR_WORKSPACE;
    for (int l = 0; l < 3; ++l) {
        if (!t->Z[l] || t->ldz[l] < t->n[l] || (R_max > 0 && (!U[l] || ldu[l] < t->n[l]))) return RHOSVD_ERR_INVALID_ARG;
    }
    if (R_max > 0 && !xi) return RHOSVD_ERR_INVALID_ARG;
    unsigned char* ws = (unsigned char*)workspace;
    rh::T2cDims d;
    for (int l = 0; l < 3; ++l) {
        d.n[l] = t->n[l];
        d.r[l] = t->r[l];
        d.ldz[l] = t->ldz[l];
        d.ldu[l] = ldu[l];
        d.Z[l] = t->Z[l];
        d.U[l] = U[l];
    }
    d.beta = t->beta;
    d.eps = eps;
    d.R_max = R_max;
    double* delta = (double*)(ws + pl.o_delta);
    int* p = p_out ? p_out : (int*)(ws + pl.o_p);
    int* offs = (int*)(ws + pl.o_offs);
    double* sws = (double*)(ws + pl.o_sws);
    double* uws = (double*)(ws + pl.o_uws);
    rh::k_t2c_norm<<<1, 1024, 0, st>>>(d, delta);
    rh::count_launch();
    const size_t smem = sizeof(double) * ((size_t)r1 * r2 + r2) + sizeof(int) * 2 * r2;
    static bool attr = false;
    if (!attr) {
        const size_t smax = sizeof(double) * ((size_t)RHOSVD_T2C_SLICE_MAX + rh::KMAX_T2C_R) + sizeof(int) * 2 * rh::KMAX_T2C_R;
        if (cudaFuncSetAttribute(rh::k_t2c_slice, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
        attr = true;
    }
    rh::k_t2c_slice<<<r3, rh::T2C_THREADS, smem, st>>>(d, delta, uws, sws, p, (int*)(ws + pl.o_sweeps));
    rh::count_launch();
    rh::k_t2c_offsets<<<1, 32, 0, st>>>(p, r3, R_max, offs, R_out, status);
    rh::count_launch();
    if (R_max > 0) {
        rh::k_t2c_factors<<<dim3(r2, r3), rh::T2C_THREADS, 0, st>>>(d, uws, sws, p, offs, status, xi);
        rh::count_launch();
    }
    return cudaGetLastError() == cudaSuccess ? RHOSVD_OK : RHOSVD_ERR_CUDA;
}
