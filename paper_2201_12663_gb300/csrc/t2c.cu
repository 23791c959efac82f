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

// One-sided Jacobi (Hestenes) on the slice B_m (r1 x r2, column-major in shared memory): each
// pair of columns (a, b) is rotated so that a^T b = 0, t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// zeta = (b^T b - a^T a) / (2 a^T b), until every pair is orthogonal to 1e-14 of ||a|| ||b|| (or
// T2C_SWEEPS sweeps); the columns end as u_k sigma_k.  Pairs by the round-robin (circle)
// schedule over r2 rounded up to even positions (position 0 fixed, the others rotated by the
// round), a warp per pair, a block barrier per round.  Then sigma_k = ||column k||, ranked
// descending (ties to the smaller index), p_m = #{sigma > delta}; the kept u_k = column / sigma_k
// go to uws (r1 x r2 per slice, ranked order) and every sigma to sws (r2 per slice).
__global__ void __launch_bounds__(T2C_THREADS) k_t2c_slice(T2cDims d, const double* delta, double* uws, double* sws,
                                                         int* p_out)
{
    const int m = blockIdx.x;
    const int r1 = d.r[0], r2 = d.r[1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = T2C_THREADS / 32;
    extern __shared__ double t2c_smem[];
    double* Bs = t2c_smem;                               // r1 x r2
    double* sg = Bs + (size_t)r1 * r2;                   // r2
    int* rk = reinterpret_cast<int*>(sg + r2);           // r2
    __shared__ int s_rot, s_p;
    const double* Bg = d.beta + (long long)m * r1 * r2;
    for (int e = tid; e < r1 * r2; e += T2C_THREADS) Bs[e] = Bg[e];
    if (tid == 0) s_p = 0;
    __syncthreads();
    const int np = (r2 + 1) & ~1;
    for (int sweep = 0; sweep < T2C_SWEEPS && np >= 2; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int t = 0; t < np - 1; ++t) {
            for (int pp = warp; pp < np / 2; pp += NW) {
                const int q2 = np - 1 - pp;
                const int a = pp == 0 ? 0 : 1 + (pp - 1 + t) % (np - 1);
                const int b = 1 + (q2 - 1 + t) % (np - 1);
                if (a >= r2 || b >= r2) continue;                   // the padding position
                double* ca = Bs + (size_t)a * r1;
                double* cb = Bs + (size_t)b * r1;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = lane; i < r1; i += 32) {
                    const double x = ca[i], y = cb[i];
                    al = fma(x, x, al);
                    be = fma(y, y, be);
                    ga = fma(x, y, ga);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                }
                double c = 1.0, sn = 0.0;
                int rot = 0;
                if (lane == 0 && ga != 0.0 && fabs(ga) > 1e-14 * sqrt(al * be)) {
                    const double zeta = (be - al) / (2.0 * ga);
                    const double az = fabs(zeta);
                    const double root = az > 1e100 ? az : sqrt(fma(zeta, zeta, 1.0));
                    const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (az + root);
                    c = 1.0 / sqrt(fma(tt, tt, 1.0));
                    sn = c * tt;
                    rot = 1;
                }
                rot = __shfl_sync(0xffffffffu, rot, 0);
                if (rot) {
                    c = __shfl_sync(0xffffffffu, c, 0);
                    sn = __shfl_sync(0xffffffffu, sn, 0);
                    for (int i = lane; i < r1; i += 32) {
                        const double x = ca[i], y = cb[i];
                        ca[i] = fma(c, x, -sn * y);
                        cb[i] = fma(sn, x, c * y);
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
    // singular values, their descending ranks, the count above delta
    const double dl = delta[0];
    for (int k = warp; k < r2; k += NW) {
        const double* ck = Bs + (size_t)k * r1;
        double ss = 0.0;
        for (int i = lane; i < r1; i += 32) ss = fma(ck[i], ck[i], ss);
        ss = warp_sum(ss);
        if (lane == 0) sg[k] = sqrt(ss);
    }
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
    for (int k = warp; k < r2; k += NW) {
        if (rk[k] >= p) continue;
        const double inv = 1.0 / sg[k];
        const double* ck = Bs + (size_t)k * r1;
        double* uk = uws + ((long long)m * r2 + rk[k]) * r1;
        for (int i = lane; i < r1; i += 32) uk[i] = ck[i] * inv;
    }
    if (tid == 0) p_out[m] = p;
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
    size_t o_delta, o_p, o_offs, o_sws, o_uws, total;
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
    const size_t smem = sizeof(double) * ((size_t)r1 * r2 + r2) + sizeof(int) * r2;
    static bool attr = false;
    if (!attr) {
        const size_t smax = sizeof(double) * ((size_t)RHOSVD_T2C_SLICE_MAX + rh::KMAX_T2C_R) + sizeof(int) * rh::KMAX_T2C_R;
        if (cudaFuncSetAttribute(rh::k_t2c_slice, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
        attr = true;
    }
    rh::k_t2c_slice<<<r3, rh::T2C_THREADS, smem, st>>>(d, delta, uws, sws, p);
    rh::count_launch();
    rh::k_t2c_offsets<<<1, 32, 0, st>>>(p, r3, R_max, offs, R_out, status);
    rh::count_launch();
    if (R_max > 0) {
        rh::k_t2c_factors<<<dim3(r2, r3), rh::T2C_THREADS, 0, st>>>(d, uws, sws, p, offs, status, xi);
        rh::count_launch();
    }
    return cudaGetLastError() == cudaSuccess ? RHOSVD_OK : RHOSVD_ERR_CUDA;
}
