// smallla.cu -- small dense FP64 linear algebra on k x k (k <= RHOSVD_K_MAX) matrices:
//   * the triangular inverse that turns Y into an orthonormal basis (CholeskyQR with
//     pivoting, three passes; the pivoted Cholesky itself and the Householder reduction of
//     M = B B^T to tridiagonal form run on a thread-block cluster per mode, cluster.cu);
//   * eigenvalues of the tridiagonal from an LDL^T representation of T + s I by bisection
//     on the differential stationary qd negative count (relative accuracy for the graded,
//     positive spectra a Gram of a normalised side matrix has);
//   * eigenvectors of the wanted (largest r) eigenvalues by twisted factorisation
//     (stationary + progressive qd, twist at min |gamma|), then the Householder
//     back-transformation.
// These give the singular values sigma_k = sqrt(lambda_k(B B^T)) and left singular
// vectors of the side matrix restricted to span(Q) (eq. SVD_Ul, eq. svdr).
#include "internal.cuh"
#include <float.h>
#include <limits.h>

namespace rh {

// ------------------------------------------------------------------ triangular inverse
// Lt^{-1} of the m x m pivoted Cholesky factor (launch_chol), scattered into W (kx x m, ld ldw) so that
// Q = X W = X P Lt^{-T} (the CholeskyQR factor) is one GEMM: W(perm[j], t) = Lt^{-1}(t, j) for
// t >= j, 0 for t < j; rows perm[j], m <= j < kx (columns of X left out) are zero.
// Column j of Lt^{-1} by forward substitution with column axpys: one warp per column, lane l
// holding entries l, l + 32, ...  grid: (ceil(KMAX / 4), nmodes), block 128.
__global__ void k_trinv(ModeMap mm, const double* L, long long lstride, int ldl, const int* perm, int pstride,
                        const int* dkx, const int* dm, double* W, long long wstride, int ldw, const int* near)
{
    const int b = mm.m[blockIdx.y];
    if (near && near[b]) return;          // the Cholesky wrote W itself (near-identity Gram)
    const int m = dm[b], kx = dkx[b];
    L += b * lstride;
    perm += b * pstride;
    W += b * wstride;
    __shared__ double rdiag[KMAX];
    for (int s = threadIdx.x; s < m; s += blockDim.x) rdiag[s] = 1.0 / L[(long long)s * ldl + s];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (j >= kx) return;
    double* Wr = W + perm[j];
    if (j >= m) {
        for (int t = lane; t < m; t += 32) Wr[(long long)t * ldw] = 0.0;
        return;
    }
    for (int t = lane; t < j; t += 32) Wr[(long long)t * ldw] = 0.0;
    constexpr int NR = KMAX / 32;
    double x[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) x[r] = (r * 32 + lane == j) ? 1.0 : 0.0;
    for (int s = j; s < m; ++s) {
        const int rs = s >> 5;
        double xs = 0.0;
#pragma unroll
        for (int r = 0; r < NR; ++r)
            if (r == rs) xs = __shfl_sync(0xffffffffu, x[r], s & 31);
        xs *= rdiag[s];
        if (lane == 0) Wr[(long long)s * ldw] = xs;
        const double* Lc = L + (long long)s * ldl;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int i = r * 32 + lane;
            if (r >= rs && i > s && i < m) x[r] = fma(-Lc[i], xs, x[r]);
        }
    }
}

// ------------------------------------------------------------------ deflation sketch
// T(j, c) = sum_x Q(x, j) Y(x, c) for j < m, c < k2: block (c, group of 8 j, mode), warp per
// j, lanes over x.
__global__ void k_deflate_proj(ModeMap mm, const double* Q, const double* Y, long long nk, DeflDims d, double* T,
                               long long tstride)
{
    const int b = mm.m[blockIdx.z];
    const int c = blockIdx.x;
    const int n = sel3(d.n, b), m = d.dm[b];
    const double* y = Y + b * nk + (long long)c * n;
    const double* q = Q + b * nk;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
        const int j = blockIdx.y * 8 + warp;
        if (j >= m) return;
        const double* qj = q + (long long)j * n;
        double s = 0.0;
        for (int x = lane; x < n; x += 32) s = fma(qj[x], y[x], s);
        s = warp_sum(s);
        if (lane == 0) T[b * tstride + (long long)c * KMAX + j] = s;
    }
}

// Y(x, c) -= sum_{j < m} Q(x, j) T(j, c): thread per (x, c).  grid (ceil(n/256), k2, modes).
__global__ void k_deflate_sub(ModeMap mm, const double* Q, double* Y, long long nk, DeflDims d, const double* T,
                              long long tstride)
{
    const int b = mm.m[blockIdx.z];
    const int c = blockIdx.y;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sel3(d.n, b), m = d.dm[b];
    if (x >= n) return;
    const double* q = Q + b * nk + x;
    const double* t = T + b * tstride + (long long)c * KMAX;
    double s0 = 0.0, s1 = 0.0;
    int j = 0;
    for (; j + 1 < m; j += 2) {
        s0 = fma(q[(long long)j * n], t[j], s0);
        s1 = fma(q[(long long)(j + 1) * n], t[j + 1], s1);
    }
    if (j < m) s0 = fma(q[(long long)j * n], t[j], s0);
    Y[b * nk + (long long)c * n + x] -= s0 + s1;
}

int launch_deflate(ModeMap mm, const double* Q, double* Y, long long nk, const int n[3], const int* dm, int k2,
                   double* T, long long tstride, int nb, int nmax, cudaStream_t st)
{
    if (nb <= 0 || k2 <= 0) return 0;
    DeflDims d;
    for (int l = 0; l < 3; ++l) d.n[l] = n[l];
    d.dm = dm;
    k_deflate_proj<<<dim3(k2, KMAX / 8, nb), 256, 0, st>>>(mm, Q, Y, nk, d, T, tstride);
    RH_CHECK_LAUNCH();
    k_deflate_sub<<<dim3((nmax + 255) / 256, k2, nb), 256, 0, st>>>(mm, Q, Y, nk, d, T, tstride);
    RH_CHECK_LAUNCH();
    return 0;
}

// Q(:, m + j) = Q2(:, j) for j < m2.  grid (ceil(n/256), k2, modes).
__global__ void k_append(ModeMap mm, double* Q, const double* Q2, long long nk, DeflDims d, const int* dm2)
{
    const int b = mm.m[blockIdx.z];
    const int j = blockIdx.y;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sel3(d.n, b), m = d.dm[b];
    if (j >= dm2[b] || x >= n) return;
    Q[b * nk + (long long)(m + j) * n + x] = Q2[b * nk + (long long)j * n + x];
}

__global__ void k_append_count(ModeMap mm, int* dm, const int* dm2, int nb)
{
    if (threadIdx.x < nb) {
        const int b = mm.m[threadIdx.x];
        dm[b] += dm2[b];
    }
}

int launch_append(ModeMap mm, double* Q, const double* Q2, long long nk, const int n[3], int* dm, const int* dm2,
                  int nb, int nmax, int k2, cudaStream_t st)
{
    if (nb <= 0 || k2 <= 0) return 0;
    DeflDims d;
    for (int l = 0; l < 3; ++l) d.n[l] = n[l];
    d.dm = dm;
    k_append<<<dim3((nmax + 255) / 256, k2, nb), 256, 0, st>>>(mm, Q, Q2, nk, d, dm2);
    RH_CHECK_LAUNCH();
    k_append_count<<<1, 32, 0, st>>>(mm, dm, dm2, nb);
    RH_CHECK_LAUNCH();
    return 0;
}

// ------------------------------------------------------------------ eigenvalues
// Number of eigenvalues of L D L^T below x: the signs of the pivots D+_i of the stationary qd
// transform L D L^T - x I = L+ D+ L+^T (t_0 = -x, D+_i = D_i + t_i, t_{i+1} = t_i W_i / D+_i - x,
// W_i = D_i L_i^2).  Written without division: t_i = N_i / Q_i with Q_0 = 1, N_0 = -x gives
// P_i = D_i Q_i + N_i = D+_i Q_i, Q_{i+1} = P_i, N_{i+1} = N_i W_i - x P_i, and D+_i < 0 exactly
// when P_i and Q_i differ in sign.  Three FP64 operations a step; the sign test and the
// exponent watch run on the integer pipe.  N and Q are rescaled by a power of two (exact) when
// their larger exponent leaves [-400, 400]; both vanishing restarts the recurrence as after a
// split.  A zero pivot needs no special case: Q = 0 makes the next t infinite and the form
// continues with its limit.
__device__ __forceinline__ int negcount(const double* D, const double* W, int k, double x)
{
    double Q = 1.0, N = -x;
    int hq = __double2hiint(Q);
    int c = 0;
    for (int i = 0; i < k; ++i) {
        const double P = fma(D[i], Q, N);
        const int hp = __double2hiint(P);
        c += (int)((unsigned)(hp ^ hq) >> 31);
        N = fma(-x, P, N * W[i]);
        Q = P;
        hq = hp;
        const int ep = (hp >> 20) & 0x7FF, en = (__double2hiint(N) >> 20) & 0x7FF;
        const int em = ep > en ? ep : en;
        if (em > 1023 + 400 || em < 1023 - 400) {
            if (em == 0) {
                Q = 1.0;
                N = -x;
            } else {
                const double sc = __hiloint2double((2046 - em) << 20, 0);   // 2^(1023 - em)
                Q *= sc;
                N *= sc;
            }
            hq = __double2hiint(Q);
        }
    }
    return c;
}

// LDL^T = T + s I with s > 0 multiplied by 4 until every pivot is positive (one warp per
// mode: the norms by all lanes, the recurrence by lane 0).  Writes D, Lo, the shift s and an
// upper bound of the spectrum of L D L^T.
// The pivots come from the leading principal minors of the matrix scaled by sig = 2^-ex
// (||T|| < 2^ex): P_{-1} = 1, P_0 = c_0, P_{i+1} = c_{i+1} P_i - e_i^2 P_{i-1} with c_i = (d_i + s) sig
// and e_i sig in place of e_i, D_i = 2^ex P_i / P_{i-1}.  The serial chain is then one FMA a step
// (the product e_i^2 P_{i-1} is ready a step early) instead of a division; the pair (P_{i-1}, P_i)
// is rescaled by one power of two when P_i leaves [2^-400, 2^400], and the quotients D_i and
// l_i = e_i / D_i are taken afterwards by all lanes.  Rounding-wise a step perturbs c_i and e_i^2
// by a few ulps, as the pivot recurrence D_{i+1} = c_{i+1} - e_i^2 / D_i does.
__global__ void k_ldl(ModeMap mm, const double* d, const double* e, int vstride, const int* dk, double* D,
                      double* Lo, DevState* st)
{
    const int b = mm.m[blockIdx.x];
    const int lane = threadIdx.x & 31;
    const int k = dk[b];
    d += b * vstride;
    e += b * vstride;
    D += b * vstride;
    Lo += b * vstride;
    // the scaled diagonal and squared off-diagonal in shared memory: the recurrence below is one
    // serial chain, and a global load on it would cost an L2 round trip a step
    __shared__ double ds[KMAX], e2[KMAX], pc[KMAX], pq[KMAX];
    double tnorm = 0.0;
    for (int i = lane; i < k; i += 32) {
        const double r = fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < k ? fabs(e[i]) : 0.0);
        tnorm = fmax(tnorm, r);
    }
    tnorm = warp_max(tnorm);
    int ex = 0;
    if (tnorm > 0.0 && tnorm < INFINITY) frexp(tnorm, &ex);
    ex = ex < -1000 ? -1000 : (ex > 1000 ? 1000 : ex);
    const double sig = ldexp(1.0, -ex), isig = ldexp(1.0, ex);
    for (int i = lane; i < k; i += 32) {
        ds[i] = d[i] * sig;
        const double es = i + 1 < k ? e[i] * sig : 0.0;
        e2[i] = es * es;
    }
    __syncwarp();
    __shared__ double s_shift;
    __shared__ int s_valid;
    if (lane == 0) {
        double s = fmax(4.0 * k * DBL_EPSILON * tnorm, DBL_MIN);
        bool ok = false;
        int valid = 0;
        for (int tries = 0; tries < 60 && !ok; ++tries) {
            ok = true;
            const double ss = s * sig;
            double q = 1.0, p = ds[0] + ss;               // P_{i-1}, P_i
            valid = 0;
            for (int i = 0; i < k; ++i) {
                const int ep = (__double2hiint(p) >> 20) & 0x7FF;
                if (ep == 0x7FF) { ok = false; break; }
                if (ep != 0 && (ep > 1023 + 400 || ep < 1023 - 400)) {
                    const double sc = __hiloint2double((2046 - ep) << 20, 0);   // 2^(1023 - ep)
                    p *= sc;
                    q *= sc;
                }
                if (!(p > 0.0) || !(q < INFINITY)) { ok = false; break; }
                pc[i] = p;
                pq[i] = q;
                valid = i + 1;
                if (i + 1 < k) {
                    const double t = -e2[i] * q;
                    const double pn = fma(ds[i + 1] + ss, p, t);
                    q = p;
                    p = pn;
                }
            }
            if (!ok) s *= 4.0;
        }
        if (!ok) st->piv_fail[b] = 1;
        s_shift = s;
        s_valid = valid;
    }
    __syncwarp();
    {
        const int valid = s_valid;
        for (int i = lane; i < k; i += 32) {
            const double Di = i < valid ? (pc[i] / pq[i]) * isig : 1.0;
            D[i] = Di;
            Lo[i] = (i + 1 < k && i < valid) ? e[i] / Di : 0.0;
        }
    }
    __syncwarp();
    const double s = s_shift;
    double hi = 0.0;
    for (int i = lane; i < k; i += 32) {
        const double r = d[i] + s + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < k ? fabs(e[i]) : 0.0);
        hi = fmax(hi, r);
    }
    hi = warp_max(hi);
    if (lane == 0) {
        st->shift[b] = s;
        st->specmax[b] = hi * (1.0 + 8.0 * DBL_EPSILON) + DBL_MIN;
    }
}

// Eigenvalue a (ascending) of L D L^T by multisection: EIG_P lanes per eigenvalue (32 / EIG_P
// eigenvalues a warp), each lane counting at one of EIG_P points inside the current bracket; the
// bracket shrinks to the two neighbouring points around the eigenvalue ((EIG_P + 1)-fold per
// round).  Points are spaced geometrically while hi > 4 lo (relative accuracy across the whole
// spectrum), linearly after.  The bracket starts at [s/2, specmax]: T + s I has no eigenvalue
// below s (1 - k u ||T|| / s).  A count is one serial chain of k steps, two dependent FP64
// operations each, and FP64 latency on this part is long: the cost is the number of rounds, so
// every lane of a warp serves one eigenvalue (EIG_P = 32, about 12 rounds to
// hi - lo <= 2 u hi; 4 points a round took twice as long).  A group that has converged keeps
// its bracket while the warp's other groups finish.
// grid: (ceil(KMAX / (EIG_WARPS * 32 / EIG_P)), nmodes), block: 32 EIG_WARPS threads.
constexpr int EIG_P = 32;
constexpr int EIG_WARPS = 4;

__global__ void k_bisect(ModeMap mm, const double* Dg, const double* Lg, int vstride, const int* dk,
                         double* mu, const DevState* st)
{
    constexpr int PER_WARP = 32 / EIG_P, PER_BLOCK = EIG_WARPS * PER_WARP;
    const int b = mm.m[blockIdx.y];
    const int k = dk[b];
    __shared__ double Dsh[KMAX], Wsh[KMAX];
    if (blockIdx.x * PER_BLOCK >= k) return;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double d = Dg[b * vstride + i];
        const double l = (i + 1 < k) ? Lg[b * vstride + i] : 0.0;
        Dsh[i] = d;
        Wsh[i] = d * l * l;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int grp = lane / EIG_P, j = lane - grp * EIG_P + 1;
    const int a = blockIdx.x * PER_BLOCK + (threadIdx.x >> 5) * PER_WARP + grp;
    const unsigned gbits = EIG_P == 32 ? 0xffffffffu : ((1u << (EIG_P & 31)) - 1u);
    const unsigned gmask = gbits << ((grp * EIG_P) & 31);
    double lo = 0.5 * st->shift[b], hi = st->specmax[b];
    bool done = a >= k;
    for (int round = 0; round < 160; ++round) {
        if (!done && hi - lo <= 2.0 * DBL_EPSILON * hi) done = true;
        if (__all_sync(0xffffffffu, done)) break;
        double x = fma(hi - lo, (double)j * (1.0 / (EIG_P + 1)), lo);
        if (hi > 4.0 * lo) {
            const float lr = log2f((float)(hi / lo));
            const double g = lo * (double)exp2f(lr * (float)j * (1.0f / (EIG_P + 1)));
            if (g > lo && g < hi) x = g;
        }
        const bool below = !done && negcount(Dsh, Wsh, k, x) <= a;     // lambda_a >= x
        const unsigned m = (__ballot_sync(0xffffffffu, below) & gmask) >> ((grp * EIG_P) & 31);
        const unsigned above = ~m & gbits;
        const int f = above ? __ffs(above) - 1 : EIG_P;                // first point above lambda_a
        const int base = grp * EIG_P;
        const double xl = __shfl_sync(0xffffffffu, x, base + (f > 0 ? f - 1 : 0));
        const double xh = __shfl_sync(0xffffffffu, x, base + (f < EIG_P ? f : EIG_P - 1));
        if (!done) {
            if (f > 0) lo = xl;
            if (f < EIG_P) hi = xh;
        }
    }
    if (j == 1 && a < k) mu[b * vstride + a] = 0.5 * (lo + hi);
}

// ------------------------------------------------------------------ rank rule
// Provisional rank from the eigenvalues lambda_j = max(mu_{k-1-j} - s, 0) (descending) of
// B B^T, q = min(k, kept) of them (a side matrix has at most `kept` nonzero singular values):
// r0 = min r with sum_{j >= r} lambda_j <= eps^2 total.  The final rule (k_rank_final) then
// checks rank candidates 0..rhi, rhi = min(q, r0 + margin), with energies computed directly.
__global__ void k_rank_select(RankArgs a)
{
    const int b = threadIdx.x >> 5, lane = threadIdx.x & 31;     // warp b: mode b
    if (b >= 3) return;
    const int k = a.dk[b];
    const double* mu = a.mu + b * a.vstride;
    const double s = a.st->shift[b];
    const int q = min(k, *a.kept);
    if (lane == 0) {
        const double total = a.total[b];
        if (a.st->piv_fail[b]) set_status(a.info, RHOSVD_ERR_NOT_CONVERGED);
        int r0;
        if (total == 0.0 || q == 0 || (a.ranks[b] == 0 && a.eps >= 1.0)) {
            r0 = 0;
        } else if (a.ranks[b] > 0) {
            r0 = min(a.ranks[b], q);
        } else {
            const double thr = a.eps * a.eps * total;
            double tail = 0.0;
            r0 = q;
            while (r0 > 0) {
                const double lam = fmax(mu[k - 1 - (r0 - 1)] - s, 0.0);
                if (tail + lam <= thr) { tail += lam; --r0; } else break;
            }
        }
        int rhi = (a.ranks[b] > 0 || r0 == 0) ? r0 : min(q, r0 + a.margin);
        if (a.ranks[b] == 0 && a.eps >= 1.0) rhi = 0;
        a.st->r0[b] = r0;
        a.st->rhi[b] = rhi;
        a.info->k[b] = k;
        a.info->total[b] = total;
        a.info->direct[b] = a.direct[b];
    }
    for (int j = lane; j < KMAX; j += 32)         // sigma: one square root a lane
        a.sigma[b][j] = (j < q) ? sqrt(fmax(mu[k - 1 - j] - s, 0.0)) : 0.0;
}

// Final eps-rank from directly computed energies (no cancellation):
//   rho^2 = ||U - Z_hi V_hi||_F^2 (residual GEMM partials), c_j = ||V_hi(j,:)||^2,
//   tail(r) = rho^2 + sum_{r <= j < rhi} c_j,  r = min r with tail(r) <= eps^2 total.
// One block per mode.
// Ritz energy partials: cpart[b][ch][j] = sum over nu in chunk ch of V_hi(j, nu)^2, thread j
// (coalesced along j).  grid (nchunk, 3), block KMAX.
__global__ void k_ritz_partial(FinalArgs a)
{
    const int b = blockIdx.y, ch = blockIdx.x, j = threadIdx.x;
    const int rhi = a.st->rhi[b];
    const int clen = (a.R + a.nchunk - 1) / a.nchunk;
    const int nu0 = ch * clen, nu1 = min(a.R, nu0 + clen);
    double e = 0.0;
    if (j < rhi) {
        const double* V = a.V + b * a.vstride + j;
        for (int nu = nu0; nu < nu1; ++nu) {
            const double v = V[(long long)nu * a.ldv];
            e = fma(v, v, e);
        }
    }
    a.cpart[((long long)b * a.nchunk + ch) * KMAX + j] = e;
}

__global__ void k_rank_final(FinalArgs a)
{
    const int b = blockIdx.x;
    const int rhi = a.st->rhi[b];
    __shared__ double c[KMAX];
    __shared__ double red[32];
    const double* part = a.rpart + b * a.rpstride;
    double s = 0.0;
    for (int t = threadIdx.x; t < a.ntiles[b]; t += blockDim.x) s += part[t];
    const double rho2 = block_sum(s, red);
    for (int j = threadIdx.x; j < rhi; j += blockDim.x) {
        const double* cp = a.cpart + (long long)b * a.nchunk * KMAX + j;
        double e = 0.0;
        for (int ch = 0; ch < a.nchunk; ++ch) e += cp[(long long)ch * KMAX];
        c[j] = e;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double total = a.st->total[b];
    // energy at or below the FP64 resolution of the n_l x R side matrix, (n_l u)^2 ||U||_F^2,
    // counts as zero: with eps = 0 (or below n_l u) the rank keeps every resolvable direction
    // and rounding left in the residual is no missed sketch energy
    const double floor_rel = (double)a.n[b] * DBL_EPSILON;
    const double thr = fmax(a.eps * a.eps, floor_rel * floor_rel) * total;
    int r;
    if (a.ranks[b] > 0 || total == 0.0 || (a.ranks[b] == 0 && a.eps >= 1.0)) {
        r = rhi;
    } else {
        double tail = rho2;
        r = rhi;
        if (tail > thr) {
            set_status(a.info, RHOSVD_ERR_SKETCH);
        } else {
            while (r > 0 && tail + c[r - 1] <= thr) { tail += c[r - 1]; --r; }
        }
    }
    const int rn = r;
    if (r > a.r_max) { set_status(a.info, RHOSVD_ERR_RANK_OVERFLOW); r = a.r_max; }
    double tail = rho2;
    for (int j = r; j < rhi; ++j) tail += c[j];
    a.st->r[b] = r;
    a.st->rho2[b] = rho2;
    a.info->r[b] = r;
    a.info->r_needed[b] = rn;
    a.info->resid[b] = rho2;
    a.info->tail[b] = sqrt(tail);
}

// dst_b(i, j) = src_b(i, j) for i < rows_b, j < cols_b (rows/cols from the device or host).
struct CopyArgs {
    const double* src;
    long long sstride;
    int lds[3];
    double* dst[3];
    int ldd[3];
    const int* drows;    // per mode or null
    int hrows[3];
    const int* dcols;    // per mode or null
    int hcols[3];
};

__global__ void k_copy2d(CopyArgs a)
{
    const int b = blockIdx.y;
    const int rows = a.drows ? a.drows[b] : a.hrows[b];
    const int cols = a.dcols ? a.dcols[b] : a.hcols[b];
    const long long total = (long long)rows * cols;
    const double* src = a.src + b * a.sstride;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % rows), j = (int)(e / rows);
        a.dst[b][(long long)j * a.ldd[b] + i] = src[(long long)j * a.lds[b] + i];
    }
}

// ------------------------------------------------------------------ eigenvectors
// Eigenvector of L D L^T for the eigenvalue mu (twisted factorisation):
// stationary qd  L D L^T - mu I = L+ D+ L+^T (top down, s_i), progressive qd
// L D L^T - mu I = U- D- U-^T (bottom up, p_i), gamma_r = s_r + p_r + mu, twist at
// argmin |gamma_r|; z_r = 1, z_i = -L+_i z_{i+1} above, z_{i+1} = -U-_i z_i below.
// One thread per vector; grid (ceil(rmax / 4), nmodes), 4 threads a block.
__global__ void k_eigvecs(ModeMap mm, const double* D, const double* Lo, const double* mu, int vstride, const int* dk,
                          const DevState* st, double* W, long long wstride, int ldw)
{
    const int b = mm.m[blockIdx.y];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;   // descending index
    const int k = dk[b];
    const int r = st->rhi[b];
    if (j >= r || j >= k) return;
    D += b * vstride;
    Lo += b * vstride;
    mu += b * vstride;
    W += b * wstride;
    const double lam = mu[k - 1 - j];
    double Lp[KMAX], Um[KMAX], sv[KMAX], pv[KMAX];
    // stationary
    double sc = -lam;
    for (int i = 0; i + 1 < k; ++i) {
        sv[i] = sc;
        double dp = D[i] + sc;
        if (dp == 0.0) dp = DBL_MIN;
        const double lp = D[i] * Lo[i] / dp;
        Lp[i] = lp;
        sc = lp * Lo[i] * sc - lam;
    }
    sv[k - 1] = sc;
    // progressive
    double pc = D[k - 1] - lam;
    pv[k - 1] = pc;
    for (int i = k - 2; i >= 0; --i) {
        double dm = D[i] * Lo[i] * Lo[i] + pc;
        if (dm == 0.0) dm = DBL_MIN;
        const double t = D[i] / dm;
        Um[i] = Lo[i] * t;
        pc = pc * t - lam;
        pv[i] = pc;
    }
    int tw = 0;
    double gbest = INFINITY;
    for (int i = 0; i < k; ++i) {
        const double g = fabs(sv[i] + pv[i] + lam);
        if (g < gbest) { gbest = g; tw = i; }
    }
    double* z = W + (long long)j * ldw;
    z[tw] = 1.0;
    double nrm2 = 1.0;
    double zc = 1.0;
    for (int i = tw - 1; i >= 0; --i) {
        zc = -Lp[i] * zc;
        z[i] = zc;
        nrm2 += zc * zc;
    }
    zc = 1.0;
    for (int i = tw; i + 1 < k; ++i) {
        zc = -Um[i] * zc;
        z[i + 1] = zc;
        nrm2 += zc * zc;
    }
    const double inv = 1.0 / sqrt(nrm2);
    for (int i = 0; i < k; ++i) z[i] *= inv;
}

// ------------------------------------------------------------------ back-transformation
// y <- H_0 H_1 ... H_{k-3} y for each of the r columns (one warp per column, 4 a block); H_j
// uses the reflector stored in A(j+1:k, j) and tau[j].  The column lives in registers (lane l
// holds entries l, l + 32, ...), and the reflectors are staged in shared memory 16 at a time by
// the whole block, so a reflector costs one warp reduction instead of an L2 round trip.  Reflector
// j is zero in rows 0..j: the 32-row groups entirely above it are skipped (less FP64 work).
// grid: (ceil(KMAX / 4), nmodes), block 128.
constexpr int BT_CH = 16;

__global__ void k_backtransform(ModeMap mm, const double* A, long long astride, int lda, const double* tau, int vstride,
                                const int* dk, const DevState* st, double* W, long long wstride, int ldw)
{
    const int b = mm.m[blockIdx.y];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k = dk[b];
    const int r = st->rhi[b];
    const int v0 = blockIdx.x * 4;
    if (v0 >= r) return;
    A += b * astride;
    tau += b * vstride;
    const int vec = v0 + warp;
    const bool live = vec < r;
    double* y = W + b * wstride + (long long)vec * ldw;
    constexpr int NQ = KMAX / 32;
    const int kp = (k + 31) & ~31;
    double yr[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int i = lane + 32 * q;
        yr[q] = (live && i < k) ? y[i] : 0.0;
    }
    __shared__ double Vs[BT_CH][KMAX];
    __shared__ double ts[BT_CH];
    for (int jhi = k - 3; jhi >= 0; jhi -= BT_CH) {
        const int nc = jhi + 1 < BT_CH ? jhi + 1 : BT_CH;       // reflectors jhi, jhi-1, .. jhi-nc+1
        __syncthreads();                                      // the previous chunk is applied
        for (int idx = tid; idx < nc * kp; idx += blockDim.x) {
            const int c = idx / kp, i = idx - c * kp, j = jhi - c;
            Vs[c][i] = (i > j && i < k) ? A[(long long)j * lda + i] : 0.0;
        }
        if (tid < nc) ts[tid] = tau[jhi - tid];
        __syncthreads();
        if (!live) continue;
        for (int c = 0; c < nc; ++c) {
            const double t = ts[c];
            if (t == 0.0) continue;
            const int q0 = (jhi - c + 1) >> 5;                 // first group holding row j + 1
            double dot = 0.0;
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q >= q0 && 32 * q < kp) dot = fma(Vs[c][lane + 32 * q], yr[q], dot);
            dot = warp_sum(dot) * t;
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q >= q0 && 32 * q < kp) yr[q] = fma(-dot, Vs[c][lane + 32 * q], yr[q]);
        }
    }
    if (live) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int i = lane + 32 * q;
            if (i < k) y[i] = yr[q];
        }
    }
}

// trace of each mode's k x k matrix (before it is overwritten)
__global__ void k_trace(ModeMap mm, const double* A, long long astride, int lda, const int* dk, double* trace)
{
    const int b = mm.m[blockIdx.x];
    const int k = dk[b];
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) s += A[b * astride + (long long)i * lda + i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) trace[b] = s;
}


int launch_chol(ModeMap mm, const double* G, long long gstride, int ldg, const int* dk, int* kx_out, double* L,
                long long lstride, int ldl, int* perm, int pstride, int* dm_out, int* fail, int pivot, double tol, int nb,
                int kbound, double* d0_out, const double* d0_ref, double floor_rel, double* W, long long wstride,
                int ldw, int* near_out, cudaStream_t st)
{
    return launch_chol_cluster(mm, G, gstride, ldg, dk, kx_out, L, lstride, ldl, perm, pstride, dm_out, fail, pivot,
                               tol, nb, kbound, d0_out, d0_ref, floor_rel, W, wstride, ldw, near_out, st);
}

int launch_trinv(ModeMap mm, const double* L, long long lstride, int ldl, const int* perm, int pstride,
                 const int* dkx, const int* dm, double* W, long long wstride, int ldw, const int* near, int nb,
                 cudaStream_t st)
{
    dim3 grid((KMAX + 3) / 4, nb);
    k_trinv<<<grid, 128, 0, st>>>(mm, L, lstride, ldl, perm, pstride, dkx, dm, W, wstride, ldw, near);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_trace(ModeMap mm, const double* A, long long astride, int lda, const int* dk, double* trace, int nb,
                 cudaStream_t st)
{
    k_trace<<<nb, 256, 0, st>>>(mm, A, astride, lda, dk, trace);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_tridiag(ModeMap mm, double* A, long long astride, int lda, const int* dk, double* d, double* e, double* tau,
                   int vstride, int nb, int kbound, cudaStream_t st)
{
    return launch_tridiag_cluster(mm, A, astride, lda, dk, d, e, tau, vstride, nb, kbound, st);
}

int launch_eigvals(ModeMap mm, const double* d, const double* e, int vstride, const int* dk, double* D, double* Lo,
                   double* mu, DevState* s, int nb, cudaStream_t st)
{
    k_ldl<<<nb, 32, 0, st>>>(mm, d, e, vstride, dk, D, Lo, s);
    RH_CHECK_LAUNCH();
    constexpr int per_block = EIG_WARPS * (32 / EIG_P);
    dim3 grid((KMAX + per_block - 1) / per_block, nb);
    k_bisect<<<grid, 32 * EIG_WARPS, 0, st>>>(mm, D, Lo, vstride, dk, mu, s);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_rank(const RankArgs& a, cudaStream_t st)
{
    k_rank_select<<<1, 96, 0, st>>>(a);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_rank_final(const FinalArgs& a, cudaStream_t st)
{
    k_ritz_partial<<<dim3(a.nchunk, 3), KMAX, 0, st>>>(a);
    RH_CHECK_LAUNCH();
    k_rank_final<<<3, 256, 0, st>>>(a);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_copy2d(const double* src, long long sstride, const int lds[3], double* const dst[3], const int ldd[3],
                  const int* drows, const int hrows[3], const int* dcols, const int hcols[3], cudaStream_t st)
{
    CopyArgs a;
    a.src = src;
    a.sstride = sstride;
    for (int l = 0; l < 3; ++l) {
        a.lds[l] = lds[l];
        a.dst[l] = dst[l];
        a.ldd[l] = ldd[l];
        a.hrows[l] = hrows ? hrows[l] : 0;
        a.hcols[l] = hcols ? hcols[l] : 0;
    }
    a.drows = drows;
    a.dcols = dcols;
    dim3 grid(256, 3);
    k_copy2d<<<grid, 256, 0, st>>>(a);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_eigvecs(ModeMap mm, const double* D, const double* Lo, const double* mu, int vstride, const int* dk,
                   const DevState* s, double* W, long long wstride, int ldw, int rmax, int nb, cudaStream_t st)
{
    // 4 vectors a block: each vector is a serial chain, and a warp-wide FP64 instruction costs the
    // SM's FP64 pipe 16 cycles, so the vectors are spread over many SMs rather than packed (three
    // modes of ~150 vectors fill about 120 of the 152 SMs with one 4-lane warp each)
    constexpr int VPB = 4;
    dim3 grid((rmax + VPB - 1) / VPB, nb);
    k_eigvecs<<<grid, VPB, 0, st>>>(mm, D, Lo, mu, vstride, dk, s, W, wstride, ldw);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_backtransform(ModeMap mm, const double* A, long long astride, int lda, const double* tau, int vstride,
                         const int* dk, const DevState* s, double* W, long long wstride, int ldw, int rmax,
                         int nb, cudaStream_t st)
{
    dim3 grid((rmax + 3) / 4, nb);
    k_backtransform<<<grid, 128, 0, st>>>(mm, A, astride, lda, tau, vstride, dk, s, W, wstride, ldw);
    RH_CHECK_LAUNCH();
    return 0;
}

}  // namespace rh
