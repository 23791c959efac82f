// basic.cu -- streaming kernels: column norms and term normalisation (Sec. 2.1, eq. can_A3),
// canonical Hadamard product and sum (Sec. 3 eq. rho_ten, Lemma 4.2, Sec. 4.3), identity
// basis for the direct mode.
#include "internal.cuh"
#include "ozgemm.cuh"

namespace rh {

// One warp per column: max |u_i| by an integer max over the sign-cleared bit patterns (a
// non-negative double orders like its bits; NaN patterns sort above Inf), then
// ||u|| = 2^ex sqrt(sum (u_i 2^-ex)^2) with max |u_i| < 2^ex, so the scaling is exact and the
// squares neither underflow nor overflow.  Writes the norm and max |u_i|.  grid (ceil(R/8), 3).
// Column nu of mode l: the stored column, or (PROD) the entrywise product of the two factor
// columns it stands for, nu = i + Ra j (one FP64 multiply, as rhosvd_cp_hadamard stores it).
template <bool PROD>
struct Col {
    const double* a;
    const double* b;
    __device__ Col(const NormArgs& na, int l, int nu)
    {
        if (PROD) {
            const int i = nu % na.Ra, j = nu / na.Ra;
            a = sel3(na.U, l) + (long long)i * sel3(na.ld, l);
            b = sel3(na.B, l) + (long long)j * sel3(na.ldb, l);
        } else {
            a = sel3(na.U, l) + (long long)nu * sel3(na.ld, l);
            b = nullptr;
        }
    }
    __device__ __forceinline__ double operator[](int x) const { return PROD ? a[x] * b[x] : a[x]; }
};

template <bool PROD>
__global__ void k_colnorms(NormArgs a)
{
    const int l = blockIdx.y;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= a.R) return;
    const Col<PROD> u(a, l, warp);
    const int n = sel3(a.n, l);
    long long mb = 0;
    for (int i = lane; i < n; i += 32) {
        const long long b = __double_as_longlong(u[i]) & 0x7FFFFFFFFFFFFFFFll;
        mb = b > mb ? b : mb;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long b = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = b > mb ? b : mb;
    }
    const double mx = __longlong_as_double(mb);
    double nrm;
    if (mb == 0) {
        nrm = 0.0;
    } else if (mb >= 0x7FF0000000000000ll) {
        nrm = mx;                     // Inf, or NaN when a NaN is present
    } else {
        int ex;
        frexp(mx, &ex);               // mx < 2^ex
        double s = 0.0;
        if (ex > -450 && ex < 450) {
            // squares stay in [2^-902, 2^900): no scaling needed, one FP64 operation an element
            // (terms that would square to subnormals lie below 2^-1022 / max^2 <= 2^-120 of the sum)
            for (int i = lane; i < n; i += 32) {
                const double v = u[i];
                s = fma(v, v, s);
            }
            s = warp_sum(s);
            nrm = sqrt(s);
            if (lane == 0) {
                a.norms[(long long)l * a.R + warp] = nrm;
                a.colmax[(long long)l * a.R + warp] = mx;
            }
            return;
        } else if (ex > -1022 && ex < 1022) {
            const double sc = __hiloint2double((1023 - ex) << 20, 0);     // 2^-ex
            for (int i = lane; i < n; i += 32) {
                const double t = u[i] * sc;
                s = fma(t, t, s);
            }
        } else {                      // 2^-ex out of range: two exact power-of-two steps
            const int e1 = -ex / 2, e2 = -ex - e1;
            const double sc1 = ldexp(1.0, e1), sc2 = ldexp(1.0, e2);
            for (int i = lane; i < n; i += 32) {
                const double t = (u[i] * sc1) * sc2;
                s = fma(t, t, s);
            }
        }
        s = warp_sum(s);
        nrm = ldexp(sqrt(s), ex);
    }
    if (lane == 0) {
        a.norms[(long long)l * a.R + warp] = nrm;
        a.colmax[(long long)l * a.R + warp] = mx;
    }
}

// k_colnorms for a Hadamard-product source with n_l <= 32 NR: the warp forms its column once
// into registers (lane holds entries lane + 32 k) and takes the maximum and the sum from there,
// in the same per-lane order as k_colnorms (so the norms agree bit for bit).
template <int NR>
__global__ void k_colnorms_prod(NormArgs a)
{
    const int l = blockIdx.y;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= a.R) return;
    const Col<true> u(a, l, warp);
    const int n = sel3(a.n, l);
    double v[NR];
    long long mb = 0;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int i = lane + 32 * k;
        v[k] = i < n ? u[i] : 0.0;
        const long long b = __double_as_longlong(v[k]) & 0x7FFFFFFFFFFFFFFFll;
        mb = b > mb ? b : mb;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long b = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = b > mb ? b : mb;
    }
    const double mx = __longlong_as_double(mb);
    double nrm;
    if (mb == 0) {
        nrm = 0.0;
    } else if (mb >= 0x7FF0000000000000ll) {
        nrm = mx;
    } else {
        int ex;
        frexp(mx, &ex);
        double s = 0.0;
        if (ex > -450 && ex < 450) {
#pragma unroll
            for (int k = 0; k < NR; ++k)
                if (lane + 32 * k < n) s = fma(v[k], v[k], s);
            nrm = sqrt(warp_sum(s));
        } else {
            const int e1 = -ex / 2, e2 = -ex - e1;
            const bool one = ex > -1022 && ex < 1022;
            const double sc = one ? __hiloint2double((1023 - ex) << 20, 0) : 1.0;
            const double sc1 = one ? 1.0 : ldexp(1.0, e1), sc2 = one ? 1.0 : ldexp(1.0, e2);
#pragma unroll
            for (int k = 0; k < NR; ++k)
                if (lane + 32 * k < n) {
                    const double t = one ? v[k] * sc : (v[k] * sc1) * sc2;
                    s = fma(t, t, s);
                }
            nrm = ldexp(sqrt(warp_sum(s)), ex);
        }
    }
    if (lane == 0) {
        a.norms[(long long)l * a.R + warp] = nrm;
        a.colmax[(long long)l * a.R + warp] = mx;
    }
}

// Per term: keep iff all three norms are finite and nonzero (keep[nu] = 1 or 0), weight
// xi' = xi prod_l ||u_l|| (0 for a dropped term).  Non-finite data sets NONFINITE.
template <bool PROD>
__global__ void k_terms(NormArgs a, const double* xi, double* keepf, double* xin, double* xi_user, rhosvd_info* info)
{
    const int R = a.R;
    const double* norms = a.norms;
    for (int nu = blockIdx.x * blockDim.x + threadIdx.x; nu < R; nu += gridDim.x * blockDim.x) {
        const double d0 = norms[nu], d1 = norms[R + nu], d2 = norms[2 * R + nu];
        const double x = PROD ? a.xa[nu % a.Ra] * a.xb[nu / a.Ra] : xi[nu];
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
// terms (to about one ulp), zero columns for dropped terms; nn2 = ||Un(:, nu)||^2 as stored, to
// about 2^-44 of itself (it only enters the total energy behind the eps^2 thresholds).
// u / d is u * (2^-e / f) with d = f 2^e, f in [0.5, 1) (one FP64 multiply an entry; two exact
// power-of-two steps when 2^-e would leave the range).  With digit planes requested, column nu
// is also cut into OZ_S64 planes as operand row nu (k = x) with exponent E_nu from
// max |Un(:, nu)| = colmax * scale (the same multiply as the entries, so max < 2^E_nu holds
// exactly).  One warp per column, grid (ceil(R/8), 3).
template <bool PROD>
__global__ void k_normalize(NormArgs a, const double* keepf, double* Un, long long ustride, double* nn2, NormSlice ns)
{
    const int l = blockIdx.y;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= a.R) return;
    const int n = sel3(a.n, l);
    const Col<PROD> u(a, l, warp);
    double* dst = Un + l * ustride + (long long)warp * n;
    const bool keep = keepf[warp] != 0.0;
    const double d = a.norms[(long long)l * a.R + warp];
    double s1 = 0.0, s2 = 1.0;
    if (keep) {
        int e;
        const double f = frexp(d, &e);
        if (e > -1000 && e < 1000) {
            s1 = ldexp(1.0 / f, -e);
        } else {
            const int e1 = -e / 2, e2 = -e - e1;
            s1 = ldexp(1.0 / f, e1);
            s2 = ldexp(1.0, e2);
        }
    }
    uint16_t* P = sel3(ns.planes, l);
    const int pld = sel3(ns.ld, l);
    const long long pst = sel3(ns.pstride, l);
    const int ptk = sel3(ns.tiles_k, l), pth = sel3(ns.tile_h, l);
    int E = -126;
    if (P) {
        const double mx = (a.colmax[(long long)l * a.R + warp] * s1) * s2;
        if (mx > 0.0) {
            frexp(mx, &E);
            E = E < -126 ? -126 : (E > 127 ? 127 : E);
        }
        if (lane == 0) sel3(ns.exps, l)[warp] = (signed char)E;
    }
    // nn2 in FP32 double-float arithmetic (the square's exact high product by fma, the cross term,
    // a two-sum of the high parts): the multiply above is the entry's one FP64 instruction
    float sh = 0.f, sl = 0.f;
    const int lim = P ? (ptk > 0 ? ptk * 16 : pld) : n;     // a multiple of 8 when planes are cut
    // one multiply an element when s1 s2 is exact (s2 = 1 unless the exponent is extreme)
    const bool one = s2 == 1.0;
    // a lane takes 8 consecutive x a round: its 8 loads are in flight together, and each digit
    // plane gets one 16-byte store (8 consecutive k of the plane row nu)
    for (int i0 = lane * 8; i0 < lim; i0 += 32 * 8) {
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = i0 + q;
            const double x = (keep && i < n) ? u[i] : 0.0;
            v[q] = one ? x * s1 : (x * s1) * s2;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (i0 + q < n) {
                dst[i0 + q] = v[q];
                float vh, vl;
                split_f64(v[q], vh, vl);
                const float p = __fmul_rn(vh, vh);
                const float pe = __fadd_rn(__fmaf_rn(vh, vh, -p), __fmul_rn(2.0f * vh, vl));   // vl^2 dropped
                const float t = __fadd_rn(sh, p), bp = __fsub_rn(t, sh);
                sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp)), pe));
                sh = t;
            }
        }
        if (P) {
            uint32_t w[OZ_S64][4];
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                uint16_t d0[OZ_S64], d1[OZ_S64];
                oz_digits(v[q], E, OZ_S64, d0, OZ_W64);
                oz_digits(v[q + 1], E, OZ_S64, d1, OZ_W64);
#pragma unroll
                for (int t = 0; t < OZ_S64; ++t) w[t][q >> 1] = (uint32_t)d0[t] | ((uint32_t)d1[t] << 16);
            }
#pragma unroll
            for (int t = 0; t < OZ_S64; ++t) {
                uint16_t* dq = ptk > 0 ? P + oz_tiled_index(OZ_S64, ptk, pth, t, warp, i0)
                                       : P + (long long)t * pst + (long long)warp * pld + i0;
                *reinterpret_cast<uint4*>(dq) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
            }
        }
    }
    const double s = warp_sum((double)sh + (double)sl);
    if (lane == 0) nn2[(long long)l * a.R + warp] = s;
}

// Transposed digit planes (S digits of 7 bits) with one fixed exponent E0 (|x| < 2^E0):
// planes[s][x ld + nu] from X(x, nu) = X[x + ldx nu], zero for nu in [K, ld).  A 64 x 32 (x by
// nu) tile goes through shared memory so that reads run along x; a thread then cuts 8 consecutive
// nu of one x and writes one 16-byte chunk to every plane.  grid (ceil(ld/32), ceil(rows/64),
// nmodes), block 256.
template <int S>
__global__ void __launch_bounds__(256) k_slice_t(SliceTArgs a)
{
    const int b = blockIdx.z;
    const int nu0 = blockIdx.x * 32, x0 = blockIdx.y * 64;
    const int rows = sel3(a.rows, b), K = sel3(a.K, b), ld = sel3(a.ld, b);
    if (x0 >= rows || nu0 >= ld) return;
    __shared__ double tile[32][64];
    const double* X = sel3(a.X, b);
    const int ldx = sel3(a.ldx, b);
    const int tid = threadIdx.x;
    for (int e = tid; e < 32 * 64; e += 256) {
        const int j = e >> 6, xx = e & 63;
        const int nu = nu0 + j, x = x0 + xx;
        tile[j][xx] = (nu < K && x < rows) ? X[(long long)nu * ldx + x] : 0.0;
    }
    __syncthreads();
    // a warp: 32 consecutive x (conflict-free column reads), one 8-wide chunk of nu
    const int xx = tid & 63, c = tid >> 6;
    const int x = x0 + xx, nuc = nu0 + c * 8;
    if (x >= rows || nuc >= ld) return;
    uint16_t* P = sel3(a.planes, b);
    const long long pst = sel3(a.pstride, b);
    const int tk = sel3(a.tiles_k, b), th = sel3(a.tile_h, b);
    uint32_t w[S][4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
        uint16_t d0[S], d1[S];
        oz_digits(tile[c * 8 + q][xx], a.E0, S, d0, OZ_W64);
        oz_digits(tile[c * 8 + q + 1][xx], a.E0, S, d1, OZ_W64);
#pragma unroll
        for (int t = 0; t < S; ++t) w[t][q >> 1] = (uint32_t)d0[t] | ((uint32_t)d1[t] << 16);
    }
#pragma unroll
    for (int t = 0; t < S; ++t) {
        uint16_t* dq = tk > 0 ? P + oz_tiled_index(S, tk, th, t, x, nuc) : P + (long long)t * pst + (long long)x * ld + nuc;
        *reinterpret_cast<uint4*>(dq) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
    }
}

// Rademacher signs of the range sketch as one tile-major BF16 plane of 128-row tiles (+-1.0, zero
// outside; the operand on the TMEM lanes of the sketch product):
// operand row j < k (sketch column), k-index nu < R; sign(nu, j) = rademacher(seed, mode, nu, j).
// One thread per 8 consecutive nu of a row (a 16-byte chunk), grid (ceil(KT * 2 * rows / 256), nb).
__global__ void k_sign_planes(SignPlaneArgs a)
{
    const int b = blockIdx.y;
    const int rows = sel3(a.rows, b), K = sel3(a.K, b), mode = sel3(a.mode, b);
    const int KT = a.tiles_k, rpad = (rows + 127) / 128 * 128;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;   // chunk index
    const long long nchunk = (long long)rpad * KT * 2;
    if (e >= nchunk) return;
    const int j = (int)(e / (KT * 2)), c = (int)(e % (KT * 2));             // row, 8-wide chunk along nu
    const int nu0 = c * 8;
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t lohi[2];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int nu = nu0 + 2 * q + hh;
            lohi[hh] = (j < rows && nu < K) ? (rademacher_bit(a.seed, mode, nu, j) ? 0x3F80u : 0xBF80u) : 0u;
        }
        w[q] = lohi[0] | (lohi[1] << 16);
    }
    uint16_t* P = sel3(a.planes, b);
    *reinterpret_cast<uint4*>(P + oz_tiled_index(1, KT, OZ_BM, 0, j, nu0)) = make_uint4(w[0], w[1], w[2], w[3]);
}

int launch_sign_planes(const SignPlaneArgs& a, int nb, int rowsmax, cudaStream_t st)
{
    if (nb <= 0 || rowsmax <= 0 || a.tiles_k <= 0) return 0;
    const long long nchunk = (long long)((rowsmax + 127) / 128 * 128) * a.tiles_k * 2;
    dim3 grid((unsigned)((nchunk + 255) / 256), nb);
    k_sign_planes<<<grid, 256, 0, st>>>(a);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_slice_t(const SliceTArgs& a, int nb, int ldmax, int rowsmax, cudaStream_t st)
{
    if (nb <= 0 || ldmax <= 0 || rowsmax <= 0) return 0;
    dim3 grid((ldmax + 31) / 32, (rowsmax + 63) / 64, nb);
    if (a.S == OZ_S_SKETCH5) k_slice_t<OZ_S_SKETCH5><<<grid, 256, 0, st>>>(a);
    else if (a.S == 0 || a.S == OZ_S64) k_slice_t<OZ_S64><<<grid, 256, 0, st>>>(a);
    else return RHOSVD_ERR_INVALID_ARG;
    RH_CHECK_LAUNCH();
    return 0;
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
    const int n = sel3(a.n, l);
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
    const int n = sel3(a.n, l);
    for (long long nu = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; nu < R;
         nu += ((long long)gridDim.x * blockDim.x) >> 5) {
        const bool fromA = nu < a.Ra;
        const double* src = fromA ? a.A[l] + nu * a.lda[l] : a.B[l] + (nu - a.Ra) * a.ldb[l];
        double* dst = a.C[l] + nu * a.ldc[l];
        for (int x = lane; x < n; x += 32) dst[x] = src[x];
        if (l == 0 && lane == 0) a.xc[nu] = fromA ? a.alpha * a.xa[nu] : a.beta * a.xb[nu - a.Ra];
    }
}


// V^(l)(j, nu) (j < r_l, nu < R, at src_l[nu lds + j]) split into a float pair (h, l) with
// h = fl32(v) and l = fl32(v - h), at dst_l[nu ldd + j] (j contiguous, like the source): the
// Khatri-Rao operand of the tensor-core core contraction forms its products from these on the
// FP32 pipe (h h' exact by fma; about 2^-46 relative in all).
__global__ void k_split_v(const double* src, long long sstride, int lds, float2* dst, long long dstride, int ldd,
                          int R, const int* dr, int mode0)
{
    const int l = mode0 + blockIdx.y;
    const int r = dr[l];
    const double* S = src + l * sstride;
    float2* D = dst + l * dstride;
    const long long total = (long long)R * r;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e % r), nu = (int)(e / r);
        const double v = S[(long long)nu * lds + j];
        const float h = __double2float_rn(v);
        D[(long long)nu * ldd + j] = make_float2(h, __double2float_rn(v - (double)h));
    }
}

int launch_split_v(const double* src, long long sstride, int lds, float2* dst, long long dstride, int ldd, int R,
                   const int* dr, int mode0, int nmodes, cudaStream_t st)
{
    dim3 grid(512, nmodes);
    k_split_v<<<grid, 256, 0, st>>>(src, sstride, lds, dst, dstride, ldd, R, dr, mode0);
    RH_CHECK_LAUNCH();
    return 0;
}

// Per-row exponents of the split factors: out_l[j] = E with max_nu |V_l(j, nu)| < 2^E for the
// pair (h, l) at Vp_l[nu ldp + j] (|v| <= |h| (1 + 2^-23), so E comes from max |h| (1 + 2^-20)),
// clamped to [-45, 1].  A block covers 32 rows j (the lanes, reading consecutive pairs) with its
// 32 warps striding over nu, eight loads in flight a thread.  grid (ceil(KMAX / 32), nmodes),
// block 1024.
__global__ void __launch_bounds__(1024) k_row_exps(const float2* Vp, long long vstride, int ldp, const int* dr,
                                                   int mode0, int R, signed char* out, long long ostride)
{
    const int l = mode0 + blockIdx.y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane;
    const int r = dr[l];
    __shared__ float part[32][33];
    if (blockIdx.x * 32 >= r) return;
    const float2* v = Vp + l * vstride + j;
    float mx = 0.f;
    if (j < r) {
        int nu = w;
        for (; nu + 7 * 32 < R; nu += 8 * 32) {
            float h[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) h[q] = v[(long long)(nu + q * 32) * ldp].x;
#pragma unroll
            for (int q = 0; q < 8; ++q) mx = fmaxf(mx, fabsf(h[q]));
        }
        for (; nu < R; nu += 32) mx = fmaxf(mx, fabsf(v[(long long)nu * ldp].x));
    }
    part[w][lane] = mx;
    __syncthreads();
    if (w == 0 && j < r) {
        for (int q = 1; q < 32; ++q) mx = fmaxf(mx, part[q][lane]);
        int E = -45;
        if (mx > 0.f) {
            frexpf(mx * (1.0f + 0x1p-20f), &E);
            E = E < -45 ? -45 : (E > 1 ? 1 : E);
        }
        out[l * ostride + j] = (signed char)E;
    }
}

int launch_row_exps(const float2* Vp, long long vstride, int ldp, const int* dr, int mode0, int nmodes, int R,
                    signed char* out, long long ostride, cudaStream_t st)
{
    k_row_exps<<<dim3((KMAX + 31) / 32, nmodes), 1024, 0, st>>>(Vp, vstride, ldp, dr, mode0, R, out, ostride);
    RH_CHECK_LAUNCH();
    return 0;
}

__global__ void k_init_state(DevState* s, int k0, int k1, int k2, int m0, int m1, int m2, int kdef)
{
    s->kin[0] = k0; s->kin[1] = k1; s->kin[2] = k2;
    s->m[0] = m0; s->m[1] = m1; s->m[2] = m2;
    s->kdef[0] = s->kdef[1] = s->kdef[2] = kdef;
}

int launch_colnorms(const NormArgs& a, cudaStream_t st)
{
    if (a.R <= 0) return 0;
    dim3 grid((a.R + 7) / 8, 3);
    const int nmax = a.n[0] > a.n[1] ? (a.n[0] > a.n[2] ? a.n[0] : a.n[2]) : (a.n[1] > a.n[2] ? a.n[1] : a.n[2]);
    if (a.Ra > 0 && nmax <= 256) k_colnorms_prod<8><<<grid, 256, 0, st>>>(a);
    else if (a.Ra > 0 && nmax <= 1024) k_colnorms_prod<32><<<grid, 256, 0, st>>>(a);
    else if (a.Ra > 0) k_colnorms<true><<<grid, 256, 0, st>>>(a);
    else k_colnorms<false><<<grid, 256, 0, st>>>(a);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_terms(const NormArgs& na, const double* xi, double* keepf, double* xin, double* xi_user,
                 rhosvd_info* info, double* Un, long long ustride, double* nn2, double* total, const NormSlice& ns,
                 cudaStream_t st)
{
    const int R = na.R;
    if (R > 0) {
        if (na.Ra > 0) k_terms<true><<<(R + 255) / 256, 256, 0, st>>>(na, xi, keepf, xin, xi_user, info);
        else k_terms<false><<<(R + 255) / 256, 256, 0, st>>>(na, xi, keepf, xin, xi_user, info);
        RH_CHECK_LAUNCH();
        dim3 grid((R + 7) / 8, 3);
        if (na.Ra > 0) k_normalize<true><<<grid, 256, 0, st>>>(na, keepf, Un, ustride, nn2, ns);
        else k_normalize<false><<<grid, 256, 0, st>>>(na, keepf, Un, ustride, nn2, ns);
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

int launch_init_state(DevState* s, int k0, int k1, int k2, int m0, int m1, int m2, int kdef, cudaStream_t st)
{
    k_init_state<<<1, 1, 0, st>>>(s, k0, k1, k2, m0, m1, m2, kdef);
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

// ---------------------------------------------------------------- self-test of the fast helpers
namespace {
__global__ void k_selftest_fastmath(const double* x, double* rcp, double* rsq, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        rcp[i] = rh::fast_rcp(x[i]);
        rsq[i] = rh::fast_rsqrt(x[i]);
    }
}
}  // namespace

extern "C" int rhosvd_selftest_fastmath(const double* x, double* rcp, double* rsq, int n, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !rcp || !rsq))) return RHOSVD_ERR_INVALID_ARG;
    if (n == 0) return RHOSVD_OK;
    k_selftest_fastmath<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, (cudaStream_t)stream>>>(x, rcp, rsq, n);
    rh::count_launch();
    return cudaGetLastError() == cudaSuccess ? RHOSVD_OK : RHOSVD_ERR_CUDA;
}

namespace rh {

struct ToF32Args {
    const double* src[4];
    float* dst[4];
    long long cnt[4];
    const int* dr;
};

// grid (blocks, nb), block 256: grid-stride over the entries of array blockIdx.y
__global__ void k_to_f32(ToF32Args a)
{
    const int b = blockIdx.y;
    const long long cnt = a.cnt[b] >= 0 ? a.cnt[b] : (long long)a.dr[0] * a.dr[1] * a.dr[2];
    const double* s = a.src[b];
    float* d = a.dst[b];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt; e += (long long)gridDim.x * blockDim.x)
        d[e] = __double2float_rn(s[e]);
}

int launch_to_f32(const double* const src[4], float* const dst[4], const long long cnt[4], const int* dr, int nb,
                  cudaStream_t st)
{
    if (nb < 1 || nb > 4) return RHOSVD_ERR_INVALID_ARG;
    ToF32Args a;
    for (int b = 0; b < 4; ++b) {
        a.src[b] = b < nb ? src[b] : nullptr;
        a.dst[b] = b < nb ? dst[b] : nullptr;
        a.cnt[b] = b < nb ? cnt[b] : 0;
    }
    a.dr = dr;
    k_to_f32<<<dim3(2 * 152, nb), 256, 0, st>>>(a);
    RH_CHECK_LAUNCH();
    return 0;
}

}  // namespace rh

// FP64 FMA rate probe: eight independent fma chains per thread (a <- a b + c), `iters` steps
// each; the chains' sum is stored so that nothing is dead code.  2 * 8 * iters FLOP a thread.
__global__ void __launch_bounds__(256) k_fp64_rate(int iters, double b, double c, double* out)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 1.0 + 1e-3 * (double)(j + (int)(t & 255));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    out[t] = s;
}

extern "C" int rhosvd_probe_fp64(int blocks, int iters, double* out, void* stream)
{
    if (blocks < 1 || blocks > (1 << 20) || iters < 1 || !out) return RHOSVD_ERR_INVALID_ARG;
    k_fp64_rate<<<blocks, 256, 0, (cudaStream_t)stream>>>(iters, 0.999999999, 1e-12, out);
    RH_CHECK_LAUNCH();
    return RHOSVD_OK;
}
