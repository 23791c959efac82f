// ozgemm.cu -- the host side and the helper kernels of the digit-plane tensor-core products (see
// ozgemm.cuh for the arithmetic, ozgemm_tma.cu for the GEMM kernels): the digit-plane slicer
// (per-row exponents, tile-major plane writes), the split-K reduction, the core's split count, and
// launch_ozgemm, which sends each product to its warp-specialised kernel.
#include "ozgemm.cuh"

namespace rh {

// status of the products launched without a caller status word (see ozgemm.cuh)
int oz_take_status(cudaStream_t st, int* out) { return oztma_take_status(st, out); }

namespace {

__device__ __forceinline__ int oz_dim(const int* d, int h) { return d ? *d : h; }

}  // namespace

// ---------------------------------------------------------------- digit-plane slicer
// Two kernels.  k_oz_rowexp: the per-row exponent E_i = e(max_k |x_ik|) (|x| < 2^E, the frexp
// exponent, clamped to [-126, 127]; -126 for an all-zero row) from the integer exponent fields,
// reading along whichever operand dimension is contiguous.  k_oz_slice_tile: 32 rows x 64 k per
// block, staged in shared memory so that both the loads (either layout) and the plane stores
// (k contiguous) are coalesced.

// frexp exponent of x from its bits (x = f 2^e, 0.5 <= |f| < 1); -4096 for zero; subnormals read
// as -1022 (they clamp to -126 anyway)
__device__ __forceinline__ int oz_frexp_exp(double x)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((bits >> 52) & 0x7FF);
    if ((bits << 1) == 0) return -4096;
    return ef == 0 ? -1022 : ef - 1022;
}

constexpr int OZ_RE_ROWS = 8;       // rows a block of k_oz_rowexp (rows-contiguous layout)

__global__ void k_oz_rowexp(OzSliceArgs a)
{
    const int b = blockIdx.y;
    const int rows = a.rows[b];
    const int live = a.drows[b] ? *a.drows[b] : rows;
    const int K = a.dK[b] ? *a.dK[b] : a.K[b];
    const double* X = a.X[b];
    const double* ks = a.kscale[b];
    const long long rs = a.rs[b], cs = a.cs[b];
    const int tid = threadIdx.x;
    __shared__ int emax[32];
    const int r0 = blockIdx.x * OZ_RE_ROWS;
    if (r0 >= rows) return;
    if (tid < 32) emax[tid] = -4096;
    __syncthreads();
    if (rs == 1) {
        // rows contiguous: a warp reads 8 rows x 4 k (four 64-byte segments)
        const int i = r0 + (tid & (OZ_RE_ROWS - 1)), kk = tid / OZ_RE_ROWS;
        int e = -4096;
        constexpr int STEP = 256 / OZ_RE_ROWS;
        if (i < live) {
            // eight independent loads in flight per thread
            int k = kk;
            for (; k + 7 * STEP < K; k += 8 * STEP) {
                double x[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) x[q] = X[(long long)i + (long long)(k + q * STEP) * cs];
#pragma unroll
                for (int q = 0; q < 8; ++q) e = max(e, oz_frexp_exp(ks ? x[q] * ks[k + q * STEP] : x[q]));
            }
            for (; k < K; k += STEP) {
                double x = X[(long long)i + (long long)k * cs];
                if (ks) x *= ks[k];
                e = max(e, oz_frexp_exp(x));
            }
        }
        atomicMax(&emax[tid & (OZ_RE_ROWS - 1)], e);
    } else {
        // k contiguous (or strided both ways): a warp per row, lanes along k
        const int lane = tid & 31, w = tid >> 5;
        const int i = r0 + w;
        int e = -4096;
        if (w < OZ_RE_ROWS && i < live) {
            int k = lane;
            for (; k + 7 * 32 < K; k += 8 * 32) {
                double x[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) x[q] = X[(long long)i * rs + (long long)(k + q * 32) * cs];
#pragma unroll
                for (int q = 0; q < 8; ++q) e = max(e, oz_frexp_exp(ks ? x[q] * ks[k + q * 32] : x[q]));
            }
            for (; k < K; k += 32) {
                double x = X[(long long)i * rs + (long long)k * cs];
                if (ks) x *= ks[k];
                e = max(e, oz_frexp_exp(x));
            }
        }
        for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        if (lane == 0 && w < OZ_RE_ROWS) emax[w] = e;
    }
    __syncthreads();
    if (tid < OZ_RE_ROWS && r0 + tid < rows) {
        int E = emax[tid];
        if (E == -4096) E = -126;
        E = min(127, max(-126, E));
        a.exps[b][r0 + tid] = (signed char)E;
    }
}

// The same exponents for k-contiguous operands of few rows and long K (the Gram B Bᵀ's B: k rows,
// K = R; the core's V¹: r1 rows, K = R): one row per block, all 256 threads along k, so that the
// launch has rows x problems blocks instead of rows / 8 (a block of 8 rows took 157 us for
// K = 20000, this form about a tenth of it).  grid (rows, nb).
__global__ void __launch_bounds__(256) k_oz_rowexp_long(OzSliceArgs a)
{
    const int b = blockIdx.y, i = blockIdx.x;
    const int rows = a.rows[b];
    if (i >= rows) return;
    const int live = a.drows[b] ? *a.drows[b] : rows;
    const int K = a.dK[b] ? *a.dK[b] : a.K[b];
    const double* X = a.X[b];
    const double* ks = a.kscale[b];
    const long long rs = a.rs[b];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ int wmax[8];
    int e = -4096;
    if (i < live) {
        const double* row = X + (long long)i * rs;
        int k = tid;
        // four independent loads in flight per thread
        for (; k + 3 * 256 < K; k += 4 * 256) {
            double x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = row[k + q * 256];
#pragma unroll
            for (int q = 0; q < 4; ++q) e = max(e, oz_frexp_exp(ks ? x[q] * ks[k + q * 256] : x[q]));
        }
        for (; k < K; k += 256) e = max(e, oz_frexp_exp(ks ? row[k] * ks[k] : row[k]));
    }
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (lane == 0) wmax[warp] = e;
    __syncthreads();
    if (tid == 0) {
        int E = wmax[0];
        for (int w = 1; w < 8; ++w) E = max(E, wmax[w]);
        if (E == -4096) E = -126;
        a.exps[b][i] = (signed char)min(127, max(-126, E));
    }
}

// The same for rows-contiguous operands of long K (rs = 1: B of B Bᵀ stored with its k rows
// adjacent, the core's V¹): two rows a block, 128 threads along k each, so that a launch has
// rows / 2 x problems blocks instead of rows / 8 (eight rows a block took ~37 us at K = 4096).
// A warp's load covers 16 k of two adjacent rows (16-byte pieces of L2-resident data).
// grid (ceil(rows / 2), nb).
__global__ void __launch_bounds__(256) k_oz_rowexp_cols(OzSliceArgs a)
{
    const int b = blockIdx.y;
    const int rows = a.rows[b];
    const int r0 = blockIdx.x * 2;
    if (r0 >= rows) return;
    const int live = a.drows[b] ? *a.drows[b] : rows;
    const int K = a.dK[b] ? *a.dK[b] : a.K[b];
    const double* X = a.X[b];
    const double* ks = a.kscale[b];
    const long long cs = a.cs[b];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = tid & 1, i = r0 + r;
    __shared__ int wmax[8][2];
    int e = -4096;
    if (i < live) {
        int k = tid >> 1;
        // eight independent loads in flight per thread
        for (; k + 7 * 128 < K; k += 8 * 128) {
            double x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) x[q] = X[(long long)i + (long long)(k + q * 128) * cs];
#pragma unroll
            for (int q = 0; q < 8; ++q) e = max(e, oz_frexp_exp(ks ? x[q] * ks[k + q * 128] : x[q]));
        }
        for (; k < K; k += 128) {
            double x = X[(long long)i + (long long)k * cs];
            if (ks) x *= ks[k];
            e = max(e, oz_frexp_exp(x));
        }
    }
    for (int o = 16; o > 1; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));   // lanes of one row
    if (lane < 2) wmax[warp][lane] = e;
    __syncthreads();
    if (tid < 2 && r0 + tid < rows) {
        int E = wmax[0][tid];
        for (int w = 1; w < 8; ++w) E = max(E, wmax[w][tid]);
        if (E == -4096) E = -126;
        a.exps[b][r0 + tid] = (signed char)min(127, max(-126, E));
    }
}

constexpr int OZ_ST_R = 32, OZ_ST_K = 64;
constexpr int OZ_FUSE_KMAX = 256;   // K up to which a slicer block finds its rows' exponents itself

// S as a template argument: the digit loops unroll and the digits stay in registers.  With FUSE
// (every problem of the call has K <= OZ_FUSE_KMAX) a block first finds the exponents of its 32
// rows itself, reading the rows' whole K (the other k tiles' blocks read the same rows, from L2),
// and the blocks of the first k tile store them for the product: one launch instead of two, the
// same exponents as k_oz_rowexp's.
template <int S, bool FUSE>
__global__ void __launch_bounds__(256) k_oz_slice_tile(OzSliceArgs a)
{
    const int b = blockIdx.z;
    const int rows = a.rows[b];
    const int tk = a.tiles_k[b];
    const int ld = tk > 0 ? tk * 16 : a.ld[b];          // tile-major: every k of the last tile
    const int i0 = blockIdx.y * OZ_ST_R, k0 = blockIdx.x * OZ_ST_K;
    if (i0 >= rows || k0 >= ld) return;
    const int live = a.drows[b] ? *a.drows[b] : rows;
    const int K = a.dK[b] ? *a.dK[b] : a.K[b];
    const double* X = a.X[b];
    const double* ks = a.kscale[b];
    const long long rs = a.rs[b], cs = a.cs[b];
    __shared__ double T[OZ_ST_R][OZ_ST_K + 1];
    __shared__ int s_e[OZ_ST_R];
    const int tid = threadIdx.x;
    if (FUSE) {
        if (tid < OZ_ST_R) s_e[tid] = -4096;
        __syncthreads();
        // (loads issued four at a time: these reads are latency-bound L2 hits)
        if (rs == 1) {
            // rows contiguous: a warp reads 32 consecutive rows at one k
            const int r = tid & 31, i = i0 + r;
            int e = -4096;
            if (i < live) {
                int k = tid >> 5;
                for (; k + 24 < K; k += 32) {
                    double x[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) x[q] = X[(long long)i + (long long)(k + 8 * q) * cs];
#pragma unroll
                    for (int q = 0; q < 4; ++q) e = max(e, oz_frexp_exp(ks ? x[q] * ks[k + 8 * q] : x[q]));
                }
                for (; k < K; k += 8) {
                    double x = X[(long long)i + (long long)k * cs];
                    if (ks) x *= ks[k];
                    e = max(e, oz_frexp_exp(x));
                }
            }
            atomicMax(&s_e[r], e);
        } else {
            // k contiguous (or strided both ways): lanes along k, a warp's four rows read together
            const int lane = tid & 31, w = tid >> 5;
            int e[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) e[q] = -4096;
            for (int k = lane; k < K; k += 32) {
                double x[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = i0 + w + 8 * q;
                    x[q] = i < live ? X[(long long)i * rs + (long long)k * cs] : 0.0;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (i0 + w + 8 * q < live) e[q] = max(e[q], oz_frexp_exp(ks ? x[q] * ks[k] : x[q]));
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int eq = e[q];
                for (int o = 16; o > 0; o >>= 1) eq = max(eq, __shfl_xor_sync(0xffffffffu, eq, o));
                if (lane == 0) s_e[w + 8 * q] = eq;
            }
        }
        __syncthreads();
        if (tid < OZ_ST_R) {
            int E = s_e[tid];
            if (E == -4096) E = -126;
            E = min(127, max(-126, E));
            s_e[tid] = E;
            if (blockIdx.x == 0 && i0 + tid < rows) a.exps[b][i0 + tid] = (signed char)E;
        }
    }
    if (rs == 1) {
        const int r = tid & 31;
        for (int kk = tid >> 5; kk < OZ_ST_K; kk += 8) {
            const int i = i0 + r, k = k0 + kk;
            double x = 0.0;
            if (i < live && k < K) {
                x = X[(long long)i + (long long)k * cs];
                if (ks) x *= ks[k];
            }
            T[r][kk] = x;
        }
    } else {
        const int kk = tid & (OZ_ST_K - 1);
        for (int r = tid / OZ_ST_K; r < OZ_ST_R; r += 256 / OZ_ST_K) {
            const int i = i0 + r, k = k0 + kk;
            double x = 0.0;
            if (i < live && k < K) {
                x = X[(long long)i * rs + (long long)k * cs];
                if (ks) x *= ks[k];
            }
            T[r][kk] = x;
        }
    }
    __syncthreads();
    uint16_t* P = a.planes[b];
    const long long ps = a.pstride[b];
    const int kk = tid & (OZ_ST_K - 1), k = k0 + kk;
    if (k >= ld) return;
    for (int r = tid / OZ_ST_K; r < OZ_ST_R; r += 256 / OZ_ST_K) {
        const int i = i0 + r;
        if (i >= rows) break;
        const int E = FUSE ? s_e[r] : (a.exps[b] ? (int)a.exps[b][i] : a.exp0);
        uint16_t d[S];
        if (S == 4)
            oz_digits_bal(T[r][kk], E, d);       // the Khatri-Rao core's operand (balanced digits)
        else
            oz_digits(T[r][kk], E, S, d, S == OZ_S64 ? OZ_W64 : 8);
        if (tk > 0) {
            const int th = a.tile_h[b];
#pragma unroll
            for (int s2 = 0; s2 < S; ++s2) P[oz_tiled_index(S, tk, th, s2, i, k)] = d[s2];
            uint16_t* P2 = a.planes2[b];
            if (P2) {
                const int th2 = a.tile_h2[b];
#pragma unroll
                for (int s2 = 0; s2 < S; ++s2) P2[oz_tiled_index(S, tk, th2, s2, i, k)] = d[s2];
            }
        } else {
            uint16_t* q = P + (long long)i * ld + k;
#pragma unroll
            for (int s2 = 0; s2 < S; ++s2) q[s2 * ps] = d[s2];
        }
    }
}

// C(i, j) = sum over the splits of the partials, in split order.  grid (ceil(MN / 256), nb).
__global__ void k_oz_reduce(OzBatch batch)
{
    const OzProblem& P = batch.p[blockIdx.y];
    const int ns = P.dsplit ? max(1, min(*P.dsplit, batch.nsplit)) : batch.nsplit;
    if (ns <= 1) return;                       // one split wrote C directly
    const int M = P.M_from_r2r3 ? (*P.dNa) * (*P.dNb) : oz_dim(P.dM, P.M);
    const int N = oz_dim(P.dN, P.N);
    const long long crs = P.crs < 0 ? (long long)N : P.crs;
    const long long ccs = P.ccs < 0 ? (long long)M : P.ccs;
    const long long total = (long long)M * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % M), j = (int)(e / M);
        const long long o = i * crs + j * ccs;
        double s = 0.0;
        for (int sp = 0; sp < ns; ++sp) s += P.Cpart[sp * P.split_stride + o];
        P.C[o] = s;
    }
}

// The core's split count from the ranks on the device: M = r2 r3 rows, N = r1 columns, K = R.
// Doubles until the tiles times the splits fill the GPU once, each split keeps at least four
// stages, every split's partial (M N values) fits split_stride, and smax is not passed.
__global__ void k_core_split(const int* r, int K, int smax, long long split_stride, int* out)
{
    const long long M = (long long)r[1] * r[2], N = r[0];
    const long long tiles = ((M + OZ_BM - 1) / OZ_BM) * ((N + OZ_CORE_NT - 1) / OZ_CORE_NT);
    const int stages = (K + OZ_BK - 1) / OZ_BK;
    int s2 = 1;
    if (M * N <= split_stride)
        while (s2 * 2 <= smax && tiles * s2 < 152 && stages / (s2 * 2) >= 4) s2 *= 2;
    *out = s2;
}

int launch_core_split(const int* r, int K, int smax, long long split_stride, int* out, cudaStream_t st)
{
    k_core_split<<<1, 1, 0, st>>>(r, K, smax, split_stride, out);
    RH_CHECK_LAUNCH();
    return 0;
}

int oz_choose_split(int M, int N, int K, int nt, int nbatch)
{
    const long long tiles = (long long)((M + OZ_BM - 1) / OZ_BM) * ((N + nt - 1) / nt) * (nbatch > 0 ? nbatch : 1);
    const int stages = (K + OZ_BK - 1) / OZ_BK;
    int s = 1;
    while (tiles * s * 2 <= 2 * 152 && stages / (s * 2) >= 4) s *= 2;
    return s;
}

int launch_oz_slice(const OzSliceArgs& a, int nb, cudaStream_t st)
{
    int rmax = 0, ldmax = 0;
    bool exps = false;
    for (int b = 0; b < nb; ++b) {
        rmax = max(rmax, a.rows[b]);
        ldmax = max(ldmax, a.tiles_k[b] > 0 ? a.tiles_k[b] * 16 : a.ld[b]);
        exps = exps || a.exps[b] != nullptr;
    }
    if (rmax <= 0 || ldmax <= 0) return 0;
    bool fuse = false;
    if (exps) {
        // every problem of one call either has exponents or not (the slicers are per operand)
        int kmax = 0;
        for (int b = 0; b < nb; ++b) {
            if (!a.exps[b]) return RHOSVD_ERR_INVALID_ARG;
            kmax = max(kmax, a.K[b]);
        }
        fuse = a.S == OZ_S64 && kmax <= OZ_FUSE_KMAX;
        bool kcontig = true, rcontig = true;
        for (int b = 0; b < nb; ++b) {
            kcontig = kcontig && a.cs[b] == 1;
            rcontig = rcontig && a.rs[b] == 1;
        }
        if (!fuse && kcontig && kmax >= 1024) {
            k_oz_rowexp_long<<<dim3(rmax, nb), 256, 0, st>>>(a);
            RH_CHECK_LAUNCH();
        } else if (!fuse && rcontig && kmax >= 1024) {
            k_oz_rowexp_cols<<<dim3((rmax + 1) / 2, nb), 256, 0, st>>>(a);
            RH_CHECK_LAUNCH();
        } else if (!fuse) {
            k_oz_rowexp<<<dim3((rmax + OZ_RE_ROWS - 1) / OZ_RE_ROWS, nb), 256, 0, st>>>(a);
            RH_CHECK_LAUNCH();
        }
    }
    dim3 grid((ldmax + OZ_ST_K - 1) / OZ_ST_K, (rmax + OZ_ST_R - 1) / OZ_ST_R, nb);
    switch (a.S) {
    case OZ_S64:
        if (fuse) k_oz_slice_tile<OZ_S64, true><<<grid, 256, 0, st>>>(a);
        else k_oz_slice_tile<OZ_S64, false><<<grid, 256, 0, st>>>(a);
        break;
    case 4: k_oz_slice_tile<4, false><<<grid, 256, 0, st>>>(a); break;
    case 1: k_oz_slice_tile<1, false><<<grid, 256, 0, st>>>(a); break;
    default: return RHOSVD_ERR_INVALID_ARG;
    }
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_ozgemm(const OzBatch& b, OzKind kind, cudaStream_t st)
{
    if (kind == OZ_CORE) {
        // the warp-specialised core, then the split-K partials summed in a fixed order
        int Mh = 0, Nh = 0;
        for (int i = 0; i < b.nbatch; ++i) {
            Mh = max(Mh, b.p[i].M);
            Nh = max(Nh, b.p[i].N);
        }
        if (Mh <= 0 || Nh <= 0) return 0;
        const int rc = launch_ozcore_tma(b, st);
        if (rc) return rc;
        if (b.nsplit > 1) {
            const long long mn = (long long)Mh * Nh;
            dim3 rg((unsigned)((mn + 255) / 256 < 4096 ? (mn + 255) / 256 : 4096), b.nbatch);
            k_oz_reduce<<<rg, 256, 0, st>>>(b);
            RH_CHECK_LAUNCH();
        }
        return 0;
    }
    if (ozgemm_tma_supports(b, kind)) {
        // the warp-specialised TMA pipeline, then the split-K partials summed in a fixed order
        int Mh = 0, Nh = 0;
        for (int i = 0; i < b.nbatch; ++i) {
            Mh = max(Mh, b.p[i].M);
            Nh = max(Nh, b.p[i].N);
        }
        if (Mh <= 0 || Nh <= 0) return 0;
        const int rc = launch_ozgemm_tma(b, kind, st);
        if (rc) return rc;
        if (b.nsplit > 1) {
            const long long mn = (long long)Mh * Nh;
            dim3 rg((unsigned)((mn + 255) / 256 < 4096 ? (mn + 255) / 256 : 4096), b.nbatch);
            k_oz_reduce<<<rg, 256, 0, st>>>(b);
            RH_CHECK_LAUNCH();
        }
        return 0;
    }
    // no operand layout that the TMA-fed kernels cannot read is produced by this library
    return RHOSVD_ERR_INVALID_ARG;
}

}  // namespace rh
