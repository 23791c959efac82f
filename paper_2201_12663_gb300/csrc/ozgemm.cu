// ozgemm.cu -- tcgen05 kernels of the sliced FP64-class GEMM (see ozgemm.cuh for the arithmetic).
//
// CTA tile 128 x NT, K pipelined in stages of 32 through two shared-memory buffers.  Operand
// planes sit in shared memory in the canonical K-major layout without swizzle (8-row x 16-byte
// core matrices, LBO = 128 B along K, SBO = 512 B along M/N).  One thread issues the
// tcgen05.mma instructions (kind::f16, BF16 in, FP32 accumulate) for every digit pair (s, t)
// with s + t <= GMAX into TMEM accumulators, one per group g = s + t.  A group of np pairs of
// W-bit digits is exact while np * 2^(2W) * (its K since the last readback) < 2^24, so it is read
// back into double-float registers at that cadence (for the 7-bit FP64-class digits: every 4
// stages for the largest groups, every 8 for the others; with 8-bit digits the largest groups
// would need a readback, and a wait for the stage's MMAs, after every stage).  With fewer
// accumulators than groups, the last one takes the remaining (smallest) groups; it is inexact
// but read back at the shortest cadence, so its FP32 partial sums never span more than a few
// stages (the tensor cores' FP32 accumulation drops the bits of each product below the
// accumulator's last place: over a long K with operands of one sign that error would grow with
// K).  16 warps: warp w reads TMEM lanes 32 (w % 4) .. +31 and a quarter of the columns.
// Every wait on an mbarrier is bounded; on expiry the kernel flags `err` and still frees TMEM.
#include "ozgemm.cuh"

namespace rh {

// status word of the tensor-core products launched without a caller status (the network
// kernels): RHOSVD_ERR_TIMEOUT once a bounded wait expired; read and cleared by oz_take_status
__device__ int g_oz_status = 0;

int oz_take_status(cudaStream_t st, int* out)
{
    int v = 0, w = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_oz_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RHOSVD_ERR_CUDA;
    if (v != 0) {
        const int zero = 0;
        if (cudaMemcpyToSymbolAsync(g_oz_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
    }
    const int rc = oztma_take_status(st, &w);
    if (rc) return rc;
    *out = v ? v : w;
    return RHOSVD_OK;
}

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle, LBO 128 B, SBO 512 B, sm_100 version 1.
__device__ __forceinline__ uint64_t oz_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((512u >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t oz_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void oz_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                 "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void oz_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}

// Bounded wait for the completion of the phase with the given parity.  Returns false on expiry.
__device__ __forceinline__ bool oz_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done = 0;
    for (long it = 0; it < (1L << 24) && !done; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    }
    return done != 0;
}

__device__ __forceinline__ void tmem_ld8(uint32_t addr, float* v)
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// (hi, lo) += x in double-float: exact two-sum, then renormalise so that |lo| stays below half
// an ulp of hi and its own roundings stay at 2^-48 of the sum
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    const float l = lo + err;
    hi = s + l;
    lo = l - (hi - s);
}

// number of digit pairs (s, t), 1 <= s <= SA, 1 <= t <= SB, in group g = s + t
__host__ __device__ constexpr int oz_npairs(int SA, int SB, int g)
{
    int c = 0;
    for (int s = 1; s <= SA; ++s)
        if (g - s >= 1 && g - s <= SB) ++c;
    return c;
}

// readback cadence (stages of 32 K) of an exact group of np pairs of W-bit digits: the group's
// FP32 sum stays exact while np 2^(2W) 32 c <= 2^24, i.e. c <= 2^(19 - 2W) / np; a power of two,
// at most 8
__host__ __device__ constexpr int oz_cad(int np, int W)
{
    const int lim = (1 << (19 - 2 * W)) / (np > 0 ? np : 1);
    int c = 1;
    while (c * 2 <= lim && c * 2 <= 8) c *= 2;
    return c;
}

// cadence of accumulator a when accumulators 0 .. NE-1 hold the exact groups g = a + 2 and
// accumulator NE (if any) the rest, which is read back at the shortest exact cadence
__host__ __device__ constexpr int oz_acc_cad(int SA, int SB, int NE, int a, int W)
{
    if (a < NE) return oz_cad(oz_npairs(SA, SB, a + 2), W);
    int m = 8;
    for (int e = 0; e < NE; ++e)
        m = oz_cad(oz_npairs(SA, SB, e + 2), W) < m ? oz_cad(oz_npairs(SA, SB, e + 2), W) : m;
    return m;
}

// every exact group fits one stage: np 2^(2W) 32 <= 2^24
__host__ __device__ constexpr bool oz_exact_ok(int SA, int SB, int NE, int W)
{
    for (int e = 0; e < NE; ++e)
        if (oz_npairs(SA, SB, e + 2) > (1 << (19 - 2 * W))) return false;
    return true;
}

// byte offset of (row r, 16-byte chunk c of the 32-wide K stage) in a plane tile
__device__ __forceinline__ uint32_t oz_off(int r, int c) { return (uint32_t)((r >> 3) * 512 + c * 128 + (r & 7) * 16); }

__device__ __forceinline__ int oz_dim(const int* d, int h) { return d ? *d : h; }

}  // namespace

template <int SA, int SB, int GMAX, int ASRC, int BSRC, int EPI, int NT, int NACC, int W>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_ozgemm(OzBatch batch)
{
    constexpr int A_PLANE = OZ_BM * OZ_BK * 2;
    constexpr int B_PLANE = NT * OZ_BK * 2;
    constexpr int STAGE = SA * A_PLANE + SB * B_PLANE;
    constexpr int NQ = NT / 4;                  // columns per thread in the epilogue
    constexpr int NG = GMAX - 1;                // groups g = 2 .. GMAX
    constexpr int NE = NACC >= NG ? NG : NACC - 1;   // exact accumulators
    constexpr int NU = NACC >= NG ? NG : NACC;       // accumulators in use
    constexpr int MINCAD = oz_acc_cad(SA, SB, NE, NU - 1, W) < oz_acc_cad(SA, SB, NE, 0, W)
                               ? oz_acc_cad(SA, SB, NE, NU - 1, W) : oz_acc_cad(SA, SB, NE, 0, W);
    static_assert(NT % 32 == 0 && NT >= 32 && NU * NT <= 512, "tile: 8-column TMEM loads per thread quarter");
    static_assert(GMAX >= 2 && GMAX <= SA + SB && NACC >= 1 && (NACC >= 2 || GMAX == 2), "groups");
    static_assert(oz_exact_ok(SA, SB, NE, W), "an exact group must fit one stage");
    static_assert(W == 7 || W == 8, "digit width");
    const int nsplit_h = batch.nsplit > 1 ? batch.nsplit : 1;
    const int split = blockIdx.z % nsplit_h;
    const OzProblem& P = batch.p[blockIdx.z / nsplit_h];
    const int nsplit = P.dsplit ? max(1, min(*P.dsplit, nsplit_h)) : nsplit_h;
    if (split >= nsplit) return;
    int M = P.M_from_r2r3 ? (*P.dNa) * (*P.dNb) : oz_dim(P.dM, P.M);
    const int N = oz_dim(P.dN, P.N);
    const int Kall = oz_dim(P.dK, P.K);
    // this CTA's K range [kbase, kbase + K): whole stages, the last split takes the rest
    const int kspan = ((Kall + nsplit - 1) / nsplit + OZ_BK - 1) / OZ_BK * OZ_BK;
    const int kbase = min(Kall, split * kspan);
    const int K = min(Kall, kbase + kspan) - kbase;
    double* const Cout = nsplit > 1 ? P.Cpart + split * P.split_stride : P.C;
    const int i0 = blockIdx.x * OZ_BM, j0 = blockIdx.y * NT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (i0 >= M || j0 >= N) {
        if (EPI == OZ_EPI_RESID && tid == 0) P.rpart[blockIdx.x + gridDim.x * blockIdx.y] = 0.0;
        return;
    }
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ double red[32];
    __shared__ int s_fail;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    // accumulator a < NACC - 1 holds group g = a + 2 exactly; accumulator NACC - 1 the rest

    const int r2 = ASRC == OZ_A_KR ? *P.dNa : 1;
    const int nkt = (K + OZ_BK - 1) / OZ_BK;

    // ---- producer: fill stage buffer `buf` with K slice kt of every plane
    auto produce = [&](int kt, int buf) {
        unsigned char* sA = oz_smem + buf * STAGE;
        unsigned char* sB = sA + SA * A_PLANE;
        const int k0 = kbase + kt * OZ_BK;
        // A: 128 rows x 4 chunks of 8
        for (int e = tid; e < OZ_BM * 4; e += OZ_THREADS) {
            const int r = e >> 2, c = e & 3;
            const int gi = i0 + r, gk = k0 + c * 8;
            if (ASRC == OZ_A_PLANES) {
#pragma unroll
                for (int s = 0; s < SA; ++s) {
                    uint4 v = make_uint4(0, 0, 0, 0);
                    if (gi < M && gk < kbase + K)
                        v = *reinterpret_cast<const uint4*>(P.A.base + s * P.A.pstride + (long long)gi * P.A.ld + gk);
                    *reinterpret_cast<uint4*>(sA + s * A_PLANE + oz_off(r, c)) = v;
                }
            } else {
                // entries V2(j, nu) V3(m, nu) from FP32 pairs on the FP32 pipe: the head product
                // is exact with its fma error, the cross terms add the rest (about 2^-46
                // relative, far below the 2^-8 SA digits); F = round(x 2^(8 SA)) on the integer pipe
                static_assert(ASRC != OZ_A_KR || SA <= 4, "the pair product carries about 46 bits");
                uint16_t d[8][SA];
                const int jj = gi % r2, mm = gi / r2;
                const int Er = (P.kr.e2 && gi < M) ? (int)P.kr.e2[jj] + (int)P.kr.e3[mm] : 0;
                const float TWO_8S = __int_as_float((127 + W * SA - Er) << 23);     // 2^(W SA - E)
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    long long F = 0;
                    if (gi < M && gk + q < kbase + K) {
                        const float2 a = P.kr.V2t[(long long)jj * P.kr.ldt + gk + q];
                        const float2 b = P.kr.V3t[(long long)mm * P.kr.ldt + gk + q];
                        const float ph = a.x * b.x;
                        float pe = fmaf(a.x, b.x, -ph);
                        pe = fmaf(a.x, b.y, fmaf(a.y, b.x, pe));
                        F = __float2ll_rn(ph * TWO_8S) + __float2ll_rn(pe * TWO_8S);
                    }
                    oz_digits_int(F, SA, d[q], W);
                }
#pragma unroll
                for (int s = 0; s < SA; ++s) {
                    uint4 v;
                    v.x = (uint32_t)d[0][s] | ((uint32_t)d[1][s] << 16);
                    v.y = (uint32_t)d[2][s] | ((uint32_t)d[3][s] << 16);
                    v.z = (uint32_t)d[4][s] | ((uint32_t)d[5][s] << 16);
                    v.w = (uint32_t)d[6][s] | ((uint32_t)d[7][s] << 16);
                    *reinterpret_cast<uint4*>(sA + s * A_PLANE + oz_off(r, c)) = v;
                }
            }
        }
        // B: NT rows x 4 chunks of 8
        for (int e = tid; e < NT * 4; e += OZ_THREADS) {
            const int r = e >> 2, c = e & 3;
            const int gj = j0 + r, gk = k0 + c * 8;
            if (BSRC == OZ_B_PLANES) {
#pragma unroll
                for (int t = 0; t < SB; ++t) {
                    uint4 v = make_uint4(0, 0, 0, 0);
                    if (gj < N && gk < kbase + K)
                        v = *reinterpret_cast<const uint4*>(P.B.base + t * P.B.pstride + (long long)gj * P.B.ld + gk);
                    *reinterpret_cast<uint4*>(sB + t * B_PLANE + oz_off(r, c)) = v;
                }
            } else {
                uint16_t d[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    d[q] = 0;
                    if (gj < N && gk + q < kbase + K)
                        d[q] = rademacher_bit(P.seed, P.mode, gk + q, gj) ? (uint16_t)0x3F80 : (uint16_t)0xBF80;
                }
                uint4 v;
                v.x = (uint32_t)d[0] | ((uint32_t)d[1] << 16);
                v.y = (uint32_t)d[2] | ((uint32_t)d[3] << 16);
                v.z = (uint32_t)d[4] | ((uint32_t)d[5] << 16);
                v.w = (uint32_t)d[6] | ((uint32_t)d[7] << 16);
                *reinterpret_cast<uint4*>(sB + oz_off(r, c)) = v;
            }
        }
    };

    // epilogue registers: rows 32 (warp % 4) + lane, columns (warp / 4) NQ .. + NQ
    const int q4 = warp & 3, cg = warp >> 2;
    const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
    float hi[NQ], lo[NQ];
#pragma unroll
    for (int c = 0; c < NQ; ++c) { hi[c] = 0.f; lo[c] = 0.f; }
    auto readback = [&](uint32_t tacc) {
#pragma unroll
        for (int c = 0; c < NQ; c += 8) {
            float v[8];
            tmem_ld8(tacc + lane_base + cg * NQ + c, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) two_sum_acc(hi[c + j], lo[c + j], v[j]);
        }
    };

    // A bounded wait that expires sets s_fail; from then on no thread produces a stage, reads
    // TMEM back or issues an MMA (every thread sees the flag after the next barrier), and the
    // epilogue stores nothing.
    bool ok = true;
    int last_commit = -1;                     // stage whose MMAs were committed last
    if (nkt > 0) produce(0, 0);
    constexpr uint32_t IDESC = oz_idesc(NT);
    for (int kt = 0; kt < nkt; ++kt) {
        const int buf = kt & 1;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (*(volatile int*)&s_fail) break;
        last_commit = kt;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t aBase = smem_u32(oz_smem + buf * STAGE);
            const uint32_t bBase = aBase + SA * A_PLANE;
            // descriptors of the stage's first A and B planes; a plane or K-half at byte offset o
            // (a multiple of 16) is the base descriptor plus o / 16 in the 14-bit address field,
            // which cannot carry: shared addresses stay below 2^18
            const uint64_t dA0 = oz_desc(aBase), dB0 = oz_desc(bBase);
            bool started[NU];
#pragma unroll
            for (int a = 0; a < NU; ++a) started[a] = false;
#pragma unroll
            for (int s = 1; s <= SA; ++s) {
#pragma unroll
                for (int t = 1; t <= SB; ++t) {
                    if (s + t > GMAX) continue;
                    const int a = (s + t - 2) < NE ? (s + t - 2) : NE;
                    const int cad = oz_acc_cad(SA, SB, NE, a, W);
                    // the first MMA of a group after its readback overwrites the accumulator
                    const uint32_t acc = ((kt % cad) != 0 || started[a]) ? 1u : 0u;
                    started[a] = true;
                    const uint32_t tacc = tmem + (uint32_t)(a * NT);
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint64_t da = dA0 + (uint64_t)(((s - 1) * A_PLANE + kk * 256) >> 4);
                        const uint64_t db = dB0 + (uint64_t)(((t - 1) * B_PLANE + kk * 256) >> 4);
                        oz_mma(tacc, da, db, IDESC, kk > 0 ? 1u : acc);
                    }
                }
            }
            oz_commit(&mbar[buf]);
        }
        // produce the next stage into the other buffer once the MMAs that read it are done
        if (kt + 1 < nkt) {
            if (kt >= 1 && !oz_wait(&mbar[buf ^ 1], (uint32_t)(((kt - 1) >> 1) & 1))) {
                ok = false;
                s_fail = 1;
            }
            if (ok) produce(kt + 1, buf ^ 1);
        }
        const bool last = (kt + 1 == nkt);
        if (ok && (last || (kt % MINCAD) == MINCAD - 1)) {      // every cadence is a multiple of MINCAD
            if (!oz_wait(&mbar[buf], (uint32_t)((kt >> 1) & 1))) {
                ok = false;
                s_fail = 1;
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int a = NU - 1; a >= 0; --a) {
                    const int cad = oz_acc_cad(SA, SB, NE, a, W);
                    if (last || (kt % cad) == cad - 1) readback(tmem + (uint32_t)(a * NT));
                }
            }
        }
    }
    __syncthreads();
    const bool failed = *(volatile int*)&s_fail != 0;
    if (failed) {
        // wait (bounded again) for the last committed MMAs before TMEM is freed
        if (last_commit >= 0) oz_wait(&mbar[last_commit & 1], (uint32_t)((last_commit >> 1) & 1));
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) atomicCAS(batch.err ? batch.err : &g_oz_status, 0, RHOSVD_ERR_TIMEOUT);
        if (EPI == OZ_EPI_RESID && tid == 0) P.rpart[blockIdx.x + gridDim.x * blockIdx.y] = 0.0;
        if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
        return;
    }
    const int row = i0 + q4 * 32 + lane;
    int ea = (ASRC == OZ_A_PLANES && P.A.exps && row < M) ? (int)P.A.exps[row] : (ASRC == OZ_A_PLANES ? P.A.exp0 : 0);
    if (ASRC == OZ_A_KR && P.kr.e2 && row < M) ea = (int)P.kr.e2[row % r2] + (int)P.kr.e3[row / r2];
    double e2 = 0.0;
    const long long ccs = P.ccs < 0 ? (long long)M : P.ccs;
    const long long crs = P.crs < 0 ? (long long)N : P.crs;
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
        const int col = j0 + cg * NQ + c;
        if (row >= M || col >= N) continue;
        const int eb = BSRC == OZ_B_PLANES ? (P.B.exps ? (int)P.B.exps[col] : P.B.exp0) : W;
        // x = 2^(E - W) sum_s plane_s, so a product carries 2^(ea + eb - 2W), built from its
        // exponent bits (ea + eb in [-252, 254]: always normal): one exact multiply instead of an
        // ldexp call on the FP64 pipe
        const double sc = __hiloint2double((ea + eb - 2 * W + 1023) << 20, 0);
        const double v = ((double)hi[c] + (double)lo[c]) * sc;
        if (EPI == OZ_EPI_STORE) {
            Cout[(long long)row * crs + (long long)col * ccs] = v;
        } else {
            const double d = P.ref[(long long)row * P.ref_rs + (long long)col * P.ref_cs] - v;
            e2 = fma(d, d, e2);
        }
    }
    if (EPI == OZ_EPI_RESID) {
        e2 = block_sum(e2, red);
        if (tid == 0) P.rpart[blockIdx.x + gridDim.x * blockIdx.y] = e2;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

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

constexpr int OZ_ST_R = 32, OZ_ST_K = 64;

// S as a template argument: the digit loops unroll and the digits stay in registers.
template <int S>
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
    const int tid = threadIdx.x;
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
        const int E = a.exps[b] ? (int)a.exps[b][i] : a.exp0;
        uint16_t d[S];
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
    const long long tiles = ((M + OZ_BM - 1) / OZ_BM) * ((N + 159) / 160);
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
    if (exps) {
        // every problem of one call either has exponents or not (the slicers are per operand)
        for (int b = 0; b < nb; ++b)
            if (!a.exps[b]) return RHOSVD_ERR_INVALID_ARG;
        k_oz_rowexp<<<dim3((rmax + OZ_RE_ROWS - 1) / OZ_RE_ROWS, nb), 256, 0, st>>>(a);
        RH_CHECK_LAUNCH();
    }
    dim3 grid((ldmax + OZ_ST_K - 1) / OZ_ST_K, (rmax + OZ_ST_R - 1) / OZ_ST_R, nb);
    switch (a.S) {
    case OZ_S64: k_oz_slice_tile<OZ_S64><<<grid, 256, 0, st>>>(a); break;
    case 4: k_oz_slice_tile<4><<<grid, 256, 0, st>>>(a); break;
    case 1: k_oz_slice_tile<1><<<grid, 256, 0, st>>>(a); break;
    default: return RHOSVD_ERR_INVALID_ARG;
    }
    RH_CHECK_LAUNCH();
    return 0;
}

template <int SA, int SB, int GMAX, int ASRC, int BSRC, int EPI, int NT, int NACC, int W>
static int run_oz(const OzBatch& b, cudaStream_t st)
{
    int Mh = 0, Nh = 0;
    for (int i = 0; i < b.nbatch; ++i) {
        Mh = max(Mh, b.p[i].M);
        Nh = max(Nh, b.p[i].N);
    }
    if (Mh <= 0 || Nh <= 0) return 0;
    constexpr int STAGE = SA * OZ_BM * OZ_BK * 2 + SB * NT * OZ_BK * 2;
    constexpr int SMEM = 2 * STAGE;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_ozgemm<SA, SB, GMAX, ASRC, BSRC, EPI, NT, NACC, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SMEM) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
        attr = true;
    }
    const int nsplit = b.nsplit > 1 ? b.nsplit : 1;
    if (nsplit > 1 && EPI != OZ_EPI_STORE) return RHOSVD_ERR_INVALID_ARG;
    dim3 grid((Mh + OZ_BM - 1) / OZ_BM, (Nh + NT - 1) / NT, b.nbatch * nsplit);
    k_ozgemm<SA, SB, GMAX, ASRC, BSRC, EPI, NT, NACC, W><<<grid, OZ_THREADS, SMEM, st>>>(b);
    RH_CHECK_LAUNCH();
    if (nsplit > 1) {
        const long long mn = (long long)Mh * Nh;
        dim3 rg((unsigned)((mn + 255) / 256 < 4096 ? (mn + 255) / 256 : 4096), b.nbatch);
        k_oz_reduce<<<rg, 256, 0, st>>>(b);
        RH_CHECK_LAUNCH();
    }
    return 0;
}

int launch_ozgemm(const OzBatch& b, OzKind kind, cudaStream_t st)
{
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
    for (int i = 0; i < b.nbatch; ++i)
        if (b.p[i].A.tiles_k > 0 || b.p[i].B.tiles_k > 0) return RHOSVD_ERR_INVALID_ARG;   // TMA path only
    switch (kind) {
    case OZ_F64_STORE:
        return run_oz<OZ_S64, OZ_S64, 9, OZ_A_PLANES, OZ_B_PLANES, OZ_EPI_STORE, OZ_NT6, 8, OZ_W64>(b, st);
    case OZ_F64_RESID:
        return run_oz<OZ_S64, OZ_S64, 9, OZ_A_PLANES, OZ_B_PLANES, OZ_EPI_RESID, OZ_NT6, 8, OZ_W64>(b, st);
    case OZ_SKETCH: return run_oz<OZ_S64, 1, 8, OZ_A_PLANES, OZ_B_SIGN, OZ_EPI_STORE, 96, 5, OZ_W64>(b, st);
    case OZ_CORE: return run_oz<4, 4, 5, OZ_A_KR, OZ_B_PLANES, OZ_EPI_STORE, 160, 3, 8>(b, st);
    case OZ_BF16: return run_oz<1, 1, 2, OZ_A_PLANES, OZ_B_PLANES, OZ_EPI_STORE, 128, 1, 8>(b, st);
    }
    return RHOSVD_ERR_INVALID_ARG;
}

}  // namespace rh
