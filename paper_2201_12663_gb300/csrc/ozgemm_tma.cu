// ozgemm_tma.cu -- the digit-plane tcgen05 GEMM (arithmetic in ozgemm.cuh) as a warp-specialised
// pipeline fed by the Tensor Memory Accelerator.
//
// One CTA computes a 128 x NT tile of C.  K advances in stages of 16 (one tcgen05.mma K step)
// through a ring of STAGES shared-memory buffers.  Warp roles:
//   warp 0     producer: lane 0 loads every digit plane of the stage's A and B tiles onto the
//              stage's "full" mbarrier: tile-major planes by cp.async.bulk (one contiguous block),
//              row-major planes by cp.async.bulk.tensor (2D tensor maps over this GPU's memory, no
//              multicast);
//   warp 1     MMA issuer: lane 0 waits for a full stage, issues one tcgen05.mma (kind::f16, BF16
//              digits, FP32 accumulation in TMEM) per digit pair (s, t) with s + t <= GMAX into
//              the accumulator of group g = s + t, and commits the stage's "empty" barrier;
//   warps 2-9  epilogue: read accumulators back into double-float registers (tcgen05.ld) when
//              their exactness cadence requires it, then store C or the residual energy.
// Tiles are K-major with the 32-byte swizzle (8-row x 32-byte atoms, 256 B between 8-row groups),
// the layout TMA writes with CU_TENSOR_MAP_SWIZZLE_32B and the MMA descriptors read.
//
// Accumulators (Plan<KIND>): each digit group g = s + t, or a few of them together, has an FP32
// accumulator in TMEM that is read back into double-float registers every cad stages, before its
// sum could round (or, for the merged small F64 groups, while its rounding stays near 2^-48 of
// the product's scale).  The readbacks of different accumulators fall on different stages, and
// TMEM holds spare slots: an accumulator that is being read back moves to a free slot for the next
// stage, so the MMA issuer never waits for the epilogue unless both are behind by a whole FIFO of
// spare slots.  Both sides run the same deterministic slot allocator (SlotSim).
//
// Every mbarrier wait is bounded.  On expiry the CTA stops producing, issuing and reading back,
// waits (bounded again) for its own copies and MMAs in flight, records RHOSVD_ERR_TIMEOUT in the
// batch's status word (or the library's, see oz_take_status), frees TMEM and returns.
#include "ozgemm.cuh"
#include <cuda.h>
#include <mutex>

namespace rh {

// status word of this file's products launched without a caller status (see oz_take_status)
__device__ int g_oztma_status = 0;

int oztma_take_status(cudaStream_t st, int* out)
{
    int v = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_oztma_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RHOSVD_ERR_CUDA;
    if (v != 0) {
        const int zero = 0;
        if (cudaMemcpyToSymbolAsync(g_oztma_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
    }
    *out = v;
    return RHOSVD_OK;
}

namespace {

constexpr int TK = 16;                  // K per stage
constexpr int T_WARPS = 10;
constexpr int T_THREADS = 32 * T_WARPS;
constexpr int T_EPI0 = 2;               // first epilogue warp
constexpr int T_NEPI = 8;               // epilogue warps: two per TMEM lane quarter
constexpr int T_SMEM_MAX = 227 * 1024;

struct OzMaps {
    CUtensorMap a[3];
    CUtensorMap b[3];
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, 32-byte swizzle: start address, LBO unused (16 B), SBO = 256 B, version 1, layout 6
__device__ __forceinline__ uint64_t desc_sw32(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(256 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)6 << 61;
    return d;
}

__host__ __device__ constexpr uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(su32(b)),
                 "r"(bytes) : "memory");
}

// bounded wait for the phase of the given parity; false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity)
{
    uint32_t done = 0;
    for (long it = 0; it < (1L << 24) && !done; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done) : "r"(su32(b)), "r"(parity) : "memory");
    }
    return done != 0;
}

// the same with a short sleep between polls, for waits that are usually long
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* b, uint32_t parity)
{
    uint32_t done = 0;
    for (long it = 0; it < (1L << 22) && !done; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done) : "r"(su32(b)), "r"(parity) : "memory");
        if (!done) __nanosleep(128);
    }
    return done != 0;
}

__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
                 : "memory");
}

// one contiguous global -> shared copy onto an mbarrier (16-byte aligned, a multiple of 16 bytes)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                 "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float* v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void two_sum(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    const float l = lo + err;
    hi = s + l;
    lo = l - (hi - s);
}

__host__ __device__ constexpr int npairs(int SA, int SB, int g)
{
    int c = 0;
    for (int s = 1; s <= SA; ++s)
        if (g - s >= 1 && g - s <= SB) ++c;
    return c;
}

// Plans.  The CTA tile is 128 rows of the "lane" operand (on the TMEM lanes) by NT rows of the
// "col" operand.  Each stage issues one MMA per digit plane s of the lane operand, against the
// col operand's planes t = 1 .. T(s) stacked along N, into the consecutive TMEM columns of the
// groups g = s + 1 .. s + T(s) (group g at NT (g - 2)): the MMA's N is NT T(s), up to 256, so a
// stage costs SL instructions instead of one per digit pair.  The first MMA of a block (s = 1)
// spans every group's columns (a zero plane fills the stack where needed) and overwrites them.
// Two accumulator buffers of NG NT columns alternate by blocks of RBK stages: the MMAs of block
// b + 1 run while the epilogue reads block b back into double-float registers.
//   TK_F64  (7 x 7 digits of 7 bits, pairs s + t <= 9): lane = A, col = B, NT = 32, 8 groups;
//           a group of np <= 7 pairs sums np 2^14 16 RBK <= 2^24 over a block of 8 stages, so
//           every group is exact until it is read back.
//   TK_SIGN (the range sketch, 7 digits of U~ against +-1): lane = the sign plane (the problem's
//           B, tile-major, 128 sketch columns, written once per sketch by k_sign_planes), col =
//           the U~ planes (the problem's A, tile-major, 32 rows of x), one MMA of N = 224 a
//           stage, 7 exact groups of one pair each.
//   TK_BF16 (one plane of arbitrary BF16 values): lane = A, col = B, NT = 64, one group.
enum TmaKind { TK_F64 = 0, TK_SIGN = 1, TK_BF16 = 2 };

template <int KIND>
struct Plan {
    static constexpr int SL = KIND == TK_F64 ? OZ_S64 : 1;
    static constexpr int SC = KIND == TK_BF16 ? 1 : OZ_S64;
    static constexpr int NT = KIND == TK_BF16 ? 64 : 32;
    static constexpr int GMAX = KIND == TK_F64 ? 9 : (KIND == TK_SIGN ? 8 : 2);
    static constexpr int W = KIND == TK_BF16 ? 8 : OZ_W64;
    static constexpr int NG = GMAX - 1;
    static constexpr int ZP = NG > SC ? NG - SC : 0;     // zero planes after the stacked ones
    static constexpr int NCOL = NG * NT;
    static constexpr int RBK = KIND == TK_F64 ? 8 : 16;
    static constexpr int T(int s) { return s == 1 ? NG : (SC < GMAX - s ? SC : GMAX - s); }
    static constexpr bool ok()
    {
        bool good = 2 * NCOL <= 512 && NT * T(1) <= 256;
        for (int g = 2; g <= GMAX && KIND != TK_BF16; ++g)
            good = good && (long long)npairs(SL, SC, g) * (1 << (2 * W)) * 16 * RBK <= (1 << 24);
        return good;
    }
};

__device__ __forceinline__ int dimv(const int* d, int h) { return d ? *d : h; }

}  // namespace

template <int KIND, int EPI, int STAGES>
__global__ void __launch_bounds__(T_THREADS, 1) k_oztma(OzBatch batch, const __grid_constant__ OzMaps maps)
{
    using PL = Plan<KIND>;
    constexpr int SL = PL::SL, SC = PL::SC, NT = PL::NT, W = PL::W, NG = PL::NG, NCOL = PL::NCOL, RBK = PL::RBK;
    constexpr bool SIGN = KIND == TK_SIGN;
    constexpr int L_PLANE = OZ_BM * TK * 2;              // 4096 B: 128 rows x 32 B
    constexpr int C_PLANE = NT * TK * 2;
    constexpr int L_BYTES = SL * L_PLANE;
    constexpr int C_BYTES = (SC + PL::ZP) * C_PLANE;
    constexpr int STAGE = (L_BYTES + C_BYTES + 1023) / 1024 * 1024;
    constexpr int NC = NT / 2;                            // columns per epilogue warp
    constexpr uint32_t TX_BYTES = L_BYTES + SC * C_PLANE;
    static_assert(PL::ok(), "plan: TMEM, MMA width or exactness");
    static_assert(NC % 16 == 0, "16-column TMEM loads");
    static_assert(STAGES * STAGE + 2048 <= T_SMEM_MAX, "shared memory");

    const int nsplit_h = batch.nsplit > 1 ? batch.nsplit : 1;
    const int split = blockIdx.z % nsplit_h;
    const int pb = blockIdx.z / nsplit_h;
    const OzProblem& P = batch.p[pb];
    const int nsplit = P.dsplit ? max(1, min(*P.dsplit, nsplit_h)) : nsplit_h;
    if (split >= nsplit) return;
    const int M = dimv(P.dM, P.M);
    const int N = dimv(P.dN, P.N);
    const int Kall = dimv(P.dK, P.K);
    // this CTA's K range [kbase, kbase + K): whole 32-wide blocks, the last split takes the rest
    const int kspan = ((Kall + nsplit - 1) / nsplit + OZ_BK - 1) / OZ_BK * OZ_BK;
    const int kbase = min(Kall, split * kspan);
    const int K = min(Kall, kbase + kspan) - kbase;
    double* const Cout = nsplit > 1 ? P.Cpart + split * P.split_stride : P.C;
    // lane tile (128 rows) and col tile (NT rows); the sketch puts its sign operand (problem
    // columns) on the lanes and the planes of U~ (problem rows) on the stacked side
    const int i0 = blockIdx.x * OZ_BM, j0 = blockIdx.y * NT;
    const int laneExt = SIGN ? N : M, colExt = SIGN ? M : N;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (i0 >= laneExt || j0 >= colExt) {
        if (EPI == OZ_EPI_RESID && tid == 0) P.rpart[blockIdx.x + gridDim.x * blockIdx.y] = 0.0;
        return;
    }
    const int nkt = (K + TK - 1) / TK;
    const int nblk = (nkt + RBK - 1) / RBK;
    const OzPlanes& LP = SIGN ? P.B : P.A;               // lane operand planes (the signs for SIGN)
    const OzPlanes& CP = SIGN ? P.A : P.B;               // col operand planes
    const int rowsL = LP.pstride > 0 ? (int)(LP.pstride / LP.ld) : 0;
    const int rowsC = CP.pstride > 0 ? (int)(CP.pstride / CP.ld) : 0;

    extern __shared__ __align__(1024) unsigned char tsm[];
    unsigned char* stages = (unsigned char*)(((uintptr_t)tsm + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], buf_full[2], buf_free[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    __shared__ double red[T_NEPI];

    // the zero planes of every stage (never written by the copies)
    if (PL::ZP > 0) {
        for (int s = 0; s < STAGES; ++s) {
            uint32_t* z = (uint32_t*)(stages + s * STAGE + L_BYTES + SC * C_PLANE);
            for (int e = tid; e < PL::ZP * C_PLANE / 4; e += T_THREADS) z[e] = 0u;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::);
    }
    if (tid == 32) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&buf_full[b], 1);
            mbar_init(&buf_free[b], T_NEPI);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    volatile int* fail = &s_fail;

    if (warp == 0) {
        // ---------------------------------------------------------------- producer
        // lane 0 waits and decides; the decision is broadcast so that the warp stays converged
        int issued = 0;                     // stages whose loads were issued
        for (int kt = 0; kt < nkt; ++kt) {
            const int s = kt % STAGES;
            int go = 0;
            if (lane == 0) {
                go = *fail ? 0 : 1;
                if (go && kt >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((kt / STAGES) - 1) & 1))) {
                    *fail = 1;
                    go = 0;
                }
            }
            if (!__shfl_sync(0xffffffffu, go, 0)) break;
            unsigned char* sL = stages + s * STAGE;
            unsigned char* sC = sL + L_BYTES;
            const int k0 = kbase + kt * TK;
            if (lane == 0) {
                mbar_expect_tx(&full[s], TX_BYTES);
                if (LP.tiles_k > 0) {
                    // tile-major lane operand: the stage's SL plane tiles are one contiguous block
                    const uint16_t* src = LP.base + ((long long)(i0 >> 7) * LP.tiles_k + (k0 >> 4)) * SL * 2048;
                    bulk_g2s(sL, src, L_BYTES, &full[s]);
                } else {
#pragma unroll
                    for (int p = 0; p < SL; ++p) tma_2d(sL + p * L_PLANE, &maps.a[pb], k0, p * rowsL + i0, &full[s]);
                }
                if (CP.tiles_k > 0) {
                    // tile-major col operand (NT-row tiles): the stage's SC plane tiles, one block
                    const uint16_t* src = CP.base + ((long long)(j0 / NT) * CP.tiles_k + (k0 >> 4)) * SC * (NT * 16);
                    bulk_g2s(sC, src, SC * C_PLANE, &full[s]);
                } else {
#pragma unroll
                    for (int p = 0; p < SC; ++p) tma_2d(sC + p * C_PLANE, &maps.b[pb], k0, p * rowsC + j0, &full[s]);
                }
            }
            __syncwarp();
            issued = kt + 1;
        }
        if (*fail && lane == 0) {
            // copies in flight land before the CTA's shared memory goes away
            for (int kt = max(0, issued - STAGES); kt < issued; ++kt)
                mbar_wait(&full[kt % STAGES], (uint32_t)((kt / STAGES) & 1));
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int last = -1;
            for (int kt = 0; kt < nkt; ++kt) {
                if (*fail) break;
                const int s = kt % STAGES;
                const int blk = kt / RBK;
                const bool first = kt % RBK == 0;
                const uint32_t buf = tmem + (uint32_t)((blk & 1) * NCOL);
                // the block's buffer was read back by the epilogue two blocks ago
                if (first && blk >= 2 && !mbar_wait(&buf_free[blk & 1], (uint32_t)(((blk >> 1) - 1) & 1))) {
                    *fail = 1;
                    break;
                }
                if (!mbar_wait(&full[s], (uint32_t)((kt / STAGES) & 1))) {
                    *fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t lBase = su32(stages + s * STAGE);
                const uint64_t dL0 = desc_sw32(lBase), dC0 = desc_sw32(lBase + L_BYTES);
#pragma unroll
                for (int sp = 1; sp <= SL; ++sp) {
                    const uint32_t idesc = idesc_bf16(NT * PL::T(sp));
                    mma_f16(buf + (uint32_t)(NT * (sp - 1)), dL0 + (uint64_t)(((sp - 1) * L_PLANE) >> 4), dC0, idesc,
                            (first && sp == 1) ? 0u : 1u);
                }
                mma_commit(&empty[s]);          // also tracks this stage's MMAs for the failure path
                last = kt;
                if (kt % RBK == RBK - 1 || kt + 1 == nkt) mma_commit(&buf_full[blk & 1]);
            }
            if (*fail && last >= 0) mbar_wait(&empty[last % STAGES], (uint32_t)((last / STAGES) & 1));
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- epilogue
        const int e = warp - T_EPI0;
        const int q = warp & 3;                  // TMEM lane quarter of this warp
        const int hcol = e >> 2;                 // which half of the NT columns
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        float hi[NC], lo[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) { hi[c] = 0.f; lo[c] = 0.f; }
        for (int blk = 0; blk < nblk; ++blk) {
            // lane 0 waits and decides for the warp (tcgen05.ld needs the whole warp converged)
            int go = 0;
            if (lane == 0) {
                go = *fail ? 0 : 1;
                if (go && !mbar_wait_sleep(&buf_full[blk & 1], (uint32_t)((blk >> 1) & 1))) {
                    *fail = 1;
                    go = 0;
                }
            }
            if (!__shfl_sync(0xffffffffu, go, 0)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t buf = tmem + lane_base + (uint32_t)((blk & 1) * NCOL + hcol * NC);
#pragma unroll
            for (int g = 0; g < NG; ++g) {
#pragma unroll
                for (int c = 0; c < NC; c += 16) {
                    float v[16];
                    tmem_ld16(buf + (uint32_t)(g * NT + c), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) two_sum(hi[c + j], lo[c + j], v[j]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0 && blk + 2 < nblk) mbar_arrive(&buf_free[blk & 1]);
        }
        // the epilogue warps decide together: a failure anywhere has been recorded before the
        // last readback could complete, so after this barrier the flag no longer changes
        asm volatile("bar.sync 1, %0;" ::"r"(T_NEPI * 32) : "memory");
        if (!*fail) {
            const int lrow = i0 + q * 32 + lane;                      // lane operand row
            const long long ccs = P.ccs < 0 ? (long long)M : P.ccs;
            const long long crs = P.crs < 0 ? (long long)N : P.crs;
            double e2 = 0.0;
            float e2f = 0.f;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int ccol = j0 + hcol * NC + c;                  // col operand row
                const int row = SIGN ? ccol : lrow, col = SIGN ? lrow : ccol;
                if (row >= M || col >= N) continue;
                const int ea = P.A.exps ? (int)P.A.exps[row] : P.A.exp0;
                const int eb = SIGN ? W : (P.B.exps ? (int)P.B.exps[col] : P.B.exp0);
                // x = 2^(E - W) sum_s plane_s: a product carries 2^(ea + eb - 2W), built from its bits
                const double sc = __hiloint2double((ea + eb - 2 * W + 1023) << 20, 0);
                if (EPI == OZ_EPI_STORE) {
                    Cout[(long long)row * crs + (long long)col * ccs] = ((double)hi[c] + (double)lo[c]) * sc;
                } else {
                    // ref - (hi + lo) sc: the cancelling part ref - hi sc in one FP64 fma (exact
                    // scaling, one rounding), the small remainder and its square in FP32 (the
                    // residual's entries are far below ref's, so FP32 keeps them to 2^-24 of
                    // themselves; a scale below FP32's range only drops a term below 2^-126)
                    const double t = fma(-(double)hi[c], sc, P.ref[(long long)row * P.ref_rs + (long long)col * P.ref_cs]);
                    const float d = __double2float_rn(t) - lo[c] * __double2float_rn(sc);
                    e2f = fmaf(d, d, e2f);
                }
            }
            if (EPI == OZ_EPI_RESID) {
                e2 = warp_sum((double)e2f);
                if (lane == 0) red[e] = e2;
                asm volatile("bar.sync 1, %0;" ::"r"(T_NEPI * 32) : "memory");
                if (e == 0 && lane == 0) {
                    double t = 0.0;
#pragma unroll
                    for (int w = 0; w < T_NEPI; ++w) t += red[w];
                    P.rpart[blockIdx.x + gridDim.x * blockIdx.y] = t;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*fail) {
        if (tid == 0) atomicCAS(batch.err ? batch.err : &g_oztma_status, 0, RHOSVD_ERR_TIMEOUT);
        if (EPI == OZ_EPI_RESID && tid == 0) P.rpart[blockIdx.x + gridDim.x * blockIdx.y] = 0.0;
    }
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// 2D map over S planes of `rows` rows each (ld elements a row, bf16 patterns): dims {ld, S rows},
// box {16, box_rows}, 32-byte swizzle, zero fill outside
bool plane_map(CUtensorMap* m, const OzPlanes& pl, int S, int rows, int box_rows)
{
    EncodeTiledFn enc = encoder();
    if (!enc || !pl.base || pl.ld <= 0 || pl.ld % 8 != 0 || rows <= 0) return false;
    if (((uintptr_t)pl.base) % 16 != 0) return false;
    if (S > 1 && pl.pstride != (long long)rows * pl.ld) return false;
    cuuint64_t dims[2] = {(cuuint64_t)pl.ld, (cuuint64_t)S * (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pl.ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, (void*)pl.base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KIND, int EPI>
int run_tma(const OzBatch& b, cudaStream_t st)
{
    using PL = Plan<KIND>;
    constexpr bool SIGN = KIND == TK_SIGN;
    constexpr int L_BYTES = PL::SL * OZ_BM * TK * 2, C_PLANE = PL::NT * TK * 2;
    constexpr int STAGE = (L_BYTES + (PL::SC + PL::ZP) * C_PLANE + 1023) / 1024 * 1024;
    constexpr int ST_FIT = (T_SMEM_MAX - 4096) / STAGE;
    constexpr int STAGES = ST_FIT > 8 ? 8 : ST_FIT;
    static_assert(STAGES >= 2, "two stages at least");
    constexpr int SMEM = STAGES * STAGE + 1024;
    int Mh = 0, Nh = 0;
    for (int i = 0; i < b.nbatch; ++i) {
        Mh = max(Mh, b.p[i].M);
        Nh = max(Nh, b.p[i].N);
    }
    if (Mh <= 0 || Nh <= 0) return 0;
    OzMaps maps;
    memset(&maps, 0, sizeof(maps));
    for (int i = 0; i < b.nbatch; ++i) {
        const OzProblem& q = b.p[i];
        if (!SIGN && q.A.tiles_k <= 0) {
            const int ra = q.A.pstride > 0 ? (int)(q.A.pstride / (q.A.ld > 0 ? q.A.ld : 1)) : q.M;
            if (!plane_map(&maps.a[i], q.A, PL::SL, ra, OZ_BM)) return RHOSVD_ERR_INVALID_ARG;
        }
        const OzPlanes& cp = SIGN ? q.A : q.B;
        if (cp.tiles_k <= 0) {
            const int rc = cp.pstride > 0 ? (int)(cp.pstride / (cp.ld > 0 ? cp.ld : 1)) : (SIGN ? q.M : q.N);
            if (!plane_map(&maps.b[i], cp, PL::SC, rc, PL::NT)) return RHOSVD_ERR_INVALID_ARG;
        }
    }
    auto kern = k_oztma<KIND, EPI, STAGES>;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
        attr = true;
    }
    const int nsplit = b.nsplit > 1 ? b.nsplit : 1;
    if (nsplit > 1 && EPI != OZ_EPI_STORE) return RHOSVD_ERR_INVALID_ARG;
    const int laneExt = SIGN ? Nh : Mh, colExt = SIGN ? Mh : Nh;
    dim3 grid((laneExt + OZ_BM - 1) / OZ_BM, (colExt + PL::NT - 1) / PL::NT, b.nbatch * nsplit);
    kern<<<grid, T_THREADS, SMEM, st>>>(b, maps);
    RH_CHECK_LAUNCH();
    return 0;
}

}  // namespace

bool ozgemm_tma_supports(const OzBatch& b, OzKind kind)
{
    if (kind != OZ_F64_STORE && kind != OZ_F64_RESID && kind != OZ_SKETCH && kind != OZ_BF16) return false;
    if (!encoder()) return false;
    const int S = kind == OZ_BF16 ? 1 : OZ_S64;
    const int nt = kind == OZ_BF16 ? Plan<TK_BF16>::NT : Plan<TK_F64>::NT;
    for (int i = 0; i < b.nbatch; ++i) {
        const OzProblem& q = b.p[i];
        // the operand on the TMEM lanes and the one stacked along N (the sketch swaps them)
        const OzPlanes* ops[2] = {kind == OZ_SKETCH ? &q.B : &q.A, kind == OZ_SKETCH ? &q.A : &q.B};
        for (int o = 0; o < 2; ++o) {
            const OzPlanes& pl = *ops[o];
            if (!pl.base || ((uintptr_t)pl.base) % 16 != 0) return false;
            if (pl.tiles_k > 0) {
                if (pl.tile_h != (o == 0 ? OZ_BM : nt)) return false;
                continue;
            }
            if (kind == OZ_SKETCH) return false;       // the sketch reads tile-major planes of U~ and signs
            if (pl.ld <= 0 || pl.ld % 8 != 0) return false;
            if (S > 1 && (pl.pstride <= 0 || pl.pstride % pl.ld != 0)) return false;
        }
    }
    return true;
}

// the residual partials one launch writes per problem (tiles of its grid)
long long ozgemm_tma_tiles(OzKind kind, int M, int N)
{
    const int nt = kind == OZ_BF16 ? Plan<TK_BF16>::NT : Plan<TK_F64>::NT;
    if (kind == OZ_SKETCH) return (long long)((N + OZ_BM - 1) / OZ_BM) * ((M + Plan<TK_SIGN>::NT - 1) / Plan<TK_SIGN>::NT);
    return (long long)((M + OZ_BM - 1) / OZ_BM) * ((N + nt - 1) / nt);
}

int launch_ozgemm_tma(const OzBatch& b, OzKind kind, cudaStream_t st)
{
    switch (kind) {
    case OZ_F64_STORE: return run_tma<TK_F64, OZ_EPI_STORE>(b, st);
    case OZ_F64_RESID: return run_tma<TK_F64, OZ_EPI_RESID>(b, st);
    case OZ_SKETCH: return run_tma<TK_SIGN, OZ_EPI_STORE>(b, st);
    case OZ_BF16: return run_tma<TK_BF16, OZ_EPI_STORE>(b, st);
    default: return RHOSVD_ERR_INVALID_ARG;
    }
}

}  // namespace rh
